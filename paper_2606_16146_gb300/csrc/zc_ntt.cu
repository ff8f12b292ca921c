// zc_ntt.cu -- NTT-form ZeroCheck prover (Fig. side-by-side-zc, left).
#include "zc_internal.cuh"

namespace zc {

zc_status ntt_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                    const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                    bool proof_on_dev, void* q_out, int q_on_dev) {
  ctx->err = "NTT form not built yet";
  return ZC_ERR_UNSUPPORTED;
}

}  // namespace zc
