// zc_internal.cuh -- context, constants and helpers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/zc.h"
#include "zc_field.cuh"
#include "zc_sha256.cuh"

namespace zc {

constexpr int kMaxDeg = 64;      // product gate degree limit
constexpr int kMaxCols = kMaxDeg + 1;
constexpr int kMaxN = 28;        // log2 of the largest column
constexpr int kMaxPts = kMaxDeg + 2;

// Field constants in device memory (one copy per context), all as raw limbs.
// "lvl k" = the value times R^k mod r.
struct DevConst {
  fr one;              // R mod r              (1 at level 1)
  fr r2;               // R^2 mod r            (to level 1: M(x, r2))
  fr rpow[kMaxDeg + 2];   // rpow[k] = R^k mod r (canonical numbers), k = 0..65
  fr rnegpow[kMaxDeg + 2];// R^-k mod r (canonical numbers)
  fr small[kMaxPts + 2];  // t at level 1, t = 0..67
  // Extrapolation of a degree-d polynomial known at 0..d-1 plus its leading
  // coefficient: H(t) = lead * pinf[t] + sum_s H(s) lext[t][s], t = d, d+1.
  // Stored per degree: ext_base[d] indexes into ext_tab.
  // Lagrange denominators 1 / prod_{s' != s} (s - s') over nodes 0..d.
  uint32_t ext_base[kMaxDeg + 1];
  uint32_t lag_base[kMaxDeg + 1];
};

// Per-degree tables live in a separate device array (variable length).
// Layout for degree d at ext_base[d]: [pinf(d), pinf(d+1), lext(d)[0..d-1],
// lext(d+1)[0..d-1]] (level 1); at lag_base[d]: dinv[0..d] (level 1).

struct ScState {        // SumCheck per-proof device state
  uint32_t S[8];         // transcript chaining value (SHA-256 words)
  fr r[kMaxN];           // eq point, level 1
  fr rinv[kMaxN];        // 1/r_i  (level 1), or 0
  fr r1inv[kMaxN];       // 1/(1 - r_i) (level 1), or 0
  uint32_t p0[kMaxN];    // the finite point computed besides 2..d-1: 0 or 1
  fr alpha[kMaxN];       // challenges, level 1
  fr claim;              // H_{i-1}(alpha_{i-1}), level 0
  fr ci;                 // prod_{j<i} eq(alpha_j, r_j), level 1
  uint32_t counter[kMaxN];  // CTAs that finished round i (last one runs the challenge)
  uint32_t err;          // bit 0: a column value >= r; bit 1: a bounded device wait gave up
  uint32_t go;           // persistent round kernel: rounds whose challenge is out
  uint32_t pad[6];
};

struct NttState {       // NTT per-proof device state
  uint32_t S[8];
  fr z;                  // level 1
  fr zpow_n;             // z^N level 1
  uint32_t err;
  uint32_t pad[7];
};

struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  void reset() { used = 0; }
  template <class T>
  T* take(size_t count, size_t align = 256) {
    size_t off = (used + align - 1) / align * align;
    size_t bytes = count * sizeof(T);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
};

}  // namespace zc

struct zc_ctx {
  int device = 0;
  uint32_t max_n = 0, max_d = 0;
  uint64_t budget = 0;
  int sm_count = 0;
  std::mutex mu;
  std::string err;
  zc::DevConst hconst;           // host copy
  zc::DevConst* dconst = nullptr; // device copy
  zc::fr* dtabs = nullptr;        // per-degree tables (device)
  std::vector<zc::fr> htabs;      // host copy
  zc::Arena arena;               // per-call scratch
  bool arena_borrowed = false;   // arena is a block of the serving pool (not freed here)
  void* pinned = nullptr;        // small pinned staging buffer
  size_t pinned_cap = 0;
  cudaEvent_t ev[8] = {};
  int nev = 0;                   // events recorded by the last prove call
  uint32_t launches = 0;         // kernels launched by the last prove call
  double dom_mulmods = 0;        // algorithmic work of the dominant kernel launch
  double dom_bytes = 0;
  int dom_a = 2, dom_b = 3;      // events bracketing that launch
  int skip_point = 0;            // 0: derive H(1) from the claim (default), 1: derive H(0)
  uint32_t cur_n = 0;            // n of the proof being enqueued (selects tuned launch shapes)
  // launch parameters set by zc_tune_set: [form - 1][n][key - 1], 0 = unset;
  // n = 0 holds the value for sizes without their own entry
  int32_t tune[2][zc::kMaxN + 1][12] = {};
  int32_t tuned(zc_form form, uint32_t n, zc_tune_key key) const {
    const int f = (int)form - 1, k = (int)key - 1;
    if (f < 0 || f > 1 || k < 0 || k > 11) return 0;
    if (n <= (uint32_t)zc::kMaxN && tune[f][n][k]) return tune[f][n][k];
    return tune[f][0][k];
  }
  // per-size NTT tables (twiddles, coset factors, quotient scale), built on
  // first use of a size; see zc_ntt.cu
  struct NttSizeTables {
    uint32_t n = 0, lb = 0, l1 = 0;
    void* mem = nullptr;
    size_t bytes = 0;
    uint64_t stamp = 0;
    zc::fr *tw_fwd = nullptr, *tw_inv = nullptr, *coset = nullptr, *outer = nullptr, *fin = nullptr;
    zc::fr* zinv = nullptr;  // per slice: (7^N w_s^j - 1)^-1 M^-1, level 1
    // step-radix domain 2^lb N + N (built on first use): the small part's
    // coset factors sigma^k / N (level 2) and sigma^-k 7^k (level 1),
    // k < N, sigma = 7 w_{2M}; constants: [0] the small part's z_H inverse
    // times kappa^-1 N^-1, [1] 7^M (level 1), [8 + m] sigma^(mN) kappa^-1,
    // m < 2^lb (level 1), kappa = sigma^M - 7^M.
    void* step_mem = nullptr;
    size_t step_bytes = 0;
    zc::fr *step_coset = nullptr, *step_unscale = nullptr, *step_const = nullptr;
  };
  std::vector<NttSizeTables> ntt_cache;
  uint64_t ntt_cache_clock = 0;
  size_t ntt_cache_budget = 16ull << 30;
  // While a prepared batch is being enqueued (possibly under graph capture)
  // the cache neither allocates nor evicts; a missing size falls back to the
  // two-level power tables.
  bool ntt_cache_frozen = false;
  zc_ctx* table_owner = nullptr;    // lanes use their parent's per-size tables
  bool owns_const = true;           // lanes share the parent's constants
  // batch lanes: child contexts with their own scratch arena and stream
  std::vector<zc_ctx*> lanes;
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_join;
  cudaEvent_t fork_ev = nullptr;
  // pipelined uploads of host columns (NTT form)
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_fork = nullptr;
  std::vector<cudaEvent_t> up_ev;
  // serving: one device pool that in-flight proofs take their scratch from
  void* serve_pool = nullptr;
  size_t serve_pool_cap = 0;
};

namespace zc {

// status helpers
#define ZC_CUDA_TRY(ctx, call)                                                       \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return ZC_ERR_CUDA;                                                            \
    }                                                                                \
  } while (0)

int gate_ncols(uint32_t gate, uint32_t d);
zc_status check_params(zc_ctx* ctx, const zc_params* p, zc_form form);
zc_status ensure_arena(zc_ctx* ctx, size_t bytes);
size_t align_up(size_t x, size_t a);

// host field helpers (generic arithmetic)
fr h_canon_mul(const fr& a, const fr& b, const DevConst& C);  // a*b mod r, canonical
fr h_pow(const fr& a, uint64_t e, const DevConst& C);          // canonical
fr h_inv(const fr& a, const DevConst& C);                      // canonical, a != 0
fr h_from_u64(uint64_t x);
fr h_root_of_unity(uint32_t logn, const DevConst& C);        // canonical generator of the 2^logn subgroup
const DevConst& host_constants();                            // the field constants, built once
void h_to_bytes(const fr& a, uint8_t* out);
bool h_from_bytes(const uint8_t* in, fr* out);
void transcript_init_words(uint32_t S[8], uint32_t form, uint32_t gate, uint32_t n, uint32_t d,
                           uint32_t logm);

// The NTT form's domain (Sec. 3.2; Sec. 4 "Degree scaling"): the big part
// 7 <w_Mb>, Mb = 2^k N, and for a step-radix domain the small part
// sigma <w_Ms>, Ms = 2^s N, s < k, sigma = 7 w_{2 Mb}; M = Mb + Ms points.
// word is what the proof header and the transcript carry: log2 Mb, or
// log2 Mb | (log2 Ms + 1) << 8.
struct NttDomain {
  uint32_t k = 0, s = 0;
  bool step = false;
  uint64_t N = 0, Mb = 0, Ms = 0, M = 0;
  uint32_t word = 0;
};
// From zc_params.log_blowup (0: 2^ceil(log2 d) N; k; or k | (s + 1) << 8);
// false when the word is malformed or the domain cannot hold the quotient.
bool ntt_domain(uint32_t n, uint32_t d, uint32_t log_blowup, NttDomain* D);

// device roots: cols (device pointers), c columns of L elements -> roots
// (device, c x 32 bytes).  Uses arena scratch.
zc_status launch_roots(zc_ctx* ctx, const fr* const* dcols, int c, uint64_t L, uint8_t* droots,
                       cudaStream_t st);
size_t root_scratch_bytes(int c, uint64_t L);
// hash-based commitment: rate-1/4 Reed-Solomon encoding of the 2^nr rows of
// 2^nc entries of each column into enc[j][k m + i] (W = 2^(nc+2)), and the
// column digests, leaves and tree levels (2W - 1 nodes of 8 words, leaves
// first) of the encoded columns
zc_status pcs_encode(zc_ctx* ctx, const fr* const* cols, int c, uint32_t nr, uint32_t nc, fr* const* enc,
                     fr* tab, cudaStream_t st);
zc_status pcs_hash_tree(zc_ctx* ctx, const fr* const* enc, int c, uint64_t m, uint64_t W, uint32_t* dig,
                        uint32_t* tree, cudaStream_t st);
void static_constants(DevConst* C, std::vector<fr>* tabs);

// v2: the eq-factored form (rounds carry H_i(0..d), transcript v2)
// The context's side stream for host-to-device copies and at least n events
// on it (created on first use, destroyed with the context).
zc_status ensure_upload_stream(zc_ctx* ctx, int n);
zc_status sumcheck_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                         const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                         bool proof_on_dev, bool v2 = false);
zc_status ntt_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                    const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                    bool proof_on_dev, void* q_out, int q_on_dev);
// scratch bytes one proof needs (device columns, device roots computed)
size_t sumcheck_scratch_bytes(const zc_ctx* ctx, const zc_params* p);
size_t ntt_scratch_bytes(const zc_params* p, int sm_count, bool q_direct);
// allocation-time set-up of the NTT form for one size (tables, attributes)
zc_status ntt_prepare(zc_ctx* ctx, const zc_params* p, cudaStream_t st);
// batch/serving lanes: child contexts with their own stream and scratch
zc_status make_lanes(zc_ctx* ctx, int K);
void destroy_lanes(zc_ctx* ctx);
void destroy_serve_pool(zc_ctx* ctx);

// ------------------------------------------------------------ device helpers
#if defined(__CUDACC__)
__device__ __forceinline__ fr ld_fr(const fr* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint4 a = __ldg(q), b = __ldg(q + 1);
  fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}
// plain (coherent) load for data written earlier by the same kernel family
__device__ __forceinline__ fr ld_fr_cg(const fr* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint4 a = q[0], b = q[1];
  fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}
__device__ __forceinline__ void st_fr(fr* p, const fr& x) {
  uint4* q = reinterpret_cast<uint4*>(p);
  q[0] = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
  q[1] = make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]);
}
__device__ __forceinline__ fr shfl_down_fr(const fr& x, int delta) {
  fr y;
#pragma unroll
  for (int i = 0; i < 8; i++) y.v[i] = __shfl_down_sync(0xffffffffu, x.v[i], delta);
  return y;
}
__device__ __forceinline__ fr shfl_fr(const fr& x, int src) {
  fr y;
#pragma unroll
  for (int i = 0; i < 8; i++) y.v[i] = __shfl_sync(0xffffffffu, x.v[i], src);
  return y;
}
// sum over the warp, result in lane 0
__device__ __forceinline__ fr warp_sum(fr x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = fr_add(x, shfl_down_fr(x, off));
  return x;
}
// canonical -> level 1 is M(x, R^2); level 1 -> canonical is M(x, 1)
__device__ __forceinline__ fr to_mont(const fr& x, const DevConst* C) { return fr_mul(x, C->r2); }
__device__ __forceinline__ fr from_mont(const fr& x) { return fr_mul(x, fr_from_u32(1)); }

// ---- plain 256-bit helpers for the binary inverse
__device__ __forceinline__ bool u256_is_one(const fr& x) {
  return x.v[0] == 1 && (x.v[1] | x.v[2] | x.v[3] | x.v[4] | x.v[5] | x.v[6] | x.v[7]) == 0;
}
__device__ __forceinline__ void u256_shr1(fr& x) {
#pragma unroll
  for (int i = 0; i < 7; i++) x.v[i] = (x.v[i] >> 1) | (x.v[i + 1] << 31);
  x.v[7] >>= 1;
}
__device__ __forceinline__ bool u256_geq(const fr& a, const fr& b) {
  for (int i = 7; i >= 0; i--)
    if (a.v[i] != b.v[i]) return a.v[i] > b.v[i];
  return true;
}
__device__ __forceinline__ void u256_sub_inplace(fr& a, const fr& b) {
  uint32_t br = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    uint64_t d = (uint64_t)a.v[i] - b.v[i] - br;
    a.v[i] = (uint32_t)d;
    br = (uint32_t)(d >> 63);
  }
}
// x/2 mod r for canonical x (x + r < 2^256 because r < 2^255)
__device__ __forceinline__ void half_mod(fr& x) {
  if (x.v[0] & 1) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      c += (uint64_t)x.v[i] + p_limb(i);
      x.v[i] = (uint32_t)c;
      c >>= 32;
    }
  }
  u256_shr1(x);
}

// a^{-1} mod r for canonical a, binary extended Euclid (Hankerson, Menezes,
// Vanstone, Guide to Elliptic Curve Cryptography, Alg. 2.22); canonical
// result, 0 for a = 0.  The loop is bounded (each pass removes at least one
// bit from u or v).
static __device__ __noinline__ fr fr_inv_binary(const fr& a) {
  if (fr_is_zero(a)) return fr_zero();
  fr u = a, v, x1 = fr_from_u32(1), x2 = fr_zero();
#pragma unroll
  for (int i = 0; i < 8; i++) v.v[i] = p_limb(i);
  for (int guard = 0; guard < 2048 && !u256_is_one(u) && !u256_is_one(v); guard++) {
    while ((u.v[0] & 1) == 0) {
      u256_shr1(u);
      half_mod(x1);
    }
    while ((v.v[0] & 1) == 0) {
      u256_shr1(v);
      half_mod(x2);
    }
    if (u256_geq(u, v)) {
      u256_sub_inplace(u, v);
      x1 = fr_sub(x1, x2);
    } else {
      u256_sub_inplace(v, u);
      x2 = fr_sub(x2, x1);
    }
  }
  return u256_is_one(u) ? x1 : x2;
}
#endif

}  // namespace zc
