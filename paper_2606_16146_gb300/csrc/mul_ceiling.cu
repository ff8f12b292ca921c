// mul_ceiling.cu -- throughput ceiling of the field multiplication on this GPU.
//
// A standalone program (built on demand by build.build_mul_ceiling(), run by
// `bench.py --workload mulpeak`).  It measures what bounds every prover
// kernel: how many BLS12-381 Fr Montgomery products per second the SMs
// sustain when they do nothing else, for
//   * the multiplier the kernels use (fr_mul, one out-of-line copy),
//   * the same code inlined at the call site (fr_mul_inl),
//   * the carry-chain IMAD form (fr_mul_cc: mad.lo.cc / madc.hi.cc),
//   * an unsaturated form for comparison: nine 29-bit limbs, each of the 18
//     product columns a 64-bit accumulator fed by 32x32->64 multiply-adds
//     (no carry chains inside the product), R = 2^261; checked against
//     fr_mul on random inputs,
// and the per-instruction rates of the integer operations they are built
// from.  Every thread runs two independent chains of dependent products.
// Prints one JSON object on stdout.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include "zc_field.cuh"

using namespace zc;

namespace {

constexpr uint32_t kM29 = 0x1fffffffu;

// r in radix 2^29
__device__ __forceinline__ uint32_t r29(int j) {
  switch (j) {
    case 0: return 0x00000001u;
    case 1: return 0x1ffffff8u;
    case 2: return 0x1f96ffbfu;
    case 3: return 0x1b4805ffu;
    case 4: return 0x1d80553bu;
    case 5: return 0x0c0404d0u;
    case 6: return 0x1520cce7u;
    case 7: return 0x0a6533afu;
    default: return 0x0073eda7u;
  }
}

struct f29 {
  uint32_t l[9];
};

// radix-2^29 limbs of (a << S); a < 2^256, S <= 5
template <int S>
__device__ __forceinline__ f29 to29(const fr& a) {
  f29 o;
#pragma unroll
  for (int j = 0; j < 9; j++) {
    const int lo = 29 * j - S;
    uint32_t x;
    if (lo < 0) {
      x = a.v[0] << (-lo);
    } else {
      const int k = lo >> 5, s = lo & 31;
      const uint32_t w1 = k + 1 < 8 ? a.v[k + 1] : 0u;
      x = s ? __funnelshift_r(a.v[k], w1, s) : a.v[k];
    }
    o.l[j] = x & kM29;
  }
  return o;
}

// (a b + m r) / 2^261, limbs normalised; a, b < 2^261 with a b < 2^261 r
// gives a result below 2r.  -r^{-1} = -1 mod 2^29 because r = 1 mod 2^29.
// Column k of a b + m r accumulates in its own 64-bit register T[k] through
// mad.wide.u32 (at most 18 products of 58 bits: below 2^63); after row i the
// low 29 bits of T[i] are zero and its carry moves to T[i+1].
__device__ __forceinline__ f29 mont29(const f29& a, const f29& b) {
  uint64_t T[18];
#pragma unroll
  for (int k = 0; k < 18; k++) T[k] = 0;
#pragma unroll
  for (int i = 0; i < 9; i++) {
#pragma unroll
    for (int j = 0; j < 9; j++) T[i + j] += static_cast<uint64_t>(a.l[i]) * b.l[j];
    const uint32_t m = (0u - static_cast<uint32_t>(T[i])) & kM29;
#pragma unroll
    for (int j = 1; j < 9; j++) T[i + j] += static_cast<uint64_t>(m) * r29(j);
    T[i + 1] += (T[i] + m) >> 29;
  }
  f29 o;
#pragma unroll
  for (int k = 9; k < 17; k++) {
    T[k + 1] += T[k] >> 29;
    o.l[k - 9] = static_cast<uint32_t>(T[k]) & kM29;
  }
  o.l[8] = static_cast<uint32_t>(T[17]);
  return o;
}

__device__ __forceinline__ fr from29(const f29& x) {
  uint32_t w[8];
  uint64_t acc = 0;
  int bits = 0, k = 0;
#pragma unroll
  for (int j = 0; j < 9; j++) {
    acc |= static_cast<uint64_t>(x.l[j]) << bits;
    bits += 29;
    if (bits >= 32) {
      if (k < 8) w[k] = static_cast<uint32_t>(acc);
      k++;
      acc >>= 32;
      bits -= 32;
    }
  }
  if (k < 8) w[k] = static_cast<uint32_t>(acc);
  return fr_reduce_final(w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]);
}

// a b 2^-256 through the 29-bit form: a is entered as a 2^5
__device__ __noinline__ fr mul_via29(fr a, fr b) { return from29(mont29(to29<5>(a), to29<0>(b))); }

enum Variant { kCall = 0, kInline = 1, kCarryChain = 2, kUnsat29 = 3, kVariants = 4 };

template <int V>
__global__ void __launch_bounds__(256) k_products(fr* out, int iters) {
  fr y;
  for (int i = 0; i < 8; i++) y.v[i] = 0x01234567u * (threadIdx.x + i + 1);
  y.v[7] &= 0x3fffffffu;
  fr x = y, x2 = y;
  x.v[0] += blockIdx.x;
  x2.v[1] ^= 7u;
  if (V == kUnsat29) {
    f29 X = to29<0>(x), X2 = to29<0>(x2);
    const f29 Y = to29<0>(y);
    for (int it = 0; it < iters; it++) {
      X = mont29(X, Y);
      X2 = mont29(X2, Y);
    }
    x = from29(X);
    x2 = from29(X2);
  } else {
    for (int it = 0; it < iters; it++) {
      if (V == kCall) { x = fr_mul(x, y); x2 = fr_mul(x2, y); }
      if (V == kInline) { x = fr_mul_inl(x, y); x2 = fr_mul_inl(x2, y); }
      if (V == kCarryChain) { x = fr_mul_cc(x, y); x2 = fr_mul_cc(x2, y); }
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = fr_add(x, x2);
}

__device__ uint32_t xorshift(uint32_t& s) {
  s ^= s << 13;
  s ^= s >> 17;
  s ^= s << 5;
  return s;
}

__global__ void k_check29(unsigned* bad, int n) {
  uint32_t s = 0x9e3779b9u ^ (blockIdx.x * 7919u + threadIdx.x * 104729u);
  unsigned nb = 0;
  for (int i = 0; i < n; i++) {
    fr a, b;
    for (int k = 0; k < 8; k++) { a.v[k] = xorshift(s); b.v[k] = xorshift(s); }
    a.v[7] &= 0x73ffffffu;
    b.v[7] &= 0x73ffffffu;
    if (i % 7 == 0) { for (int k = 0; k < 8; k++) a.v[k] = p_limb(k); a.v[0] -= 1; }
    if (i % 11 == 0) { for (int k = 0; k < 8; k++) b.v[k] = p_limb(k); b.v[0] -= 1; }
    if (i % 13 == 0) b = fr_zero();
    if (!fr_equal(mul_via29(a, b), fr_mul(a, b))) nb++;
  }
  atomicAdd(bad, nb);
}

// ---- per-instruction rates: 8 independent chains per thread, 4 x 8 ops per iteration
enum Op { kMadWide = 0, kMadLo = 1, kMadHi = 2, kAdd = 3, kAddCarryPair = 4, kOps = 5 };

template <int OP>
__global__ void __launch_bounds__(256) k_op(uint64_t* out, unsigned long long* cycles, int iters) {
  uint32_t a[8], b[8];
  uint64_t w[8];
  for (int c = 0; c < 8; c++) {
    a[c] = threadIdx.x * 2654435761u + c * 97u + blockIdx.x;
    b[c] = a[c] ^ 0x5bd1e995u;
    w[c] = (static_cast<uint64_t>(a[c]) << 32) | b[c];
  }
  const long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 4; u++) {
#pragma unroll
      for (int c = 0; c < 8; c++) {
        if (OP == kMadWide) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[c]) : "r"(a[c]), "r"(b[c]));
        if (OP == kMadLo) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(b[c]), "r"(b[c]));
        if (OP == kMadHi) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(b[c]), "r"(b[c]));
        if (OP == kAdd) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(b[c]));
        if (OP == kAddCarryPair)
          asm volatile("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %2;" : "+r"(a[c]), "+r"(b[c]) : "r"(c));
      }
    }
  }
  const long long t1 = clock64();
  uint64_t s = 0;
  for (int c = 0; c < 8; c++) s += w[c] + a[c] + b[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) atomicMax(cycles, static_cast<unsigned long long>(t1 - t0));
}

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                \
      return 1;                                                                    \
    }                                                                              \
  } while (0)

template <typename K>
int resident(K kernel, int threads) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0);
  return b > 0 ? b : 1;
}

}  // namespace

int main(int argc, char** argv) {
  const int iters = argc > 1 ? std::atoi(argv[1]) : 1000;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const int threads = 256, max_blocks = 8;
  fr* out = nullptr;
  uint64_t* out64 = nullptr;
  unsigned* bad = nullptr;
  unsigned long long* cyc = nullptr;
  CK(cudaMalloc(&out, sizeof(fr) * sms * max_blocks * threads));
  CK(cudaMalloc(&out64, sizeof(uint64_t) * sms * max_blocks * threads));
  CK(cudaMalloc(&bad, sizeof(unsigned)));
  CK(cudaMalloc(&cyc, sizeof(unsigned long long)));
  CK(cudaMemset(bad, 0, sizeof(unsigned)));
  const int check_n = 200;
  k_check29<<<sms * 2, threads>>>(bad, check_n);
  CK(cudaGetLastError());
  unsigned mismatches = 0;
  CK(cudaMemcpy(&mismatches, bad, sizeof(unsigned), cudaMemcpyDeviceToHost));

  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const char* vname[kVariants] = {"fr_mul_call", "fr_mul_inline", "fr_mul_carry_chain", "unsat29_core"};
  double rate[kVariants] = {0, 0, 0, 0};
  for (int v = 0; v < kVariants; v++) {
    const int blocks = sms * max_blocks;
    for (int rep = 0; rep < 2; rep++) {
      CK(cudaEventRecord(e0));
      switch (v) {
        case kCall: k_products<kCall><<<blocks, threads>>>(out, iters); break;
        case kInline: k_products<kInline><<<blocks, threads>>>(out, iters); break;
        case kCarryChain: k_products<kCarryChain><<<blocks, threads>>>(out, iters); break;
        default: k_products<kUnsat29><<<blocks, threads>>>(out, iters); break;
      }
      CK(cudaGetLastError());
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double r = static_cast<double>(blocks) * threads * iters * 2 / (ms * 1e-3);
      if (r > rate[v]) rate[v] = r;
    }
  }

  const char* oname[kOps] = {"mad.wide.u32", "mad.lo.u32", "mad.hi.u32", "add.u32", "add.cc+addc.u32"};
  const int per_step[kOps] = {1, 1, 1, 1, 2};
  double op_rate[kOps] = {0, 0, 0, 0, 0};
  double mhz = 0;
  const int op_iters = 4 * iters;
  for (int o = 0; o < kOps; o++) {
    int per_sm = 0;
    switch (o) {
      case kMadWide: per_sm = resident(k_op<kMadWide>, threads); break;
      case kMadLo: per_sm = resident(k_op<kMadLo>, threads); break;
      case kMadHi: per_sm = resident(k_op<kMadHi>, threads); break;
      case kAdd: per_sm = resident(k_op<kAdd>, threads); break;
      default: per_sm = resident(k_op<kAddCarryPair>, threads); break;
    }
    if (per_sm > max_blocks) per_sm = max_blocks;
    for (int rep = 0; rep < 2; rep++) {
      CK(cudaMemset(cyc, 0, sizeof(unsigned long long)));
      CK(cudaEventRecord(e0));
      switch (o) {
        case kMadWide: k_op<kMadWide><<<sms * per_sm, threads>>>(out64, cyc, op_iters); break;
        case kMadLo: k_op<kMadLo><<<sms * per_sm, threads>>>(out64, cyc, op_iters); break;
        case kMadHi: k_op<kMadHi><<<sms * per_sm, threads>>>(out64, cyc, op_iters); break;
        case kAdd: k_op<kAdd><<<sms * per_sm, threads>>>(out64, cyc, op_iters); break;
        default: k_op<kAddCarryPair><<<sms * per_sm, threads>>>(out64, cyc, op_iters); break;
      }
      CK(cudaGetLastError());
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      unsigned long long c = 0;
      CK(cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost));
      // one wave: every block is resident, so the longest block spans the kernel
      const double warp_instr = static_cast<double>(per_sm) * (threads / 32) * op_iters * 4 * 8 * per_step[o];
      const double r = warp_instr / static_cast<double>(c);
      if (r > op_rate[o]) op_rate[o] = r;
      if (o == kAdd && rep == 1) mhz = static_cast<double>(c) / (ms * 1e3);
    }
  }
  CK(cudaDeviceSynchronize());

  std::printf("{\"sms\": %d, \"threads_per_block\": %d, \"blocks_per_sm\": %d, \"products_per_thread\": %d, "
              "\"sm_mhz_under_load\": %.0f, \"unsat29_check\": {\"mismatches\": %u, \"products\": %d}, "
              "\"mulmod_per_s\": {",
              sms, threads, max_blocks, 2 * iters, mhz, mismatches, sms * 2 * threads * check_n);
  for (int v = 0; v < kVariants; v++) std::printf("%s\"%s\": %.4e", v ? ", " : "", vname[v], rate[v]);
  std::printf("}, \"warp_instr_per_clk_per_sm\": {");
  for (int o = 0; o < kOps; o++) std::printf("%s\"%s\": %.3f", o ? ", " : "", oname[o], op_rate[o]);
  std::printf("}}\n");
  return mismatches ? 2 : 0;
}
