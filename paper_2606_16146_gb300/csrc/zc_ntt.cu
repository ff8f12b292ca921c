// zc_ntt.cu -- NTT-form ZeroCheck prover (Fig. side-by-side-zc, left;
// Sec. 3.2).
//
//   N1  g_j <- INTT_H(e_j)                    (per column, size N)
//   N2  for each coset slice s_j = 7 w_M^j H (j < s = M/N):
//         ghat_j = NTT_N(g_j(k) (7 w_M^j)^k / N), fhat = gate(ghat),
//         qhat = fhat / z_H, with z_H constant on the slice: 7^N w_s^j - 1
//   N3  q <- INTT_D(qhat) = 7^-k M^-1 DFT_M^-1(qhat)
//   N4  root(q), z = squeeze (again while z^N = 1)
//   N5  openings g_j(z), q(z)
//
// Transforms are "four-step" (Bailey) factorisations done as passes over
// HBM; each pass runs many sub-DFTs of length L <= 4096 in shared memory
// (self-sorting Stockham stages of radix 8/4/2).  Digit orders are chosen so
// that no pass ever transposes:
//   * N1 is the reversed-input structure: its first pass reads the natural
//     evaluations with a stride (a gather), its output is natural.
//   * N2 is the natural-input structure: each slice comes out digit-reversed.
//   * The gate is pointwise, so qhat keeps that order, which is exactly the
//     input order of N3 written as a three-digit reversed-input transform
//     (slice digit outermost); N3's output, q, is natural.
// Twiddles between passes come from two-level power tables of the 2^30-th
// root of unity (w^e = HI[e >> 15] * LO[e & 32767]).  The coset factor
// (7 w_M^j)^k / N of N2 is a two-level table per slice applied on load, with
// the Montgomery conversion folded in (inputs are canonical, "level 0").
#include <algorithm>
#include <cstring>

#include "zc_internal.cuh"
#include "zc_transcript.cuh"

namespace zc {

constexpr int kLog30 = 30;
constexpr uint32_t kLoBits = 15;
constexpr uint32_t kLoMask = (1u << kLoBits) - 1;
constexpr int kMaxNttN = 24;

struct NttTables {
  bool ready = false;
  fr w32h;                 // 7^((r-1)/2^32), canonical, host copy
  fr* dft_fwd = nullptr;   // w_4096^m, m < 4096 (level 1)
  fr* dft_inv = nullptr;
  fr* wf_lo = nullptr;     // w_2^30^b, b < 2^15 (level 1)
  fr* wf_hi = nullptr;     // w_2^30^(a 2^15)
  fr* wi_lo = nullptr;     // inverse root
  fr* wi_hi = nullptr;
  fr* s7_lo = nullptr;     // 7^-b (level 0)
  fr* s7_hi = nullptr;     // 7^-(a 2^15) (level 1)
  fr* p7_lo = nullptr;     // 7^b (level 1)
  fr* p7_hi = nullptr;     // 7^(a 2^15) (level 1)
  void* mem = nullptr;
};

static NttTables g_tabs_by_dev[64];
static std::mutex g_tabs_mu;

struct NttTabArgs {
  fr* dft_fwd; fr* dft_inv; fr* wf_lo; fr* wf_hi; fr* wi_lo; fr* wi_hi; fr* s7_lo; fr* s7_hi;
  fr* p7_lo; fr* p7_hi;
  fr w30;        // 2^30-th root (level 1)
  fr w30i;       // its inverse (level 1)
  fr seveninv;   // 7^-1 (level 1)
  const DevConst* C;
};

__device__ fr fr_pow_dev(fr base, uint64_t e, const DevConst* C) {  // level 1 in/out
  fr acc = C->one;
  while (e) {
    if (e & 1) acc = fr_mul(acc, base);
    base = fr_mul(base, base);
    e >>= 1;
  }
  return acc;
}

__global__ void k_ntt_tables(NttTabArgs A) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const DevConst* C = A.C;
  if (i < 4096) {
    // w_4096 = w30^(2^18)
    A.dft_fwd[i] = fr_pow_dev(A.w30, (uint64_t)i << 18, C);
    A.dft_inv[i] = fr_pow_dev(A.w30i, (uint64_t)i << 18, C);
  }
  if (i < (1u << kLoBits)) {
    A.wf_lo[i] = fr_pow_dev(A.w30, i, C);
    A.wf_hi[i] = fr_pow_dev(A.w30, (uint64_t)i << kLoBits, C);
    A.wi_lo[i] = fr_pow_dev(A.w30i, i, C);
    A.wi_hi[i] = fr_pow_dev(A.w30i, (uint64_t)i << kLoBits, C);
    A.s7_lo[i] = from_mont(fr_pow_dev(A.seveninv, i, C));          // level 0
    A.s7_hi[i] = fr_pow_dev(A.seveninv, (uint64_t)i << kLoBits, C);  // level 1
    A.p7_lo[i] = fr_pow_dev(C->small[7], i, C);
    A.p7_hi[i] = fr_pow_dev(C->small[7], (uint64_t)i << kLoBits, C);
  }
}

// w^e for the 2^30-th root (or its inverse), e < 2^30, level 1
__device__ __forceinline__ fr root_pow(const fr* lo, const fr* hi, uint32_t e) {
  return fr_mul(ld_fr(hi + (e >> kLoBits)), ld_fr(lo + (e & kLoMask)));
}

// ---------------------------------------------------------------- passes --

enum { PRE_NONE = 0, PRE_COSET = 1, PRE_TAB = 2 };
enum { POST_NONE = 0, POST_TW = 1, POST_OUTER = 2, POST_FINAL = 3, POST_TAB = 4 };

struct NttPassArgs {
  const fr* in[kMaxCols];
  fr* out[kMaxCols];
  uint32_t items;         // columns in this launch
  uint32_t logL;          // sub-DFT length
  uint32_t logW;          // sub-DFTs per CTA
  // element (b, t) address: ((b >> lbdiv) * bs_hi) + (b & (bdiv-1)) * bs_lo + t * ts
  uint32_t in_lbdiv, out_lbdiv;
  uint64_t in_bs_hi, in_bs_lo, in_ts;
  uint64_t out_bs_hi, out_bs_lo, out_ts;
  const fr* dft;          // 4096-th roots, forward or inverse
  int pre;
  const fr* pre_lo;       // per-item coset tables (item stride pre_stride)
  const fr* pre_hi;
  uint32_t pre_shift;     // k = b * pre_kb + t * pre_kt; factor = hi[k >> shift] * lo[k & mask]
  uint64_t pre_kb, pre_kt;
  int post;
  const fr* tw_lo;
  const fr* tw_hi;
  uint32_t tw_lbmod;      // POST_TW: e = (b mod 2^lbmod) * t
  uint32_t tw_shift;      // exponent in the 2^30 table: (e mod 2^(30-shift)) << shift
  uint32_t outer_lbdiv;   // POST_OUTER: e = (b >> lbdiv) * ((t << lbdiv) + (b mod 2^lbdiv))
  uint64_t fin_N;         // POST_FINAL: k = fin_N * t + b
  // table modes: PRE_TAB factor = pre_tab[b * pre_kb + t * pre_kt];
  // POST_TAB factor = post_tab[(b >> p_lbdiv) * p_hs + (b & (2^p_lbdiv - 1)) * p_ls + t * p_ts]
  const fr* pre_tab;
  const fr* post_tab;
  uint32_t p_lbdiv;
  uint64_t p_hs, p_ls, p_ts;
  uint32_t* err;          // if set: the pass reads the proof's input columns, and a value >= r sets bit 0
};

// radix-2/4/8 butterflies on x[0..R) in registers, X[k] = sum_r x[r] w_R^(rk).
// Inputs are canonical.  A value that only feeds a multiplication (as
// fr_mul's second operand, which may be any value below 2r) is left lazily
// reduced in [0, 2r): the stage outputs (the next stage multiplies all but
// one of them by its twiddle and reduces that one, the pass's store reduces
// or multiplies every one), and the terms multiplied by w_4, w_8, w_8^3.
// OUT: 0 every output canonical, 1 a0 canonical and a1..a3 lazy, 2 all lazy.
template <int OUT>
__device__ __forceinline__ void dft4(fr& a0, fr& a1, fr& a2, fr& a3, const fr& w4) {
  const fr u0 = fr_add(a0, a2), u1 = fr_sub(a0, a2);
  const fr v0 = fr_add(a1, a3), v1 = fr_mul(w4, fr_sub_lazy(a1, a3));
  a0 = OUT == 2 ? fr_add_lazy(u0, v0) : fr_add(u0, v0);
  a2 = OUT >= 1 ? fr_sub_lazy(u0, v0) : fr_sub(u0, v0);
  a1 = OUT >= 1 ? fr_add_lazy(u1, v1) : fr_add(u1, v1);
  a3 = OUT >= 1 ? fr_sub_lazy(u1, v1) : fr_sub(u1, v1);
}

// outputs lazy
__device__ __forceinline__ void dft8(fr (&x)[8], const fr* tab) {
  fr e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  fr o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<0>(e0, e1, e2, e3, ld_fr(tab + 1024));
  dft4<1>(o0, o1, o2, o3, ld_fr(tab + 1024));
  o1 = fr_mul(ld_fr(tab + 512), o1);    // w_8
  o2 = fr_mul(ld_fr(tab + 1024), o2);   // w_4
  o3 = fr_mul(ld_fr(tab + 1536), o3);   // w_8^3
  x[0] = fr_add_lazy(e0, o0);
  x[4] = fr_sub_lazy(e0, o0);
  x[1] = fr_add_lazy(e1, o1);
  x[5] = fr_sub_lazy(e1, o1);
  x[2] = fr_add_lazy(e2, o2);
  x[6] = fr_sub_lazy(e2, o2);
  x[3] = fr_add_lazy(e3, o3);
  x[7] = fr_sub_lazy(e3, o3);
}

// The CTA tile in shared memory: element i's two 16-byte halves live in two
// planes, and the 16-byte index is XOR-swizzled (i ^ ((i >> 3) & 7)) so
// that unit-stride and radix-strided (8, 64) warp accesses spread over all
// banks.
struct SmTile {
  uint4* p;     // plane 0: p[0, T), plane 1: p[T, 2T)
  uint32_t T;
  __device__ __forceinline__ uint32_t sw(uint32_t i) const { return i ^ ((i >> 3) & 7); }
  __device__ __forceinline__ fr get(uint32_t i) const {
    const uint32_t s = sw(i);
    const uint4 a = p[s], b = p[T + s];
    fr x;
    x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
    x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
    return x;
  }
  __device__ __forceinline__ void put(uint32_t i, const fr& x) const {
    const uint32_t s = sw(i);
    p[s] = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
    p[T + s] = make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]);
  }
};

// One Stockham stage of radix R = 2^lr on the CTA tile sm[t * W + w]; each
// thread owns 8 elements (8 / R independent groups).
template <int LR>
__device__ __forceinline__ void stockham_stage(const SmTile& sm, uint32_t logL, uint32_t logW,
                                               uint32_t logNs, const fr* tab) {
  constexpr int R = 1 << LR;
  constexpr int GROUPS = 8 / R;
  const uint32_t L = 1u << logL, W = 1u << logW;
  const uint32_t qL = L >> LR;   // L / R
  const uint32_t ngroups = (L << logW) >> LR;
  fr x[8];
  uint32_t jj[GROUPS], ww[GROUPS];
#pragma unroll
  for (int g = 0; g < GROUPS; g++) {
    uint32_t j_all = threadIdx.x * GROUPS + g;
    uint32_t w = j_all & (W - 1), j = j_all >> logW;
    jj[g] = j;
    ww[g] = w;
    if (j_all < ngroups) {
#pragma unroll
      for (int r = 0; r < R; r++) x[g * R + r] = sm.get((j + r * qL) * W + w);
    }
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < GROUPS; g++) {
    if (threadIdx.x * GROUPS + g >= ngroups) continue;
    const uint32_t j = jj[g];
    const uint32_t k = j & ((1u << logNs) - 1);
    if (logNs > 0) {
      // the previous stage left its outputs lazy: x[0] is reduced, the
      // others are reduced by their twiddle w_{Ns R}^{r k} = tab[r k 4096 / (Ns R)].
      // These products, and the pass's load and store factors, use the
      // inlined multiplier (fewer instructions than the shared call); the
      // DFT-8's own products stay calls (inlined they spilled registers and
      // measured slower).
      const uint32_t sh = 12 - (logNs + LR);
      x[g * R] = fr_reduce1(x[g * R]);
#pragma unroll
      for (int r = 1; r < R; r++) x[g * R + r] = fr_mul_inl(ld_fr(tab + ((r * k) << sh)), x[g * R + r]);
    }
    if (R == 8) {
      fr y[8];
#pragma unroll
      for (int r = 0; r < 8; r++) y[r] = x[r];
      dft8(y, tab);
#pragma unroll
      for (int r = 0; r < 8; r++) x[r] = y[r];
    } else if (R == 4) {
      dft4<2>(x[g * 4], x[g * 4 + 1], x[g * 4 + 2], x[g * 4 + 3], ld_fr(tab + 1024));
    } else {
      fr a = x[g * 2], b = x[g * 2 + 1];
      x[g * 2] = fr_add_lazy(a, b);
      x[g * 2 + 1] = fr_sub_lazy(a, b);
    }
  }
#pragma unroll
  for (int g = 0; g < GROUPS; g++) {
    if (threadIdx.x * GROUPS + g >= ngroups) continue;
    const uint32_t j = jj[g], w = ww[g];
    const uint32_t k = j & ((1u << logNs) - 1);
    const uint32_t idxD = ((j >> logNs) << (logNs + LR)) + k;
#pragma unroll
    for (int r = 0; r < R; r++) sm.put((idxD + (r << logNs)) * W + w, x[g * R + r]);
  }
  __syncthreads();
}

template <int TILE, int MINB>
__global__ void __launch_bounds__(TILE / 8, MINB) k_ntt_pass(NttPassArgs A) {
  extern __shared__ __align__(16) uint4 sm_planes[];
  const SmTile sm{sm_planes, (uint32_t)TILE};
  // items (columns) vary fastest across consecutive CTAs, so the per-element
  // factor tables, shared by every column, are reused from L2
  const uint32_t items = A.items;
  const int item = (int)(blockIdx.x % items);
  const uint64_t blk = blockIdx.x / items;
  const fr* __restrict__ in = A.in[item];
  fr* out = A.out[item];
  const uint32_t logL = A.logL, logW = A.logW;
  const uint32_t L = 1u << logL, W = 1u << logW;
  const uint64_t b0 = blk << logW;
  const uint32_t n_el = L << logW;  // <= TILE (smaller only for tiny transforms)
  const bool in_t_fast = A.in_ts == 1, out_t_fast = A.out_ts == 1;
  const uint64_t in_bdiv_mask = (1ull << A.in_lbdiv) - 1, out_bdiv_mask = (1ull << A.out_lbdiv) - 1;

  // ---- load (with the coset factor when asked)
  if (A.pre == PRE_NONE && n_el == (uint32_t)TILE) {
    // no factor to apply: both 16-byte halves of every element go straight
    // from global to their planes (cp.async, no register staging), all of
    // this thread's copies in flight together
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint32_t idx = threadIdx.x + (uint32_t)u * (TILE / 8);
      uint32_t w, t;
      if (in_t_fast) { t = idx & (L - 1); w = idx >> logL; }
      else { w = idx & (W - 1); t = idx >> logW; }
      const uint64_t b = b0 + w;
      const uint64_t a = (b >> A.in_lbdiv) * A.in_bs_hi + (b & in_bdiv_mask) * A.in_bs_lo + t * A.in_ts;
      const uint32_t s = sm.sw(t * W + w);
      const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(sm.p + s);
      const uint32_t d1 = (uint32_t)__cvta_generic_to_shared(sm.p + TILE + s);
      const char* g = reinterpret_cast<const char*>(in + a);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0), "l"(g) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d1), "l"(g + 16) : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    if (A.err) {
      // the input check reads back what this thread copied
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t idx = threadIdx.x + (uint32_t)u * (TILE / 8);
        uint32_t w, t;
        if (in_t_fast) { t = idx & (L - 1); w = idx >> logL; }
        else { w = idx & (W - 1); t = idx >> logW; }
        if (!fr_is_canonical(sm.get(t * W + w))) atomicOr(A.err, 1u);
      }
    }
  } else
  for (uint32_t idx = threadIdx.x; idx < n_el; idx += blockDim.x) {
    uint32_t w, t;
    if (in_t_fast) { t = idx & (L - 1); w = idx >> logL; }
    else { w = idx & (W - 1); t = idx >> logW; }
    const uint64_t b = b0 + w;
    const uint64_t a = (b >> A.in_lbdiv) * A.in_bs_hi + (b & in_bdiv_mask) * A.in_bs_lo + t * A.in_ts;
    fr x = ld_fr(in + a);
    if (A.err && !fr_is_canonical(x)) atomicOr(A.err, 1u);
    if (A.pre == PRE_TAB) {
      x = fr_mul_inl(ld_fr(A.pre_tab + b * A.pre_kb + t * A.pre_kt), x);
    } else if (A.pre == PRE_COSET) {
      const uint64_t k = b * A.pre_kb + t * A.pre_kt;
      // one slice per launch: every column uses the same tables
      fr f = fr_mul(ld_fr(A.pre_hi + (k >> A.pre_shift)),
                    ld_fr(A.pre_lo + (k & ((1ull << A.pre_shift) - 1))));
      x = fr_mul(x, f);
    }
    sm.put(t * W + w, x);
  }
  __syncthreads();

  // ---- Stockham stages: radix 8 while >= 3 bits remain, then 4 or 2
  uint32_t logNs = 0;
  while (logL - logNs >= 3) {
    stockham_stage<3>(sm, logL, logW, logNs, A.dft);
    logNs += 3;
  }
  if (logL - logNs == 2) stockham_stage<2>(sm, logL, logW, logNs, A.dft);
  else if (logL - logNs == 1) stockham_stage<1>(sm, logL, logW, logNs, A.dft);

  // ---- store (with the twiddle / final scale)
  for (uint32_t idx = threadIdx.x; idx < n_el; idx += blockDim.x) {
    uint32_t w, t;
    if (out_t_fast) { t = idx & (L - 1); w = idx >> logL; }
    else { w = idx & (W - 1); t = idx >> logW; }
    const uint64_t b = b0 + w;
    fr y = sm.get(t * W + w);  // lazily reduced: multiplied (as the second operand) or reduced here
    if (A.post == POST_TAB) {
      const uint64_t ti = (b >> A.p_lbdiv) * A.p_hs + (b & ((1ull << A.p_lbdiv) - 1)) * A.p_ls + t * A.p_ts;
      y = fr_mul_inl(ld_fr(A.post_tab + ti), y);
    } else if (A.post == POST_TW) {
      const uint64_t e = (b & ((1ull << A.tw_lbmod) - 1)) * t;
      const uint32_t ex = (uint32_t)((e << A.tw_shift) & ((1ull << kLog30) - 1));
      y = ex ? fr_mul(root_pow(A.tw_lo, A.tw_hi, ex), y) : fr_reduce1(y);
    } else if (A.post == POST_OUTER) {
      const uint64_t jsl = b >> A.outer_lbdiv;
      const uint64_t kp = ((uint64_t)t << A.outer_lbdiv) + (b & ((1ull << A.outer_lbdiv) - 1));
      const uint64_t e = jsl * kp;
      const uint32_t ex = (uint32_t)((e << A.tw_shift) & ((1ull << kLog30) - 1));
      y = ex ? fr_mul(root_pow(A.tw_lo, A.tw_hi, ex), y) : fr_reduce1(y);
    } else if (A.post == POST_FINAL) {
      const uint64_t k = A.fin_N * t + b;
      fr f = fr_mul(ld_fr(A.tw_hi + (k >> kLoBits)), ld_fr(A.tw_lo + (k & kLoMask)));  // level 0
      y = fr_mul(f, y);
    } else {
      y = fr_reduce1(y);
    }
    const uint64_t a = (b >> A.out_lbdiv) * A.out_bs_hi + (b & out_bdiv_mask) * A.out_bs_lo + t * A.out_ts;
    st_fr(out + a, y);
  }
}

// ----------------------------------------------------- per-size tables --
// For one (n, log2 s): the four-step twiddles of size N in both directions,
// the coset factors (7 w_M^j)^k / N of every slice (level 2, which also
// converts canonical coefficients to Montgomery form), the outer twiddles of
// the quotient INTT and its final scale 7^-k (level 0).  They depend only on
// the sizes, so a context builds them on first use and reuses them.
struct NttSizeArgs {
  fr* tw_fwd;   // [b * L1 + t] = w_N^(b t), b < L2, t < L1
  fr* tw_inv;   // [b * L2 + t] = w_N^-(b t), b < L1, t < L2
  fr* coset;    // [j * N + k] = (7 w_M^j)^k / N   (level 2)
  fr* outer;    // [j * N + k] = w_M^-(j k)
  fr* fin;      // [k] = 7^-k                       (level 0)
  uint32_t n, lb, l1, l2;
  fr ninv_l2;
  const NttTables* T;
  const DevConst* C;
};

__global__ void k_ntt_size_tables(NttSizeArgs A, NttTables T) {
  const uint64_t N = 1ull << A.n, M = N << A.lb;
  const uint32_t logm = A.n + A.lb;
  const uint64_t L1 = 1ull << A.l1, L2 = 1ull << A.l2;
  const uint64_t total = 2 * N + 3 * M;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    if (e < N) {
      const uint64_t b = e / L1, t = e % L1;
      const uint32_t ex = (uint32_t)((((b * t) & (N - 1)) << (kLog30 - A.n)) & ((1ull << kLog30) - 1));
      st_fr(A.tw_fwd + e, root_pow(T.wf_lo, T.wf_hi, ex));
    } else if (e < 2 * N) {
      const uint64_t i = e - N, b = i / L2, t = i % L2;
      const uint32_t ex = (uint32_t)((((b * t) & (N - 1)) << (kLog30 - A.n)) & ((1ull << kLog30) - 1));
      st_fr(A.tw_inv + i, root_pow(T.wi_lo, T.wi_hi, ex));
    } else if (e < 2 * N + M) {
      const uint64_t i = e - 2 * N, j = i >> A.n, k = i & (N - 1);
      const uint32_t ex = (uint32_t)(((j * k) & (M - 1)) << (kLog30 - logm));
      fr f = fr_mul(fr_mul(ld_fr(T.p7_hi + (k >> kLoBits)), ld_fr(T.p7_lo + (k & kLoMask))),
                    root_pow(T.wf_lo, T.wf_hi, ex));
      st_fr(A.coset + i, fr_mul(f, A.ninv_l2));
    } else if (e < 2 * N + 2 * M) {
      const uint64_t i = e - 2 * N - M, j = i >> A.n, k = i & (N - 1);
      const uint32_t ex = (uint32_t)(((j * k) & (M - 1)) << (kLog30 - logm));
      st_fr(A.outer + i, root_pow(T.wi_lo, T.wi_hi, ex));
    } else {
      const uint64_t k = e - 2 * N - 2 * M;
      st_fr(A.fin + k, fr_mul(ld_fr(T.s7_hi + (k >> kLoBits)), ld_fr(T.s7_lo + (k & kLoMask))));
    }
  }
}

// ------------------------------------------------------- per-proof kernels --

struct NttSliceTabArgs {
  fr* lo;            // [s][2^hbits] c_j^b (level 1)
  fr* hi;            // [s][2^(n-hbits)] c_j^(a 2^hbits) / N (level 2)
  fr* zinv;          // [s] (7^N w_s^j - 1)^-1 M^-1 (level 1)
  uint32_t s, n, hbits, logm;
  fr ninv_l2;        // N^-1 at level 2
  fr minv_l1;        // M^-1 at level 1
  const fr* wf_lo; const fr* wf_hi;
  const DevConst* C;
};

__global__ void k_ntt_slice_tables(NttSliceTabArgs A) {
  const DevConst* C = A.C;
  const uint32_t nlo = 1u << A.hbits, nhi = 1u << (A.n - A.hbits);
  const uint32_t per = nlo + nhi;
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint64_t)A.s * per) {
    const uint32_t j = (uint32_t)(i / per), e = (uint32_t)(i % per);
    // c_j = 7 w_M^j
    const uint32_t ex = (j << (kLog30 - A.logm)) & ((1u << kLog30) - 1);
    fr cj = fr_mul(C->small[7], root_pow(A.wf_lo, A.wf_hi, ex));
    if (e < nlo) {
      A.lo[(size_t)j * nlo + e] = fr_pow_dev(cj, e, C);
    } else {
      const uint32_t a = e - nlo;
      fr v = fr_pow_dev(cj, (uint64_t)a << A.hbits, C);
      A.hi[(size_t)j * nhi + a] = fr_mul(v, A.ninv_l2);  // level 2
    }
  }
  if (i < A.s) {
    // z_H on slice j: (7 w_M^j w_N^i)^N - 1 = 7^N w_s^j - 1
    const uint32_t j = (uint32_t)i;
    fr s7n = fr_pow_dev(C->small[7], 1ull << A.n, C);
    const uint32_t ex = (j << (kLog30 - (A.logm - A.n))) & ((1u << kLog30) - 1);
    fr zj = fr_sub(fr_mul(s7n, root_pow(A.wf_lo, A.wf_hi, ex)), C->one);
    fr inv = fr_inv_binary(from_mont(zj));        // canonical
    A.zinv[j] = fr_mul(fr_mul(inv, C->r2), A.minv_l1);
  }
}

struct NttGateArgs {
  const fr* col[kMaxCols];  // slice evaluations, level 1
  fr* qhat;                 // slice output
  const fr* zinv;           // constant of this slice
  const fr* sub;            // nullptr, or values subtracted after the scaling (level 1)
  uint64_t N;
  uint32_t gate, d, c;       // gate word, degree, columns
};

// f at the slice points, times the slice constant 1 / (z_H M): Plonk; product
// q w1 .. w_{d-1} - o; sum g_1 .. g_d + g_{d+1} + .. + g_c (all at level 1).
__global__ void __launch_bounds__(256) k_ntt_gate(NttGateArgs A) {
  const fr zi = ld_fr(A.zinv);
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < A.N;
       p += (uint64_t)gridDim.x * blockDim.x) {
    fr f;
    if (A.gate == ZC_GATE_PLONK) {
      // a (qL + qM b) + qR b + qO c with one reduction for the three products
      const fr b = ld_fr(A.col[6] + p);
      const fr u = fr_add(ld_fr(A.col[0] + p), fr_mul_inl(ld_fr(A.col[2] + p), b));
      f = fr_mul_sum3(ld_fr(A.col[5] + p), u, ld_fr(A.col[1] + p), b, ld_fr(A.col[3] + p), ld_fr(A.col[7] + p));
      f = fr_add(f, ld_fr(A.col[4] + p));
    } else {
      f = ld_fr(A.col[0] + p);
      for (uint32_t j = 1; j < A.d; j++) f = fr_mul_inl(f, ld_fr(A.col[j] + p));
      if (A.gate == ZC_GATE_PRODUCT) f = fr_sub(f, ld_fr(A.col[A.d] + p));
      else
        for (uint32_t j = A.d; j < A.c; j++) f = fr_add(f, ld_fr(A.col[j] + p));
    }
    f = fr_mul_inl(zi, f);
    if (A.sub) f = fr_sub(f, ld_fr(A.sub + p));
    st_fr(A.qhat + p, f);
  }
}

// ------------------------------------------------ step-radix domain --
// D = D_big u D_small, D_big = 7 <w_M> (M = 2^lb N), D_small = sigma H with
// sigma = 7 w_{2M} (Sec. 4, degree scaling: a transform of M + N points
// from power-of-two transforms plus element-wise work).  q = q_big +
// (x^M - 7^M) q_small: q_big is the INTT over D_big of qhat there; on
// D_small, x^M = sigma^M, so q_small = INTT over D_small of
// (qhat - q_big) / kappa, kappa = sigma^M - 7^M.

struct NttStepTabArgs {
  fr* coset;      // [k] sigma^k / N, level 2
  fr* unscale;    // [k] w_{2M}^-k, level 1
  uint32_t n, shift2m;  // exponent shift of w_{2M} in the 2^30 tables: 30 - log2(2M)
  fr ninv_l2;
  NttTables T;
};

__global__ void k_ntt_step_tables(NttStepTabArgs A) {
  const uint64_t N = 1ull << A.n;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t ex = (uint32_t)((k << A.shift2m) & ((1ull << kLog30) - 1));
    const fr p7 = fr_mul(ld_fr(A.T.p7_hi + (k >> kLoBits)), ld_fr(A.T.p7_lo + (k & kLoMask)));  // 7^k
    st_fr(A.coset + k, fr_mul(fr_mul(p7, root_pow(A.T.wf_lo, A.T.wf_hi, ex)), A.ninv_l2));
    st_fr(A.unscale + k, root_pow(A.T.wi_lo, A.T.wi_hi, ex));
  }
}

// q_big evaluated on D_small starts with its reduction modulo x^N - sigma^N,
// scaled by 1/kappa: rho[k] = sum_m q[k + m N] sigma^(mN) / kappa.
struct NttStepReduceArgs {
  const fr* q;       // q_big, M canonical coefficients
  fr* rho;           // N outputs, level 0
  const fr* cm;      // 2^lb constants sigma^(mN) / kappa, level 1
  uint64_t N;
  uint32_t parts;    // M / N
};

__global__ void k_ntt_step_reduce(NttStepReduceArgs A) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < A.N;
       k += (uint64_t)gridDim.x * blockDim.x) {
    fr acc = fr_mul(ld_fr(A.q + k), ld_fr(A.cm));
    for (uint32_t m = 1; m < A.parts; m++) acc = fr_add(acc, fr_mul(ld_fr(A.q + k + m * A.N), ld_fr(A.cm + m)));
    st_fr(A.rho + k, acc);
  }
}

// q_small[k] = w_{2M}^-k x[k] (x: the small part's INTT, which carried the
// factor 7^-k); q[M + k] = q_small[k], q[k] -= 7^M q_small[k].
struct NttStepCombineArgs {
  fr* q;             // M + N coefficients; x in q[M .. M + N)
  const fr* unscale;
  const fr* s7m;     // 7^M, level 1
  uint64_t N, M;
};

__global__ void k_ntt_step_combine(NttStepCombineArgs A) {
  const fr c = ld_fr(A.s7m);
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < A.N;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const fr t = fr_mul(ld_fr(A.q + A.M + k), ld_fr(A.unscale + k));
    st_fr(A.q + A.M + k, t);
    st_fr(A.q + k, fr_sub(ld_fr(A.q + k), fr_mul(t, c)));
  }
}

struct NttZArgs {
  NttState* st;
  const uint8_t* roots;  // c column roots then root(q)
  int c;
  uint32_t n;
  uint32_t S0[8];
  fr* zpow;              // z^(2^i), i < 31 (level 1)
  const DevConst* C;
};

__global__ void k_ntt_z(NttZArgs A) {
  if (threadIdx.x != 0) return;
  const DevConst* C = A.C;
  uint32_t S[8];
  for (int i = 0; i < 8; i++) S[i] = A.S0[i];
  for (int j = 0; j <= A.c; j++) tr_absorb32(S, A.roots + 32 * j);
  fr z;
  uint32_t err = 1;
  for (int tries = 0; tries < 64; tries++) {
    z = fr_mul(tr_squeeze(S), C->r2);
    fr zn = z;
    for (uint32_t i = 0; i < A.n; i++) zn = fr_mul(zn, zn);
    if (!fr_equal(zn, C->one)) {
      err = 0;
      A.st->zpow_n = zn;
      break;
    }
  }
  A.st->z = z;
  A.st->err |= err;
  fr p = z;
  for (int i = 0; i < 31; i++) {
    A.zpow[i] = p;
    p = fr_mul(p, p);
  }
}

// Evaluate sum_k x[k] z^k for each item (level-0 x); every warp takes a
// contiguous segment, lane l the elements seg + l + 32 m, Horner in z^32.
struct NttOpenArgs {
  const fr* x[kMaxCols + 1];
  uint64_t len[kMaxCols + 1];
  const fr* zpow;     // z^(2^i)
  fr* partials;       // [item][blocks]
  uint32_t nblk;
  uint32_t seg;       // elements per warp segment (multiple of 32)
};

__device__ fr zpow_of(const fr* zp, uint64_t e, const fr& one) {
  fr acc = one;
  for (int i = 0; e; i++, e >>= 1)
    if (e & 1) acc = fr_mul(acc, ld_fr(zp + i));
  return acc;
}

__global__ void __launch_bounds__(256) k_ntt_open(NttOpenArgs A, const DevConst* C) {
  const int item = blockIdx.y;
  const fr* x = A.x[item];
  const uint64_t len = A.len[item];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const fr z32 = ld_fr(A.zpow + 5);
  fr tot = fr_zero();
  const uint64_t nseg = (len + A.seg - 1) / A.seg;
  for (uint64_t sgi = (uint64_t)blockIdx.x * 8 + warp; sgi < nseg; sgi += (uint64_t)gridDim.x * 8) {
    const uint64_t base = sgi * A.seg;
    const uint64_t cnt = A.seg < len - base ? A.seg : len - base;
    const uint32_t mcount = (uint32_t)((cnt + 31) / 32);
    fr acc = fr_zero();
    for (int32_t m = (int32_t)mcount - 1; m >= 0; m--) {
      const uint64_t k = base + lane + 32ull * (uint32_t)m;
      const fr xk = k < len ? ld_fr(x + k) : fr_zero();
      // while the warp's accumulators and values are all zero (the zero top
      // of an honest quotient) the step would multiply zeros: skip it
      if (__all_sync(0xffffffffu, fr_is_zero(acc) && fr_is_zero(xk))) continue;
      acc = fr_add(fr_mul_inl(z32, acc), xk);
    }
    if (__all_sync(0xffffffffu, fr_is_zero(acc))) continue;
    acc = fr_mul(acc, zpow_of(A.zpow, base + lane, C->one));
    tot = fr_add(tot, acc);
  }
  __shared__ fr red[8];
  tot = warp_sum(tot);
  if (lane == 0) red[warp] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    fr s = fr_zero();
    for (int w = 0; w < 8; w++) s = fr_add(s, red[w]);
    st_fr(A.partials + (size_t)item * A.nblk + blockIdx.x, s);
  }
}

struct NttFinalArgs {
  const fr* partials;
  uint32_t nblk;
  int c;
  uint32_t gate, n, d, logm;
  fr ninv_l1;
  const uint8_t* qroot;
  NttState* st;
  uint8_t* proof;
};

__global__ void k_ntt_final(NttFinalArgs A) {
  // one warp per opening: lanes add strided block partials, then shuffles
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int item = threadIdx.x >> 5; item <= A.c; item += nw) {
    fr s = fr_zero();
    for (uint32_t b = lane; b < A.nblk; b += 32) s = fr_add(s, ld_fr_cg(A.partials + (size_t)item * A.nblk + b));
    s = warp_sum(s);
    if (lane == 0) {
      if (item < A.c) s = fr_mul(s, A.ninv_l1);  // coefficients carry the factor N
      uint8_t* o = A.proof + 52 + 32 * item;
      for (int i = 0; i < 8; i++)
        for (int b = 0; b < 4; b++) o[4 * i + b] = (uint8_t)(s.v[i] >> (8 * b));
    }
  }
  if (threadIdx.x == 0) {
    const char* mg = A.st->err ? "ZCE!" : "ZCN1";
    for (int b = 0; b < 4; b++) A.proof[b] = (uint8_t)mg[b];
    uint32_t hv[4] = {A.gate, A.n, A.d, A.logm};
    for (int q = 0; q < 4; q++)
      for (int b = 0; b < 4; b++) A.proof[4 + 4 * q + b] = (uint8_t)(hv[q] >> (8 * b));
    for (int b = 0; b < 32; b++) A.proof[20 + b] = A.qroot[b];
  }
}

__global__ void k_ntt_state_init(NttState* st) {
  if (threadIdx.x == 0) st->err = 0;
}

// ------------------------------------------------------------------ host --

static zc_status ensure_tables(zc_ctx* ctx, cudaStream_t st, NttTables** out) {
  std::lock_guard<std::mutex> lk(g_tabs_mu);
  NttTables& T = g_tabs_by_dev[ctx->device];
  if (!T.ready) {
    const size_t n4 = 4096, n15 = 1u << kLoBits;
    size_t bytes = sizeof(fr) * (2 * n4 + 8 * n15);
    if (cudaMalloc(&T.mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "cudaMalloc NTT tables";
      return ZC_ERR_OOM;
    }
    fr* p = static_cast<fr*>(T.mem);
    T.dft_fwd = p; p += n4;
    T.dft_inv = p; p += n4;
    T.wf_lo = p; p += n15;
    T.wf_hi = p; p += n15;
    T.wi_lo = p; p += n15;
    T.wi_hi = p; p += n15;
    T.s7_lo = p; p += n15;
    T.s7_hi = p; p += n15;
    T.p7_lo = p; p += n15;
    T.p7_hi = p; p += n15;
    const DevConst& C = ctx->hconst;
    // w_2^32 = 7^((r-1)/2^32); w_2^30 = (w_2^32)^4
    uint32_t e[8];
    for (int i = 0; i < 7; i++) e[i] = p_limb(i + 1);
    e[7] = 0;
    fr seven = h_from_u64(7);
    fr acc = h_from_u64(1), base = seven;
    for (int i = 0; i < 8; i++)
      for (int b = 0; b < 32; b++) {
        if ((e[i] >> b) & 1) acc = h_canon_mul(acc, base, C);
        base = h_canon_mul(base, base, C);
      }
    T.w32h = acc;
    fr w30 = h_canon_mul(acc, acc, C);
    w30 = h_canon_mul(w30, w30, C);
    NttTabArgs a{};
    a.dft_fwd = T.dft_fwd; a.dft_inv = T.dft_inv;
    a.wf_lo = T.wf_lo; a.wf_hi = T.wf_hi; a.wi_lo = T.wi_lo; a.wi_hi = T.wi_hi;
    a.s7_lo = T.s7_lo; a.s7_hi = T.s7_hi;
    a.p7_lo = T.p7_lo; a.p7_hi = T.p7_hi;
    a.w30 = fr_mul_g(w30, C.r2);
    a.w30i = fr_mul_g(h_inv(w30, C), C.r2);
    a.seveninv = fr_mul_g(h_inv(seven, C), C.r2);
    a.C = ctx->dconst;
    k_ntt_tables<<<(n15 + 255) / 256, 256, 0, st>>>(a);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      ctx->err = "NTT table set-up failed";
      return ZC_ERR_CUDA;
    }
    T.ready = true;
  }
  *out = &T;
  return ZC_OK;
}

// Pass kernel variants: tile of 2^logTile elements (TILE / 8 threads, each
// owning 8 elements per stage) and a minimum number of resident CTAs per SM
// (caps registers).  The context's tuning picks the tile and residency.
template <int TILE, int MINB>
static void launch_pass_variant(const NttPassArgs& a, dim3 grid, cudaStream_t st) {
  k_ntt_pass<TILE, MINB><<<grid, TILE / 8, TILE * sizeof(fr), st>>>(a);
}

static void set_pass_attributes() {
  cudaFuncSetAttribute(k_ntt_pass<1024, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 1024 * 32);
  cudaFuncSetAttribute(k_ntt_pass<2048, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2048 * 32);
  cudaFuncSetAttribute(k_ntt_pass<2048, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2048 * 32);
  cudaFuncSetAttribute(k_ntt_pass<4096, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * 32);
}

static int g_attr_done[64] = {0};
static void ensure_pass_attributes(int dev) {
  std::lock_guard<std::mutex> lk(g_tabs_mu);
  if (!g_attr_done[dev]) {
    set_pass_attributes();
    g_attr_done[dev] = 1;
  }
}

// launch one batched pass over `items` columns
static zc_status run_pass(zc_ctx* ctx, cudaStream_t st, NttPassArgs& a, int items, uint64_t B) {
  const uint32_t logL = a.logL;
  uint32_t logTile = (uint32_t)ctx->tuned(ZC_FORM_NTT, ctx->cur_n, ZC_TUNE_NTT_TILE_LOG);
  const int minb = ctx->tuned(ZC_FORM_NTT, ctx->cur_n, ZC_TUNE_NTT_MINB);
  if (logTile < logL) logTile = logL < 10 ? 10 : logL;
  if (logTile > 12) logTile = 12;
  if (logTile < 10) logTile = 10;
  a.logW = logTile - logL;
  while (a.logW > 0 && (1ull << a.logW) > B) a.logW--;
  const uint64_t W = 1ull << a.logW;
  const uint64_t blocks = (B + W - 1) / W;
  if (B % W) {
    ctx->err = "NTT pass: batch not a multiple of the tile";
    return ZC_ERR_ARG;
  }
  a.items = (uint32_t)items;
  dim3 grid((unsigned)(blocks * (uint64_t)items));
  if (logTile == 12) launch_pass_variant<4096, 1>(a, grid, st);
  else if (logTile == 11 && minb != 1) launch_pass_variant<2048, 2>(a, grid, st);
  else if (logTile == 11) launch_pass_variant<2048, 1>(a, grid, st);
  else launch_pass_variant<1024, 4>(a, grid, st);
  ctx->launches++;
  return ZC_OK;
}

// The per-size tables of (n, lb), built on first use; nullptr when they
// would exceed the context's table budget (the passes then form every factor
// from the two-level power tables instead).
static zc_ctx::NttSizeTables* size_tables(zc_ctx* user, const NttTables* T, uint32_t n, uint32_t lb,
                                          uint32_t l1, uint32_t l2, cudaStream_t st) {
  zc_ctx* ctx = user->table_owner ? user->table_owner : user;
  const uint64_t N = 1ull << n, M = N << lb;
  for (auto& e : ctx->ntt_cache)
    if (e.n == n && e.lb == lb && e.l1 == l1) {
      e.stamp = ++ctx->ntt_cache_clock;
      return &e;
    }
  const uint64_t s = 1ull << lb;
  const size_t bytes = sizeof(fr) * (2 * N + 3 * M + s);
  if (ctx->ntt_cache_frozen || bytes > ctx->ntt_cache_budget) return nullptr;
  size_t used = 0;
  for (auto& e : ctx->ntt_cache) used += e.bytes + e.step_bytes;
  while (!ctx->ntt_cache.empty() && used + bytes > ctx->ntt_cache_budget) {
    size_t old = 0;
    for (size_t i = 1; i < ctx->ntt_cache.size(); i++)
      if (ctx->ntt_cache[i].stamp < ctx->ntt_cache[old].stamp) old = i;
    cudaStreamSynchronize(st);
    cudaFree(ctx->ntt_cache[old].mem);
    if (ctx->ntt_cache[old].step_mem) cudaFree(ctx->ntt_cache[old].step_mem);
    used -= ctx->ntt_cache[old].bytes + ctx->ntt_cache[old].step_bytes;
    ctx->ntt_cache.erase(ctx->ntt_cache.begin() + old);
  }
  zc_ctx::NttSizeTables e;
  if (cudaMalloc(&e.mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  e.n = n;
  e.lb = lb;
  e.l1 = l1;
  e.bytes = bytes;
  fr* q = static_cast<fr*>(e.mem);
  e.tw_fwd = q; q += N;
  e.tw_inv = q; q += N;
  e.coset = q; q += M;
  e.outer = q; q += M;
  e.fin = q; q += M;
  e.zinv = q;
  {
    // (z_H on slice j)^-1 M^-1 = (7^N w_s^j - 1)^-1 M^-1, level 1, on the host
    const DevConst& C = ctx->hconst;
    const fr ws = h_pow(T->w32h, (1ull << 32) >> lb, C);
    const fr s7n = h_pow(h_from_u64(7), N, C), minv = h_inv(h_from_u64(M), C);
    std::vector<fr> zi(s);
    fr wj = h_from_u64(1);
    for (uint64_t j = 0; j < s; j++) {
      const fr v = fr_sub_g(h_canon_mul(s7n, wj, C), h_from_u64(1));
      zi[j] = h_canon_mul(h_canon_mul(h_inv(v, C), minv, C), C.one, C);
      wj = h_canon_mul(wj, ws, C);
    }
    if (cudaMemcpyAsync(e.zinv, zi.data(), sizeof(fr) * s, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(e.mem);
      return nullptr;
    }
  }
  NttSizeArgs a{};
  a.tw_fwd = e.tw_fwd;
  a.tw_inv = e.tw_inv;
  a.coset = e.coset;
  a.outer = e.outer;
  a.fin = e.fin;
  a.n = n;
  a.lb = lb;
  a.l1 = l1;
  a.l2 = l2;
  const DevConst& C = ctx->hconst;
  a.ninv_l2 = fr_mul_g(fr_mul_g(h_inv(h_from_u64(N), C), C.r2), C.r2);
  a.C = ctx->dconst;
  const uint64_t total = 2 * N + 3 * M;
  k_ntt_size_tables<<<(unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->sm_count * 16), 256, 0,
                      st>>>(a, *T);
  ctx->launches++;
  e.stamp = ++ctx->ntt_cache_clock;
  ctx->ntt_cache.push_back(e);
  return &ctx->ntt_cache.back();
}

static void pass_defaults(NttPassArgs& a) {
  std::memset(&a, 0, sizeof a);
  a.in_lbdiv = 63;
  a.out_lbdiv = 63;
}

static NttDomain domain_of(const zc_params* p) {
  NttDomain D;
  ntt_domain(p->n, p->d, p->log_blowup, &D);  // validated by check_params
  return D;
}

size_t ntt_scratch_bytes(const zc_params* p, int sm_count, bool q_direct) {
  const NttDomain D = domain_of(p);
  const uint32_t n = p->n, lb = D.k;
  const int c = gate_ncols(p->gate, p->d);
  const uint64_t N = 1ull << n, Mb = N << lb, s = 1ull << lb, M = D.M;
  const uint32_t hbits = (n + 1) / 2;
  const uint32_t nlo = 1u << hbits, nhi = 1u << (n - hbits);
  const uint32_t nblk_open = 2 * (uint32_t)sm_count;
  const size_t psize = 20 + 32 + 32 * ((size_t)c + 1);
  size_t need = 2 * align_up(sizeof(fr) * N, 256) * c;  // coefficients + slice buffer
  need += align_up(sizeof(fr) * M, 256);                  // qhat (both parts)
  if (!q_direct) need += align_up(sizeof(fr) * M, 256);   // q
  if (D.step) need += 2 * align_up(sizeof(fr) * N, 256);  // q_big reduced, and its LDE
  need += align_up(sizeof(fr) * s * (nlo + nhi), 256) + align_up(sizeof(fr) * s, 256);
  need += align_up(sizeof(fr) * (c + 1) * nblk_open, 256) + align_up(sizeof(fr) * 32, 256);
  need += align_up(sizeof(NttState), 256) + align_up(psize, 256) + align_up(32 * (size_t)(c + 1), 256);
  need += root_scratch_bytes(c, N) + root_scratch_bytes(1, M) + 8192;
  (void)Mb;
  return need;
}

// Side stream and per-column events for pipelined uploads of host columns
// (created on first use, freed by zc_destroy).
zc_status ensure_upload_stream(zc_ctx* ctx, int c) {
  if (!ctx->up_stream) {
    if (cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->up_fork, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "cannot create the upload stream";
      return ZC_ERR_CUDA;
    }
  }
  while ((int)ctx->up_ev.size() < c) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "cannot create an upload event";
      return ZC_ERR_CUDA;
    }
    ctx->up_ev.push_back(e);
  }
  return ZC_OK;
}

// Transforms of 2^n points run as two four-step passes (sub-DFTs of
// 2^ceil(n/2) and 2^floor(n/2) points) from n = 12 on (a single pass holds at
// most 2^12 points; at 2^12 the two passes' extra CTAs already win), or from
// a tuned size, else as one pass per transform.
static bool ntt_two_pass(const zc_ctx* ctx, uint32_t n) {
  if (n > 12) return true;  // one pass holds at most a 2^12 transform
  const int32_t t = ctx->tuned(ZC_FORM_NTT, n, ZC_TUNE_NTT_TWO_LOG);
  return n >= (uint32_t)(t > 0 ? t : 12) && n >= 2;
}

// The step-radix tables of a cache entry (lb = k): built once, with the
// host-computed constants of the small part.  False if they cannot be made.
static bool step_tables(zc_ctx* user, zc_ctx::NttSizeTables* e, const NttTables* T, cudaStream_t st) {
  if (e->step_mem) return true;
  zc_ctx* ctx = user->table_owner ? user->table_owner : user;
  if (ctx->ntt_cache_frozen) return false;
  const uint32_t n = e->n, lb = e->lb;
  const uint64_t N = 1ull << n, M = N << lb, parts = 1ull << lb;
  if (n + lb + 1 > (uint32_t)kLog30 || parts > 64) return false;
  const size_t nconst = 8 + parts;
  const size_t bytes = sizeof(fr) * (2 * N + nconst);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  fr* q = static_cast<fr*>(mem);
  fr* coset = q;
  fr* unscale = q + N;
  fr* cst = q + 2 * N;
  const DevConst& C = ctx->hconst;
  // sigma = 7 w_{2M}; kappa = sigma^M - 7^M; z_H on D_small = sigma^N - 1
  const fr w2m = h_pow(T->w32h, (1ull << 32) >> (n + lb + 1), C);
  const fr seven = h_from_u64(7), one = h_from_u64(1);
  const fr sigma = h_canon_mul(seven, w2m, C);
  const fr s7m = h_pow(seven, M, C);
  const fr kinv = h_inv(fr_sub_g(h_pow(sigma, M, C), s7m), C);
  const fr ninv = h_inv(h_from_u64(N), C);
  const fr sn = h_pow(sigma, N, C);
  std::vector<fr> hc(nconst, fr_zero());
  hc[0] = h_canon_mul(h_canon_mul(h_canon_mul(h_inv(fr_sub_g(sn, one), C), kinv, C), ninv, C), C.one, C);
  hc[1] = h_canon_mul(s7m, C.one, C);
  fr pm = one;
  for (uint64_t m = 0; m < parts; m++) {
    hc[8 + m] = h_canon_mul(h_canon_mul(pm, kinv, C), C.one, C);  // level 1
    pm = h_canon_mul(pm, sn, C);
  }
  if (cudaMemcpyAsync(cst, hc.data(), sizeof(fr) * nconst, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(mem);
    return false;
  }
  NttStepTabArgs a{};
  a.coset = coset;
  a.unscale = unscale;
  a.n = n;
  a.shift2m = kLog30 - (n + lb + 1);
  a.ninv_l2 = fr_mul_g(fr_mul_g(ninv, C.r2), C.r2);
  a.T = *T;
  k_ntt_step_tables<<<(unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)ctx->sm_count * 16), 256, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) {
    cudaFree(mem);
    return false;
  }
  e->step_mem = mem;
  e->step_bytes = bytes;
  e->step_coset = coset;
  e->step_unscale = unscale;
  e->step_const = cst;
  user->launches++;
  return true;
}

// ---- Reed-Solomon row encoding for the hash-based commitment (zc_pcs.cu):
// row i of column j (w = 2^nc coefficients) evaluated at the W = 4w points
// 7 w_W^k, written to enc[j][k m + i].  Slice s (k = s + 4 k') is one pass
// of w-point transforms over the m rows with the factor (7 w_W^s)^l applied
// on load; canonical columns in, canonical codewords out.

struct PcsTabArgs {
  fr* tab;            // [s w + l] = (7 w_W^s)^l, level 1
  uint32_t nc;        // w = 2^nc
  uint32_t shiftW;    // 30 - log2 W
  NttTables T;
};

__global__ void k_pcs_tables(PcsTabArgs A) {
  const uint32_t w = 1u << A.nc, total = 4 * w;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const uint32_t s = e >> A.nc, l = e & (w - 1);
    const fr p7 = fr_mul(ld_fr(A.T.p7_hi + (l >> kLoBits)), ld_fr(A.T.p7_lo + (l & kLoMask)));  // 7^l
    const uint32_t ex = (uint32_t)((((uint64_t)s * l) << A.shiftW) & ((1ull << kLog30) - 1));
    st_fr(A.tab + e, fr_mul(p7, root_pow(A.T.wf_lo, A.T.wf_hi, ex)));
  }
}

zc_status pcs_encode(zc_ctx* ctx, const fr* const* cols, int c, uint32_t nr, uint32_t nc, fr* const* enc,
                     fr* tab, cudaStream_t st) {
  if (nc < 1 || nc > 12 || c < 1 || c > kMaxCols) {
    ctx->err = "pcs: rows of 2 .. 2^12 elements";
    return ZC_ERR_UNSUPPORTED;
  }
  ensure_pass_attributes(ctx->device);
  NttTables* T = nullptr;
  zc_status s0 = ensure_tables(ctx, st, &T);
  if (s0 != ZC_OK) return s0;
  const uint64_t w = 1ull << nc, m = 1ull << nr;
  PcsTabArgs ta{};
  ta.tab = tab;
  ta.nc = nc;
  ta.shiftW = kLog30 - (nc + 2);
  ta.T = *T;
  k_pcs_tables<<<(unsigned)std::min<uint64_t>((4 * w + 255) / 256, 1024), 256, 0, st>>>(ta);
  ctx->launches++;
  ctx->cur_n = nc;
  for (uint32_t sl = 0; sl < 4; sl++) {
    NttPassArgs a;
    pass_defaults(a);
    for (int j = 0; j < c; j++) {
      a.in[j] = cols[j];
      a.out[j] = enc[j] + sl * m;     // position k = sl + 4 k'
    }
    a.logL = nc;
    a.in_bs_lo = w; a.in_ts = 1;      // row b, coefficient t
    a.out_bs_lo = 1; a.out_ts = 4 * m;
    a.dft = T->dft_fwd;
    a.pre = PRE_TAB; a.pre_tab = tab + sl * w;
    a.pre_kb = 0; a.pre_kt = 1;
    zc_status rs = run_pass(ctx, st, a, c, m);
    if (rs != ZC_OK) return rs;
  }
  return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

zc_status ntt_prepare(zc_ctx* ctx, const zc_params* p, cudaStream_t st) {
  ensure_pass_attributes(ctx->device);
  NttTables* T = nullptr;
  zc_status s0 = ensure_tables(ctx, st, &T);
  if (s0 != ZC_OK) return s0;
  const NttDomain D = domain_of(p);
  const uint32_t n = p->n, lb = D.k;
  const bool two = ntt_two_pass(ctx, n);
  zc_ctx::NttSizeTables* ST = size_tables(ctx, T, n, lb, two ? (n + 1) / 2 : n, two ? n / 2 : 0, st);
  if (D.step && (!ST || !step_tables(ctx, ST, T, st))) {
    ctx->err = "step-radix domain: tables unavailable";
    return ZC_ERR_OOM;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

zc_status ntt_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                    const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                    bool proof_on_dev, void* q_out, int q_on_dev) {
  const uint32_t gate = p->gate, n = p->n, d = p->d;
  ctx->cur_n = n;
  if (n > (uint32_t)kMaxNttN) {
    ctx->err = "NTT form supports n <= 24";
    return ZC_ERR_UNSUPPORTED;
  }
  const NttDomain D = domain_of(p);
  if (D.step && D.s != 0) {
    ctx->err = "step-radix domains take a small part of N points (s = 0)";
    return ZC_ERR_UNSUPPORTED;
  }
  const uint32_t lb = D.k;          // the big part 7 <w_Mb>, Mb = 2^lb N
  const uint32_t logm = n + lb;     // log2 Mb
  if (logm + (D.step ? 1 : 0) > (uint32_t)kLog30) {
    ctx->err = "domain larger than 2^30";
    return ZC_ERR_UNSUPPORTED;
  }
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n, Mb = 1ull << logm, s = 1ull << lb;
  const uint64_t M = D.M;           // Mb, or Mb + N (step radix)
  const size_t psize = 20 + 32 + 32 * ((size_t)c + 1);
  ensure_pass_attributes(ctx->device);
  NttTables* T = nullptr;
  zc_status s0 = ensure_tables(ctx, st, &T);
  if (s0 != ZC_OK) return s0;

  const uint32_t hbits = (n + 1) / 2;
  const uint32_t nlo = 1u << hbits, nhi = 1u << (n - hbits);
  const uint32_t nblk_open = 2 * (uint32_t)ctx->sm_count;
  const bool q_direct = q_out && q_on_dev;
  zc_status s1 = ensure_arena(ctx, ntt_scratch_bytes(p, ctx->sm_count, q_direct));
  if (s1 != ZC_OK) return s1;
  Arena& ar = ctx->arena;
  ar.reset();
  fr* coef[kMaxCols];
  fr* slb[kMaxCols];
  for (int j = 0; j < c; j++) coef[j] = ar.take<fr>(N);
  for (int j = 0; j < c; j++) slb[j] = ar.take<fr>(N);
  fr* qhat = ar.take<fr>(M);
  fr* qv = q_direct ? static_cast<fr*>(q_out) : ar.take<fr>(M);
  fr* rho = D.step ? ar.take<fr>(N) : nullptr;   // q_big reduced mod x^N - sigma^N
  fr* vsm = D.step ? ar.take<fr>(N) : nullptr;   // its values on D_small
  fr* tlo = ar.take<fr>(s * nlo);
  fr* thi = ar.take<fr>(s * nhi);
  fr* zinv = ar.take<fr>(s);
  fr* opart = ar.take<fr>((size_t)(c + 1) * nblk_open);
  fr* zpow = ar.take<fr>(32);
  NttState* dstate = ar.take<NttState>(1);
  uint8_t* dproof = ar.take<uint8_t>(psize);
  uint8_t* droots = ar.take<uint8_t>(32 * (size_t)(c + 1));
  if (!droots) {
    ctx->err = "scratch arena too small";
    return ZC_ERR_OOM;
  }
  ctx->launches = 0;
  ctx->nev = 7;

  const bool two = ntt_two_pass(ctx, n);
  const uint32_t l1 = two ? (n + 1) / 2 : n;   // first digit
  const uint32_t l2 = two ? n / 2 : 0;         // second digit
  const uint64_t L1 = 1ull << l1, L2 = 1ull << l2;
  zc_status rs;
  zc_ctx::NttSizeTables* ST = size_tables(ctx, T, n, lb, l1, l2, st);
  if (D.step && (!ST || !step_tables(ctx, ST, T, st))) {
    ctx->err = "step-radix domain: per-size tables unavailable";
    return ZC_ERR_OOM;
  }

  // N1's first pass (rows over i2, twiddled) for the columns [j0, j1)
  auto n1_first = [&](const fr* const* in, int j0, int j1) -> zc_status {
    NttPassArgs a;
    pass_defaults(a);
    for (int j = j0; j < j1; j++) {
      a.in[j - j0] = in[j];
      a.out[j - j0] = coef[j];
    }
    a.logL = l2;                       // rows of length L2 over i2
    a.in_bs_lo = 1; a.in_ts = L1;      // element (i1, i2) read from e[i1 + L1 i2]
    a.out_bs_lo = L2; a.out_ts = 1;
    a.dft = T->dft_inv;
    a.err = &dstate->err;              // every input element passes through here once
    a.post = POST_TW; a.tw_lo = T->wi_lo; a.tw_hi = T->wi_hi;
    a.tw_lbmod = l1; a.tw_shift = kLog30 - n;
    if (ST) {  // w_N^-(i1 k2) = tw_inv[i1 L2 + k2]
      a.post = POST_TAB; a.post_tab = ST->tw_inv;
      a.p_lbdiv = 63; a.p_ls = L2; a.p_ts = 1;
    }
    return run_pass(ctx, st, a, j1 - j0, L1);
  };
  // N1's second pass (columns of length L1, in place) for the columns [j0, j1)
  auto n1_second = [&](int j0, int j1) -> zc_status {
    NttPassArgs a;
    pass_defaults(a);
    for (int j = j0; j < j1; j++) {
      a.in[j - j0] = coef[j];
      a.out[j - j0] = coef[j];
    }
    a.logL = l1;
    a.in_bs_lo = 1; a.in_ts = L2;
    a.out_bs_lo = 1; a.out_ts = L2;
    a.dft = T->dft_inv;
    return run_pass(ctx, st, a, j1 - j0, L2);
  };

  k_ntt_state_init<<<1, 32, 0, st>>>(dstate);
  ctx->launches++;

  // Host columns: uploaded one by one on a side stream; with two passes the
  // first N1 pass of column j starts as soon as column j has arrived.
  const fr* src[kMaxCols];
  const bool pipelined = !on_dev && two;
  if (on_dev) {
    for (int j = 0; j < c; j++) src[j] = static_cast<const fr*>(cols[j]);
  } else if (pipelined) {
    zc_status us = ensure_upload_stream(ctx, c);
    if (us != ZC_OK) return us;
    ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->up_fork, st));
    ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->up_stream, ctx->up_fork, 0));
    for (int j = 0; j < c; j++) {
      ZC_CUDA_TRY(ctx, cudaMemcpyAsync(slb[j], cols[j], N * sizeof(fr), cudaMemcpyHostToDevice,
                                       ctx->up_stream));
      ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->up_ev[j], ctx->up_stream));
      src[j] = slb[j];
    }
    for (int j = 0; j < c; j++) {
      ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->up_ev[j], 0));
      if ((rs = n1_first(src, j, j + 1)) != ZC_OK) return rs;
    }
  } else {
    for (int j = 0; j < c; j++) {
      ZC_CUDA_TRY(ctx, cudaMemcpyAsync(slb[j], cols[j], N * sizeof(fr), cudaMemcpyHostToDevice, st));
      src[j] = slb[j];
    }
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], st));
  if (roots) {
    std::memcpy(ctx->pinned, roots, 32 * (size_t)c);
    ZC_CUDA_TRY(ctx, cudaMemcpyAsync(droots, ctx->pinned, 32 * (size_t)c, cudaMemcpyHostToDevice, st));
  } else {
    zc_status rs = launch_roots(ctx, src, c, N, droots, st);
    if (rs != ZC_OK) return rs;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], st));

  // per-slice coset tables and z_H inverses (only without per-size tables)
  const DevConst& C = ctx->hconst;
  fr ninv = h_inv(h_from_u64(N), C), minv = h_inv(h_from_u64(M), C);
  if (!ST) {
    NttSliceTabArgs ta{};
    ta.lo = tlo;
    ta.hi = thi;
    ta.zinv = zinv;
    ta.s = (uint32_t)s;
    ta.n = n;
    ta.hbits = hbits;
    ta.logm = logm;
    ta.ninv_l2 = fr_mul_g(fr_mul_g(ninv, C.r2), C.r2);
    ta.minv_l1 = fr_mul_g(minv, C.r2);
    ta.wf_lo = T->wf_lo;
    ta.wf_hi = T->wf_hi;
    ta.C = ctx->dconst;
    uint64_t tot = s * (nlo + nhi);
    k_ntt_slice_tables<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ta);
    ctx->launches++;
  }

  // ---- N1: g_j = DFT^-1(e_j) (the factor 1/N is applied later), natural out
  if (two) {
    if (!pipelined && (rs = n1_first(src, 0, c)) != ZC_OK) return rs;
    if ((rs = n1_second(0, c)) != ZC_OK) return rs;  // all columns in one launch
  } else {
    NttPassArgs a;
    pass_defaults(a);
    for (int j = 0; j < c; j++) {
      a.in[j] = src[j];
      a.out[j] = coef[j];
    }
    a.logL = n;
    a.in_bs_lo = 0; a.in_ts = 1;
    a.out_bs_lo = 0; a.out_ts = 1;
    a.dft = T->dft_inv;
    a.err = &dstate->err;
    if ((rs = run_pass(ctx, st, a, c, 1)) != ZC_OK) return rs;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], st));

  // ---- N2: per slice, coset NTT of every column, gate, divide by z_H.
  // slice_lde: the coset NTT of the `items` coefficient vectors in[] into
  // out[] on one slice, with the coset factor table pre (per-size tables)
  // or slice j's two-level tables (without them).
  auto slice_lde = [&](const fr* const* in, fr* const* out, int items, const fr* pre, uint64_t j,
                       bool mark) -> zc_status {
    NttPassArgs a;
    pass_defaults(a);
    for (int i = 0; i < items; i++) {
      a.in[i] = in[i];
      a.out[i] = out[i];
    }
    a.pre = PRE_COSET;
    a.pre_lo = tlo + j * nlo;
    a.pre_hi = thi + j * nhi;
    a.pre_shift = hbits;
    a.dft = T->dft_fwd;
    if (two) {
      a.logL = l1;                     // columns over k1: k = L2 k1 + k2
      a.in_bs_lo = 1; a.in_ts = L2;
      a.out_bs_lo = 1; a.out_ts = L2;
      a.pre_kb = 1; a.pre_kt = L2;
      a.post = POST_TW; a.tw_lo = T->wf_lo; a.tw_hi = T->wf_hi;
      a.tw_lbmod = l2; a.tw_shift = kLog30 - n;
      if (ST) {  // coset factor of k = k2 + L2 k1; twiddle w_N^(k2 i1) = tw_fwd[k2 L1 + i1]
        a.pre = PRE_TAB; a.pre_tab = pre;
        a.post = POST_TAB; a.post_tab = ST->tw_fwd;
        a.p_lbdiv = 63; a.p_ls = L1; a.p_ts = 1;
      }
      if ((rs = run_pass(ctx, st, a, items, L2)) != ZC_OK) return rs;
      if (mark) ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[7], st));
      pass_defaults(a);
      for (int i = 0; i < items; i++) {
        a.in[i] = out[i];
        a.out[i] = out[i];
      }
      a.logL = l2;                     // rows over k2
      a.in_bs_lo = L2; a.in_ts = 1;
      a.out_bs_lo = L2; a.out_ts = 1;
      a.dft = T->dft_fwd;
      if ((rs = run_pass(ctx, st, a, items, L1)) != ZC_OK) return rs;
    } else {
      a.logL = n;
      a.in_bs_lo = 0; a.in_ts = 1;
      a.out_bs_lo = 0; a.out_ts = 1;
      a.pre_kb = 0; a.pre_kt = 1;
      if (ST) {
        a.pre = PRE_TAB; a.pre_tab = pre;
      }
      if ((rs = run_pass(ctx, st, a, items, 1)) != ZC_OK) return rs;
      if (mark) ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[7], st));
    }
    return ZC_OK;
  };
  // gate and division by z_H (constant zi on the slice), minus sub if given
  auto slice_gate = [&](fr* out, const fr* zi, const fr* sub) {
    NttGateArgs ga{};
    for (int i = 0; i < c; i++) ga.col[i] = slb[i];
    ga.qhat = out;
    ga.zinv = zi;
    ga.sub = sub;
    ga.N = N;
    ga.gate = gate;
    ga.d = d;
    ga.c = (uint32_t)c;
    uint32_t gb = (uint32_t)std::min<uint64_t>((N + 255) / 256, (uint64_t)ctx->sm_count * 8);
    k_ntt_gate<<<gb, 256, 0, st>>>(ga);
    ctx->launches++;
  };
  for (uint64_t j = 0; j < s; j++) {
    if ((rs = slice_lde(coef, slb, c, ST ? ST->coset + j * N : nullptr, j, j == 0)) != ZC_OK) return rs;
    slice_gate(qhat + j * N, (ST ? ST->zinv : zinv) + j, nullptr);
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[3], st));

  // ---- N3: q = 7^-k M^-1 DFT_M^-1(qhat), digits (s, L1, L2) or (s, N).
  // inverse: the INTT of ns = 2^lbs slices qin[] into qout[] (natural
  // order, with the factor 7^-k; M^-1 came with the slice constants).
  auto inverse = [&](fr* qin, fr* qout, uint64_t s, uint32_t lb, uint32_t logm) -> zc_status {
  {
    NttPassArgs a;
    if (two) {
      pass_defaults(a);
      a.in[0] = qin; a.out[0] = qin;
      a.logL = l2;                     // rows (j, i2) over i3
      a.in_bs_lo = L2; a.in_ts = 1;
      a.out_bs_lo = L2; a.out_ts = 1;
      a.dft = T->dft_inv;
      a.post = POST_TW; a.tw_lo = T->wi_lo; a.tw_hi = T->wi_hi;
      a.tw_lbmod = l1; a.tw_shift = kLog30 - n;
      if (ST) {  // w_N^-(i2 k3) = tw_inv[(b mod L1) L2 + k3]
        a.post = POST_TAB; a.post_tab = ST->tw_inv;
        a.p_lbdiv = l1; a.p_hs = 0; a.p_ls = L2; a.p_ts = 1;
      }
      if ((rs = run_pass(ctx, st, a, 1, s * L1)) != ZC_OK) return rs;
      pass_defaults(a);
      a.in[0] = qin; a.out[0] = qin;
      a.logL = l1;                     // columns (j, k3) over i2 within a slice
      a.in_lbdiv = l2; a.in_bs_hi = N; a.in_bs_lo = 1; a.in_ts = L2;
      a.out_lbdiv = l2; a.out_bs_hi = N; a.out_bs_lo = 1; a.out_ts = L2;
      a.dft = T->dft_inv;
      a.post = POST_OUTER; a.tw_lo = T->wi_lo; a.tw_hi = T->wi_hi;
      a.outer_lbdiv = l2; a.tw_shift = kLog30 - logm;
      if (ST) {  // w_M^-(j k'), k' = L2 k2 + k3: outer[j N + k']
        a.post = POST_TAB; a.post_tab = ST->outer;
        a.p_lbdiv = l2; a.p_hs = N; a.p_ls = 1; a.p_ts = L2;
      }
      if ((rs = run_pass(ctx, st, a, 1, s * L2)) != ZC_OK) return rs;
    } else {
      pass_defaults(a);
      a.in[0] = qin; a.out[0] = qin;
      a.logL = n;                      // one row per slice
      a.in_bs_lo = N; a.in_ts = 1;
      a.out_bs_lo = N; a.out_ts = 1;
      a.dft = T->dft_inv;
      a.post = POST_OUTER; a.tw_lo = T->wi_lo; a.tw_hi = T->wi_hi;
      a.outer_lbdiv = 0; a.tw_shift = kLog30 - logm;
      if (ST) {
        a.post = POST_TAB; a.post_tab = ST->outer;
        a.p_lbdiv = 63; a.p_ls = N; a.p_ts = 1;
      }
      if ((rs = run_pass(ctx, st, a, 1, s)) != ZC_OK) return rs;
    }
    pass_defaults(a);
    a.in[0] = qin; a.out[0] = qout;
    a.logL = lb;                       // across slices
    a.in_bs_lo = 1; a.in_ts = N;
    a.out_bs_lo = 1; a.out_ts = N;
    a.dft = T->dft_inv;
    a.post = POST_FINAL; a.tw_lo = T->s7_lo; a.tw_hi = T->s7_hi;
    a.fin_N = N;
    if (ST) {  // 7^-k, k = N t + b
      a.post = POST_TAB; a.post_tab = ST->fin;
      a.p_lbdiv = 63; a.p_ls = 1; a.p_ts = N;
    }
    if ((rs = run_pass(ctx, st, a, 1, N)) != ZC_OK) return rs;
  }
    return ZC_OK;
  };
  if ((rs = inverse(qhat, qv, s, lb, logm)) != ZC_OK) return rs;
  if (D.step) {
    // q_big on D_small (reduce, then the slice LDE with sigma's factors),
    // the small part's gate minus it, its INTT, and q = q_big + (x^Mb -
    // 7^Mb) q_small.
    NttStepReduceArgs ra{};
    ra.q = qv;
    ra.rho = rho;
    ra.cm = ST->step_const + 8;
    ra.N = N;
    ra.parts = (uint32_t)s;
    const unsigned eg = (unsigned)std::min<uint64_t>((N + 255) / 256, (uint64_t)ctx->sm_count * 8);
    k_ntt_step_reduce<<<eg, 256, 0, st>>>(ra);
    ctx->launches++;
    const fr* rin[1] = {rho};
    fr* rout[1] = {vsm};
    if ((rs = slice_lde(rin, rout, 1, ST->step_coset, 0, false)) != ZC_OK) return rs;
    if ((rs = slice_lde(coef, slb, c, ST->step_coset, 0, false)) != ZC_OK) return rs;
    slice_gate(qhat + Mb, ST->step_const, vsm);
    if ((rs = inverse(qhat + Mb, qv + Mb, 1, 0, n)) != ZC_OK) return rs;
    NttStepCombineArgs ca{};
    ca.q = qv;
    ca.unscale = ST->step_unscale;
    ca.s7m = ST->step_const + 1;
    ca.N = N;
    ca.M = Mb;
    k_ntt_step_combine<<<eg, 256, 0, st>>>(ca);
    ctx->launches++;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[4], st));
  // a host q leaves on the side stream while the root and the openings run
  const bool q_async = q_out && !q_direct && !q_on_dev;
  if (q_async) {
    zc_status us = ensure_upload_stream(ctx, 1);
    if (us != ZC_OK) return us;
    ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->up_stream, ctx->ev[4], 0));
    ZC_CUDA_TRY(ctx, cudaMemcpyAsync(q_out, qv, M * sizeof(fr), cudaMemcpyDeviceToHost, ctx->up_stream));
    ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->up_ev[0], ctx->up_stream));
  }

  // ---- N4: root(q), z
  {
    const fr* qp[1] = {qv};
    if ((rs = launch_roots(ctx, qp, 1, M, droots + 32 * (size_t)c, st)) != ZC_OK) return rs;
    NttZArgs za{};
    za.st = dstate;
    za.roots = droots;
    za.c = c;
    za.n = n;
    transcript_init_words(za.S0, ZC_FORM_NTT, gate, n, d, D.word);
    za.zpow = zpow;
    za.C = ctx->dconst;
    k_ntt_z<<<1, 32, 0, st>>>(za);
    ctx->launches++;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[5], st));

  // ---- N5, N6: openings and the proof
  {
    NttOpenArgs oa{};
    for (int j = 0; j < c; j++) {
      oa.x[j] = coef[j];
      oa.len[j] = N;
    }
    oa.x[c] = qv;
    oa.len[c] = M;
    oa.zpow = zpow;
    oa.partials = opart;
    oa.nblk = nblk_open;
    oa.seg = 32 * 128;
    k_ntt_open<<<dim3(nblk_open, c + 1), 256, 0, st>>>(oa, ctx->dconst);
    ctx->launches++;
    NttFinalArgs fa{};
    fa.partials = opart;
    fa.nblk = nblk_open;
    fa.c = c;
    fa.gate = gate;
    fa.n = n;
    fa.d = d;
    fa.logm = D.word;
    fa.ninv_l1 = fr_mul_g(ninv, C.r2);
    fa.qroot = droots + 32 * (size_t)c;
    fa.st = dstate;
    fa.proof = dproof;
    k_ntt_final<<<1, 256, 0, st>>>(fa);
    ctx->launches++;
  }
  ZC_CUDA_TRY(ctx, cudaGetLastError());
  ZC_CUDA_TRY(ctx, cudaMemcpyAsync(proof, dproof, psize,
                                   proof_on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   st));
  if (q_async) {
    ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->up_ev[0], 0));
  } else if (q_out && !q_direct) {
    ZC_CUDA_TRY(ctx, cudaMemcpyAsync(q_out, qv, M * sizeof(fr), cudaMemcpyDeviceToHost, st));
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[6], st));
  // dominant launch: one N2 column pass over all c columns of a slice
  const double Lc = two ? (double)l1 : (double)n;
  ctx->dom_mulmods = (double)c * (double)N / 2 * Lc + (double)c * (double)N;
  ctx->dom_bytes = 2.0 * 32 * c * (double)N;
  ctx->dom_a = 2;
  ctx->dom_b = 7;
  if (!proof_on_dev || !on_dev || (q_out && !q_direct)) {
    ZC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (std::memcmp(proof, "ZCE!", 4) == 0) {
      ctx->err = "column value >= r";
      return ZC_ERR_ARG;
    }
  }
  return ZC_OK;
}

}  // namespace zc
