// zc_sumcheck.cu -- SumCheck-form ZeroCheck prover (Fig. side-by-side-zc,
// right; Sec. 3.3).
//
// Round i sends G_i(t) = sum_{x_{>i}} f_M(alpha_{<i}, t, x_{>i}) eq_r(...),
// t = 0..d+1.  The eq factor splits as
//   eq_r(alpha_{<i}, t, x) = c_i * l_i(t) * eq_{>i}(x),
//   c_i = prod_{j<i} eq(alpha_j, r_j),  l_i(t) = (1-r_i)(1-t) + r_i t,
// so the kernels accumulate H_i(t) = sum_x f(alpha, t, x) eq_{>i}(x) and the
// challenge step scales it.  eq_{>i}(x) is never stored as a full table or
// folded: it is the product of two small factor tables E_hi[x >> m_lo] and
// E_lo[x & (2^m_lo - 1)] (the Build-MLE step of Sec. 3.3 done per round on
// ~sqrt(N) entries).  H_i has degree d; the kernels evaluate it at the points
// {0, 2, ..., d-1} and at infinity (its leading coefficient, the product of
// the slopes), and the challenge step takes H_i(1) from the round identity
// (1-r_i) H_i(0) + r_i H_i(1) = H_{i-1}(alpha_{i-1})  (Sec. 3.4).  Round 1
// evaluates t = 1 as well, because its claimed sum (zero) only holds for a
// satisfying witness and the proof must carry the true values.
//
// Variable order: x_1 is the most significant index bit, so round i pairs
// entries k and k + h and the MLE update T[k] <- T[k] + alpha (T[k+h] - T[k])
// writes the first half in place.  Round i >= 2 fuses the update by
// alpha_{i-1} with the evaluation of round i (Plonk gate).
//
// Storage levels (see zc_field.cuh): Plonk selectors stay canonical (level
// 0), the wires a, b, c are converted once to level 1, so every gate term
// lands on level 0 and the sums need no conversion.  Product-gate tables stay
// at level 0; the product of d factors lands on level 1-d, which the eq
// weight (stored at level d) and a per-degree constant for o bring back to 0.
#include <algorithm>
#include <cstring>

#include "zc_internal.cuh"

namespace zc {

// ------------------------------------------------------------------ args --

struct ScSetupArgs {
  ScState* st;
  const uint8_t* roots;  // c x 32 bytes, device
  uint32_t S0[8];
  int c, n;
  const DevConst* C;
};

struct EqTask {      // one factor table
  uint32_t offset;   // into the E array
  uint32_t first_var;  // 0-based index of its most significant variable
  uint32_t nvars;
  uint32_t level;    // 1 or d (extra R^(level-1) factor)
};

struct ScEqArgs {
  ScState* st;
  fr* E;
  EqTask task[2 * kMaxN];
  uint32_t ntask;
  uint32_t total;     // total entries
  int n;
  int skip_point;
  const DevConst* C;
};

struct ScPlonkArgs {
  const fr* src[8];
  fr* dst[8];
  uint64_t h;         // number of pairs this round
  const fr* ehi;
  const fr* elo;
  uint32_t m_lo;
  int round;          // 0-based
  ScState* st;
  fr* partials;
  const DevConst* C;
};

struct ScFoldArgs {
  const fr* src[kMaxCols];
  fr* dst[kMaxCols];
  uint64_t h;         // output size per column
  int c;
  int round;          // alpha index
  ScState* st;
};

struct ScProdArgs {
  const fr* col[kMaxCols];
  uint64_t h;
  const fr* ehi;
  const fr* elo;
  uint32_t m_lo;
  int d;
  int np;             // points this round
  int G;              // threads per pair
  int round;
  ScState* st;
  fr* partials;
  fr kcomp;           // R^(2-d) mod r, canonical number
  const DevConst* C;
};

struct ScChalArgs {
  const fr* partials;
  int nblk;
  int np;
  int d;
  int round;
  int n;
  ScState* st;
  uint8_t* proof;     // device proof buffer
  const DevConst* C;
  const fr* tabs;
};

struct ScFinalArgs {
  const fr* src[kMaxCols];
  uint32_t level[kMaxCols];
  int c, n;
  uint32_t gate, d;
  ScState* st;
  uint8_t* proof;
  const uint32_t* in_err;
};

// ----------------------------------------------------------- helpers --

__device__ __forceinline__ void fr_to_le_bytes(const fr& x, uint8_t* out) {
#pragma unroll
  for (int i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)x.v[i];
    out[4 * i + 1] = (uint8_t)(x.v[i] >> 8);
    out[4 * i + 2] = (uint8_t)(x.v[i] >> 16);
    out[4 * i + 3] = (uint8_t)(x.v[i] >> 24);
  }
}

// 32-byte digest (big-endian words) -> integer mod r as a canonical fr
__device__ __forceinline__ fr digest_to_canon(const uint32_t h[8]) {
  fr x;
#pragma unroll
  for (int i = 0; i < 8; i++) x.v[i] = sha_bswap(h[i]);  // bytes little-endian
  // at most two subtractions: 2^256 < 3r
  for (int k = 0; k < 2; k++) {
    if (!fr_is_canonical(x)) {
      int64_t br = 0;
      for (int i = 0; i < 8; i++) {
        int64_t dd = (int64_t)x.v[i] - p_limb(i) + br;
        x.v[i] = (uint32_t)dd;
        br = dd >> 32;
      }
    }
  }
  return x;
}

// S <- SHA-256(S | msg)
__device__ void tr_absorb(uint32_t S[8], const uint8_t* msg, uint32_t len) {
  Sha256 s;
  s.init();
  for (int i = 0; i < 8; i++) {
    uint32_t w = S[i];
    s.put_byte((uint8_t)(w >> 24));
    s.put_byte((uint8_t)(w >> 16));
    s.put_byte((uint8_t)(w >> 8));
    s.put_byte((uint8_t)w);
  }
  s.update(msg, len);
  uint8_t out[32];
  s.final(out);
  for (int i = 0; i < 8; i++)
    S[i] = ((uint32_t)out[4 * i] << 24) | ((uint32_t)out[4 * i + 1] << 16) |
           ((uint32_t)out[4 * i + 2] << 8) | out[4 * i + 3];
}

// S <- SHA-256(S | 0x43), challenge = int_le(S) mod r (canonical)
__device__ fr tr_squeeze(uint32_t S[8]) {
  uint32_t w[16];
  for (int i = 0; i < 8; i++) w[i] = S[i];
  w[8] = 0x43800000u;  // 0x43, then the padding bit
  for (int i = 9; i < 15; i++) w[i] = 0;
  w[15] = 33 * 8;
  uint32_t h[8];
  sha256_init(h);
  sha256_compress(h, w);
  for (int i = 0; i < 8; i++) S[i] = h[i];
  return digest_to_canon(h);
}

__device__ __forceinline__ bool fr_is_one_canon(const fr& x) {
  return x.v[0] == 1 && (x.v[1] | x.v[2] | x.v[3] | x.v[4] | x.v[5] | x.v[6] | x.v[7]) == 0;
}

// small integer t times x by double-and-add (t < 128), additions only
__device__ __forceinline__ fr fr_mul_small(const fr& x, uint32_t t) {
  fr acc = fr_zero();
  bool started = false;
  for (int b = 6; b >= 0; b--) {
    if (started) acc = fr_add(acc, acc);
    if ((t >> b) & 1) {
      acc = started ? fr_add(acc, x) : x;
      started = true;
    }
  }
  return acc;
}

// Block-wide sum of NV field values per thread; result written by thread 0
// to out[0..NV).  blockDim.x must be a multiple of 32 (<= 1024).
template <int NV>
__device__ void block_sum_store(fr (&v)[NV], fr* out) {
  __shared__ fr red[32][NV];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int p = 0; p < NV; p++) {
    fr s = warp_sum(v[p]);
    if (lane == 0) red[warp][p] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int p = 0; p < NV; p++) {
      fr s = lane < nw ? red[lane][p] : fr_zero();
      s = warp_sum(s);
      if (lane == 0) st_fr(out + p, s);
    }
  }
}

// ---------------------------------------------------------------- kernels --

// Transcript: absorb the column roots, squeeze r_1..r_n.
__global__ void k_sc_setup(ScSetupArgs A) {
  if (threadIdx.x != 0) return;
  uint32_t S[8];
  for (int i = 0; i < 8; i++) S[i] = A.S0[i];
  for (int j = 0; j < A.c; j++) tr_absorb(S, A.roots + 32 * j, 32);
  for (int i = 0; i < A.n; i++) {
    fr r = tr_squeeze(S);
    A.st->r[i] = fr_mul(r, A.C->r2);
  }
  for (int i = 0; i < 8; i++) A.st->S[i] = S[i];
  A.st->claim = fr_zero();
  A.st->ci = A.C->one;
  A.st->err = 0;
}

// Factor tables of eq_{>i} for every round, and 1/r_i, 1/(1-r_i).
// Blocks [0, ninv_blocks) compute inverses, the rest fill table entries.
__global__ void k_sc_eq(ScEqArgs A) {
  const DevConst* C = A.C;
  if (blockIdx.x == 0) {
    // inverses: thread t < 2n handles r_{t/2} (even t) or 1 - r_{t/2} (odd t)
    int t = threadIdx.x;
    if (t < 2 * A.n) {
      int i = t >> 1;
      fr r = A.st->r[i];
      fr x = (t & 1) ? fr_sub(C->one, r) : r;   // level 1
      fr xc = from_mont(x);                      // canonical
      fr inv = fr_inv_binary(xc);                // canonical (0 -> 0)
      fr invm = fr_mul(inv, C->r2);              // level 1
      if (t & 1) A.st->r1inv[i] = invm;
      else A.st->rinv[i] = invm;
      if (!(t & 1)) {
        bool rzero = fr_is_zero(r);
        bool rone = fr_equal(r, C->one);
        A.st->p0[i] = A.skip_point == 0 ? (rzero ? 1u : 0u) : (rone ? 0u : 1u);
      }
    }
    return;
  }
  uint32_t e = (blockIdx.x - 1) * blockDim.x + threadIdx.x;
  if (e >= A.total) return;
  uint32_t ti = 0;
  while (ti + 1 < A.ntask && A.task[ti + 1].offset <= e) ti++;
  const EqTask& T = A.task[ti];
  uint32_t x = e - T.offset;
  fr acc = C->one;
  for (uint32_t l = 0; l < T.nvars; l++) {
    uint32_t bit = (x >> (T.nvars - 1 - l)) & 1;
    fr r = A.st->r[T.first_var + l];
    acc = fr_mul(acc, bit ? r : fr_sub(C->one, r));
  }
  if (T.level > 1) acc = fr_mul(acc, C->rpow[T.level]);  // level 1 -> level L
  st_fr(A.E + e, acc);
}

// One round of the Plonk-gate SumCheck.  FIRST: round 1, reads the input
// columns, converts a, b, c to level 1 (written to dst), evaluates t = 0, 1,
// 2 and infinity.  Otherwise: folds by alpha_{round-1} (reading 4 entries,
// writing 2 per column and pair) and evaluates t = p0, 2 and infinity.
// Columns stream in the order b, qM, qL, a, qR, qO, c, qC so that only the
// running gate value per point stays live:
//   f = a (qL + qM b) + qR b + qO c + qC.
template <bool FIRST>
__global__ void __launch_bounds__(256, 1) k_sc_plonk_round(ScPlonkArgs A) {
  constexpr int NF = FIRST ? 3 : 2;   // finite points
  constexpr int NP = NF + 1;
  const DevConst* C = A.C;
  const uint64_t h = A.h;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
  fr acc[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) acc[p] = fr_zero();
  const fr alpha = FIRST ? fr_zero() : A.st->alpha[A.round - 1];
  const uint32_t p0 = FIRST ? 0u : A.st->p0[A.round];
  uint32_t bad = 0;

  for (uint64_t k = tid; k < h; k += T) {
    // load (and fold) column j; returns its values at the finite points and its slope
    auto column = [&](int j, fr (&v)[NF], fr& dl) {
      fr lo, hi;
      if (FIRST) {
        lo = ld_fr(A.src[j] + k);
        hi = ld_fr(A.src[j] + k + h);
        bad |= (!fr_is_canonical(lo)) | (!fr_is_canonical(hi));
        if (j >= 5) {
          lo = to_mont(lo, C);
          hi = to_mont(hi, C);
          st_fr(A.dst[j] + k, lo);
          st_fr(A.dst[j] + k + h, hi);
        }
      } else {
        fr x0 = ld_fr(A.src[j] + k), x1 = ld_fr(A.src[j] + k + 2 * h);
        fr y0 = ld_fr(A.src[j] + k + h), y1 = ld_fr(A.src[j] + k + 3 * h);
        lo = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
        hi = fr_add(y0, fr_mul(alpha, fr_sub(y1, y0)));
        st_fr(A.dst[j] + k, lo);
        st_fr(A.dst[j] + k + h, hi);
      }
      dl = fr_sub(hi, lo);
      if (FIRST) {
        v[0] = lo;
        v[1] = hi;
        v[NF - 1] = fr_add(hi, dl);
      } else {
        v[0] = p0 ? hi : lo;
        v[NF - 1] = fr_add(hi, dl);
      }
    };
    fr bv[NF], s[NF], t[NF], u[NF], db, dt, dinf;
    column(6, bv, db);                              // b
    column(2, t, dt);                               // qM
    dinf = fr_mul(dt, db);
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_mul(t[p], bv[p]);
    column(0, t, dt);                               // qL
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], t[p]);
    column(5, t, dt);                               // a
    dinf = fr_mul(dinf, dt);
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_mul(t[p], s[p]);
    column(1, t, dt);                               // qR
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], fr_mul(t[p], bv[p]));
    column(3, t, dt);                               // qO
    column(7, u, db);                               // c
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], fr_mul(t[p], u[p]));
    column(4, t, dt);                               // qC
#pragma unroll
    for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], t[p]);
    const fr w = ld_fr(A.ehi + (k >> A.m_lo));
#pragma unroll
    for (int p = 0; p < NF; p++) acc[p] = fr_add(acc[p], fr_mul(s[p], w));
    acc[NF] = fr_add(acc[NF], fr_mul(dinf, w));
  }
  if (FIRST && bad) atomicOr(&A.st->err, 1u);
  // each thread handled pairs with one fixed low part k_lo
  const fr wl = ld_fr(A.elo + (tid & ((1ull << A.m_lo) - 1)));
#pragma unroll
  for (int p = 0; p < NP; p++) acc[p] = fr_mul(acc[p], wl);
  block_sum_store<NP>(acc, A.partials + (size_t)blockIdx.x * NP);
}

// MLE update by alpha_{round-1}: dst[j][k] = src[j][k] + alpha (src[j][k+h] - src[j][k])
__global__ void __launch_bounds__(256) k_sc_fold(ScFoldArgs A) {
  fr alpha = A.st->alpha[A.round - 1];
  const uint64_t total = A.h * (uint64_t)A.c;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    int j = (int)(e / A.h);
    uint64_t k = e - (uint64_t)j * A.h;
    fr x0 = ld_fr(A.src[j] + k), x1 = ld_fr(A.src[j] + k + A.h);
    st_fr(A.dst[j] + k, fr_add(x0, fr_mul(alpha, fr_sub(x1, x0))));
  }
}

// point index -> evaluation point (kInf for infinity)
constexpr uint32_t kInf = 0xffffffffu;
__device__ __forceinline__ uint32_t prod_point(int p, int np, int d, bool first, uint32_t p0) {
  if (p == np - 1) return kInf;
  if (first) return (uint32_t)p;        // 0, 1, ..., d-1
  return p == 0 ? p0 : (uint32_t)p + 1;  // p0, 2, ..., d-1
}

// Product-gate evaluation: f = q w1 .. w_{d-1} - o.  Each pair is shared by G
// threads, each evaluating up to PP consecutive points; tables at level 0.
template <int PP>
__global__ void __launch_bounds__(256) k_sc_prod_eval(ScProdArgs A) {
  const DevConst* C = A.C;
  const int G = A.G, d = A.d, np = A.np;
  const bool first = A.round == 0;
  const uint32_t p0 = first ? 0u : A.st->p0[A.round];
  const int g = threadIdx.x % G;
  const uint64_t slot = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const uint64_t nslots = (uint64_t)gridDim.x * blockDim.x / G;
  const int pbeg = g * PP;
  const int pcnt = max(0, min(PP, np - pbeg));
  uint32_t bad = 0;
  fr acc[PP];
#pragma unroll
  for (int p = 0; p < PP; p++) acc[p] = fr_zero();
  uint32_t tpt[PP];
#pragma unroll
  for (int p = 0; p < PP; p++) tpt[p] = p < pcnt ? prod_point(pbeg + p, np, d, first, p0) : 0u;

  for (uint64_t k = slot; k < A.h && pcnt > 0; k += nslots) {
    fr prod[PP];
    for (int j = 0; j <= d; j++) {
      fr lo = ld_fr(A.col[j] + k), hi = ld_fr(A.col[j] + k + A.h);
      if (first) bad |= (!fr_is_canonical(lo)) | (!fr_is_canonical(hi));
      fr dl = fr_sub(hi, lo);
      // value at the first finite point, then step by dl
      fr e = lo;
      uint32_t tcur = 0;
#pragma unroll
      for (int p = 0; p < PP; p++) {
        if (p >= pcnt) break;
        fr x;
        if (tpt[p] == kInf) {
          x = dl;
        } else {
          if (p == 0) {
            e = fr_add(lo, fr_mul_small(dl, tpt[p]));
          } else {
            for (uint32_t s = tcur; s < tpt[p]; s++) e = fr_add(e, dl);
          }
          tcur = tpt[p];
          x = e;
        }
        if (j == d) {
          // o enters at level 0; bring it to level 1-d with kcomp.  The
          // leading coefficient has no o term.
          if (tpt[p] != kInf) prod[p] = fr_sub(prod[p], fr_mul(x, A.kcomp));
        } else {
          prod[p] = j == 0 ? x : fr_mul(prod[p], x);
        }
      }
    }
    fr w = fr_mul(ld_fr(A.ehi + (k >> A.m_lo)), ld_fr(A.elo + (k & ((1ull << A.m_lo) - 1))));
#pragma unroll
    for (int p = 0; p < PP; p++)
      if (p < pcnt) acc[p] = fr_add(acc[p], fr_mul(prod[p], w));
  }
  if (bad) atomicOr(&A.st->err, 1u);
  // reduce over the threads of the CTA that share g
  __shared__ fr red[256 / 32][32][PP];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < PP; p++) {
    fr s = acc[p];
    for (int off = 16; off >= G; off >>= 1) s = fr_add(s, shfl_down_fr(s, off));
    if (lane < G) red[warp][lane][p] = s;
  }
  __syncthreads();
  int nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < G * PP; q += blockDim.x) {
    int gg = q / PP, p = q % PP;
    int pg = gg * PP + p;
    if (pg >= np) continue;
    fr s = fr_zero();
    for (int w2 = 0; w2 < nw; w2++) s = fr_add(s, red[w2][gg][p]);
    st_fr(A.partials + (size_t)blockIdx.x * np + pg, s);
  }
}

// Reduce the per-CTA partial sums, finish G_i, hash, derive alpha_i and the
// next claim.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_sc_challenge(ScChalArgs A) {
  const DevConst* C = A.C;
  const int d = A.d, np = A.np, i = A.round;
  const bool first = i == 0;
  __shared__ fr Hc[kMaxPts];
  __shared__ fr H[kMaxPts + 1];   // H(0..d+1)
  __shared__ fr Hinf;
  __shared__ fr tmp[2][kMaxPts];
  __shared__ uint8_t msg[32 * kMaxPts];
  __shared__ fr s_alpha;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = warp; p < np; p += nw) {
    fr s = fr_zero();
    for (int b = lane; b < A.nblk; b += 32) s = fr_add(s, ld_fr_cg(A.partials + (size_t)b * np + p));
    s = warp_sum(s);
    if (lane == 0) Hc[p] = s;
  }
  __syncthreads();
  const fr r = A.st->r[i];
  if (threadIdx.x == 0) {
    Hinf = Hc[np - 1];
    if (first) {
      for (int t = 0; t < d; t++) H[t] = Hc[t];
    } else {
      uint32_t p0 = A.st->p0[i];
      for (int t = 2; t < d; t++) H[t] = Hc[t - 1];
      fr claim = A.st->claim;   // level 0
      if (p0 == 0) {
        H[0] = Hc[0];
        // H(1) = (claim - (1-r) H(0)) / r
        H[1] = fr_mul(fr_sub(claim, fr_mul(fr_sub(C->one, r), H[0])), A.st->rinv[i]);
      } else {
        H[1] = Hc[0];
        // H(0) = (claim - r H(1)) / (1-r)
        H[0] = fr_mul(fr_sub(claim, fr_mul(r, H[1])), A.st->r1inv[i]);
      }
    }
  }
  __syncthreads();
  // extrapolate H(d), H(d+1) from H(0..d-1) and the leading coefficient
  const fr* ext = A.tabs + C->ext_base[d];
  if (threadIdx.x < d) {
    int s = threadIdx.x;
    tmp[0][s] = fr_mul(H[s], ext[2 + s]);
    tmp[1][s] = fr_mul(H[s], ext[2 + d + s]);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    int t = threadIdx.x;
    fr s = fr_mul(Hinf, ext[t]);
    for (int q = 0; q < d; q++) s = fr_add(s, tmp[t][q]);
    H[d + t] = s;
  }
  __syncthreads();
  // G(t) = c_i l_i(t) H(t), level 0 = canonical
  const fr two_r_m1 = fr_sub(fr_add(r, r), C->one);
  const fr one_m_r = fr_sub(C->one, r);
  if (threadIdx.x < d + 2) {
    int t = threadIdx.x;
    fr l = fr_add(one_m_r, fr_mul(C->small[t], two_r_m1));
    fr g = fr_mul(H[t], fr_mul(A.st->ci, l));
    uint8_t* out = msg + 32 * t;
    fr_to_le_bytes(g, out);
    uint8_t* pout = A.proof + 16 + 32 * ((size_t)i * (d + 2) + t);
    for (int b = 0; b < 32; b++) pout[b] = out[b];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t S[8];
    for (int q = 0; q < 8; q++) S[q] = A.st->S[q];
    tr_absorb(S, msg, 32 * (d + 2));
    fr a = fr_mul(tr_squeeze(S), C->r2);
    for (int q = 0; q < 8; q++) A.st->S[q] = S[q];
    A.st->alpha[i] = a;
    s_alpha = a;
  }
  __syncthreads();
  // next claim H_i(alpha) by Lagrange over the nodes 0..d
  const fr a = s_alpha;
  const fr* dinv = A.tabs + C->lag_base[d];
  if (threadIdx.x <= d) {
    int s = threadIdx.x;
    fr num = C->one;
    for (int q = 0; q <= d; q++)
      if (q != s) num = fr_mul(num, fr_sub(a, C->small[q]));
    tmp[0][s] = fr_mul(fr_mul(H[s], num), dinv[s]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    fr s = fr_zero();
    for (int q = 0; q <= d; q++) s = fr_add(s, tmp[0][q]);
    A.st->claim = s;
    fr l = fr_add(one_m_r, fr_mul(a, two_r_m1));
    A.st->ci = fr_mul(A.st->ci, l);
  }
}

// Final MLE values v_j = T_j[0] + alpha_n (T_j[1] - T_j[0]) and the header.
__global__ void k_sc_final(ScFinalArgs A) {
  int j = threadIdx.x;
  uint8_t* pv = A.proof + 16 + 32 * ((size_t)A.n * (A.d + 2));
  if (j < A.c) {
    fr alpha = A.st->alpha[A.n - 1];
    fr x0 = ld_fr_cg(A.src[j]), x1 = ld_fr_cg(A.src[j] + 1);
    fr v = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
    if (A.level[j] == 1) v = from_mont(v);
    fr_to_le_bytes(v, pv + 32 * j);
  }
  if (j == 0) {
    uint32_t bad = A.st->err;
    const char* mg = bad ? "ZCE!" : "ZCS1";
    for (int b = 0; b < 4; b++) A.proof[b] = (uint8_t)mg[b];
    uint32_t hv[3] = {A.gate, (uint32_t)A.n, A.d};
    for (int q = 0; q < 3; q++)
      for (int b = 0; b < 4; b++) A.proof[4 + 4 * q + b] = (uint8_t)(hv[q] >> (8 * b));
  }
}

// ------------------------------------------------------------------ host --

static void eq_round_split(int n, int round, uint32_t* m_lo, uint32_t* m_hi) {
  uint32_t m = (uint32_t)(n - 1 - round);  // variables after x_{round+1}
  uint32_t lo = m / 2;
  if (lo > 11) lo = 11;
  *m_lo = lo;
  *m_hi = m - lo;
}

zc_status sumcheck_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                         const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                         bool proof_on_dev) {
  const uint32_t gate = p->gate, n = p->n, d = p->d;
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n;
  const bool plonk = gate == ZC_GATE_PLONK;
  const int SMs = ctx->sm_count;
  const size_t psize = 16 + 32 * ((size_t)n * (d + 2) + c);

  // ---- scratch layout
  const int grid_max_plonk = 2 * SMs / 8 * 8 > 0 ? 2 * SMs / 8 * 8 : 8;
  const int PP = 4;
  int G = 1;
  while (G * PP < (int)d + 1) G *= 2;
  const int grid_max_prod = 2 * SMs;
  const int npmax = (int)d + 1;
  uint32_t eq_total = 0;
  EqTask tasks[2 * kMaxN];
  uint32_t eq_off_hi[kMaxN], eq_off_lo[kMaxN], mlo_r[kMaxN];
  for (uint32_t i = 0; i < n; i++) {
    uint32_t mlo, mhi;
    eq_round_split((int)n, (int)i, &mlo, &mhi);
    mlo_r[i] = mlo;
    tasks[2 * i] = EqTask{eq_total, i + 1, mhi, plonk ? 1u : d};
    eq_off_hi[i] = eq_total;
    eq_total += 1u << mhi;
    tasks[2 * i + 1] = EqTask{eq_total, n - mlo, mlo, 1u};
    eq_off_lo[i] = eq_total;
    eq_total += 1u << mlo;
  }
  size_t need = 0;
  need += align_up(sizeof(fr) * N, 256) * c;                        // tables
  need += align_up(sizeof(fr) * (size_t)std::max(grid_max_plonk, grid_max_prod) * (npmax + 1), 256);
  need += align_up(sizeof(fr) * eq_total, 256);
  need += align_up(sizeof(ScState), 256);
  need += align_up(psize, 256);
  need += align_up(32 * (size_t)c, 256);
  if (!roots) need += root_scratch_bytes(c, N);
  need += 4096;
  zc_status s = ensure_arena(ctx, need);
  if (s != ZC_OK) return s;
  Arena& ar = ctx->arena;
  ar.reset();
  fr* tab[kMaxCols];
  for (int j = 0; j < c; j++) tab[j] = ar.take<fr>(N);
  fr* partials = ar.take<fr>((size_t)std::max(grid_max_plonk, grid_max_prod) * (npmax + 1));
  fr* E = ar.take<fr>(eq_total);
  ScState* dst = ar.take<ScState>(1);
  uint8_t* dproof = ar.take<uint8_t>(psize);
  uint8_t* droots = ar.take<uint8_t>(32 * (size_t)c);
  if (!dproof || !droots) {
    ctx->err = "scratch arena too small";
    return ZC_ERR_OOM;
  }

  const fr* src[kMaxCols];
  if (on_dev) {
    for (int j = 0; j < c; j++) src[j] = reinterpret_cast<const fr*>(cols[j]);
  } else {
    for (int j = 0; j < c; j++) {
      ZC_CUDA_TRY(ctx, cudaMemcpyAsync(tab[j], cols[j], N * sizeof(fr), cudaMemcpyHostToDevice, st));
      src[j] = tab[j];
    }
  }
  ctx->launches = 0;
  ctx->nev = 6;
  ctx->dom_a = 2;
  ctx->dom_b = 3;
  // round-1 evaluation: per pair (d+1)(g+1)+1 mulmods, reads c*N*32 bytes
  const double g_mul = plonk ? 5.0 : (double)(d - 1);
  ctx->dom_mulmods = (double)(N / 2) * ((d + 1) * (g_mul + 1) + 1);
  ctx->dom_bytes = 32.0 * (double)c * (double)N;
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], st));
  if (roots) {
    std::memcpy(ctx->pinned, roots, 32 * (size_t)c);
    ZC_CUDA_TRY(ctx, cudaMemcpyAsync(droots, ctx->pinned, 32 * (size_t)c, cudaMemcpyHostToDevice, st));
  } else {
    s = launch_roots(ctx, src, c, N, droots, st);
    if (s != ZC_OK) return s;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], st));

  ScSetupArgs sa{};
  sa.st = dst;
  sa.roots = droots;
  transcript_init_words(sa.S0, ZC_FORM_SUMCHECK, gate, n, d, 0);
  sa.c = c;
  sa.n = (int)n;
  sa.C = ctx->dconst;
  k_sc_setup<<<1, 32, 0, st>>>(sa);
  ctx->launches++;
  ScEqArgs ea{};
  ea.st = dst;
  ea.E = E;
  for (uint32_t t = 0; t < 2 * n; t++) ea.task[t] = tasks[t];
  ea.ntask = 2 * n;
  ea.total = eq_total;
  ea.n = (int)n;
  ea.skip_point = ctx->skip_point;
  ea.C = ctx->dconst;
  k_sc_eq<<<1 + (eq_total + 255) / 256, 256, 0, st>>>(ea);
  ctx->launches++;
  ZC_CUDA_TRY(ctx, cudaGetLastError());
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[2], st));

  const fr* cur[kMaxCols];
  for (int j = 0; j < c; j++) cur[j] = src[j];
  for (uint32_t i = 0; i < n; i++) {
    const uint64_t h = N >> (i + 1);  // pairs this round
    int nblk, np;
    if (plonk) {
      ScPlonkArgs pa{};
      for (int j = 0; j < 8; j++) {
        pa.src[j] = cur[j];
        pa.dst[j] = tab[j];
      }
      pa.h = h;
      pa.ehi = E + eq_off_hi[i];
      pa.elo = E + eq_off_lo[i];
      pa.m_lo = mlo_r[i];
      pa.round = (int)i;
      pa.st = dst;
      pa.partials = partials;
      pa.C = ctx->dconst;
      uint64_t want = (h + 255) / 256;
      nblk = (int)std::min<uint64_t>(want, (uint64_t)grid_max_plonk);
      if (i == 0) {
        np = 4;
        k_sc_plonk_round<true><<<nblk, 256, 0, st>>>(pa);
  ctx->launches++;
        for (int j = 5; j < 8; j++) cur[j] = tab[j];  // wires now at level 1 in scratch
      } else {
        np = 3;
        k_sc_plonk_round<false><<<nblk, 256, 0, st>>>(pa);
  ctx->launches++;
        for (int j = 0; j < 8; j++) cur[j] = tab[j];
      }
    } else {
      if (i > 0) {
        ScFoldArgs fa{};
        for (int j = 0; j < c; j++) {
          fa.src[j] = cur[j];
          fa.dst[j] = tab[j];
        }
        fa.h = 2 * h;
        fa.c = c;
        fa.round = (int)i;
        fa.st = dst;
        uint64_t tot = 2 * h * (uint64_t)c;
        int fb = (int)std::min<uint64_t>((tot + 255) / 256, (uint64_t)SMs * 8);
        k_sc_fold<<<fb, 256, 0, st>>>(fa);
  ctx->launches++;
        for (int j = 0; j < c; j++) cur[j] = tab[j];
      }
      np = i == 0 ? (int)d + 1 : (int)d;
      ScProdArgs pa{};
      for (int j = 0; j < c; j++) pa.col[j] = cur[j];
      pa.h = h;
      pa.ehi = E + eq_off_hi[i];
      pa.elo = E + eq_off_lo[i];
      pa.m_lo = mlo_r[i];
      pa.d = (int)d;
      pa.np = np;
      pa.G = G;
      pa.round = (int)i;
      pa.st = dst;
      pa.partials = partials;
      pa.kcomp = ctx->hconst.rnegpow[d - 2];
      pa.C = ctx->dconst;
      uint64_t slots_per_blk = 256 / G;
      uint64_t want = (h + slots_per_blk - 1) / slots_per_blk;
      nblk = (int)std::min<uint64_t>(want, (uint64_t)grid_max_prod);
      k_sc_prod_eval<4><<<nblk, 256, 0, st>>>(pa);
  ctx->launches++;
    }
    ScChalArgs ca{};
    ca.partials = partials;
    ca.nblk = nblk;
    ca.np = np;
    ca.d = (int)d;
    ca.round = (int)i;
    ca.n = (int)n;
    ca.st = dst;
    ca.proof = dproof;
    ca.C = ctx->dconst;
    ca.tabs = ctx->dtabs;
    if (i == 0) ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[3], st));
    k_sc_challenge<<<1, 256, 0, st>>>(ca);
    ctx->launches++;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[4], st));
  ScFinalArgs fa{};
  for (int j = 0; j < c; j++) {
    fa.src[j] = cur[j];
    fa.level[j] = (plonk && j >= 5) ? 1u : 0u;
  }
  fa.c = c;
  fa.n = (int)n;
  fa.gate = gate;
  fa.d = d;
  fa.st = dst;
  fa.proof = dproof;
  k_sc_final<<<1, 128, 0, st>>>(fa);
  ctx->launches++;
  ZC_CUDA_TRY(ctx, cudaGetLastError());
  ZC_CUDA_TRY(ctx, cudaMemcpyAsync(proof, dproof, psize,
                                   proof_on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   st));
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[5], st));
  if (!proof_on_dev || !on_dev) {
    ZC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (std::memcmp(proof, "ZCE!", 4) == 0) {
      ctx->err = "column value >= r";
      return ZC_ERR_ARG;
    }
  }
  return ZC_OK;
}

}  // namespace zc

// ------------------------------------------------- static-scratch variant --
//
// zc_prove_sumcheck_static: the SumCheck prover for callers that cannot
// allocate device memory at proving time -- code running under an allocator
// that forbids new device allocations (a fixed memory pool reserved up
// front), a stream-ordered pipeline that must not insert the implicit
// synchronisation a cudaMalloc/cudaFree brings, or a host that links the
// library into a process whose device memory is already fully reserved.
// Everything the prover needs beyond the caller's inputs and output lives in
// file-scope device arrays of fixed size: every GPU that loads the library
// holds them until the process exits.  Host code never dereferences these
// symbols: it asks the runtime for their device addresses once per device.

namespace zc {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB
constexpr int kStaticTabCap = 8192;                   // per-degree table entries
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) DevConst g_static_const;
static __device__ __align__(256) fr g_static_tabs[kStaticTabCap];

struct StaticDev {
  bool ready = false;
  void* scratch = nullptr;
  DevConst* dconst = nullptr;
  fr* dtabs = nullptr;
  DevConst hconst;
};
static StaticDev g_static_dev[kStaticMaxDevices];
static std::mutex g_static_mu;

// Set-up for the current device: look up the device addresses of the static
// arrays and copy the field constants into them.  Runs on the first call per
// device (synchronous copies), so that first call must not be inside a
// stream capture.
static zc_status static_setup(int dev, StaticDev** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticDev& S = g_static_dev[dev];
  if (!S.ready) {
    std::vector<fr> tabs;
    static_constants(&S.hconst, &tabs);
    if (tabs.size() > (size_t)kStaticTabCap) return ZC_ERR_UNSUPPORTED;
    if (cudaGetSymbolAddress(&S.scratch, g_static_scratch) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&S.dconst, g_static_const) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&S.dtabs, g_static_tabs) != cudaSuccess) {
      cudaGetLastError();
      return ZC_ERR_CUDA;
    }
    if (cudaMemcpy(S.dconst, &S.hconst, sizeof(DevConst), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(S.dtabs, tabs.data(), sizeof(fr) * tabs.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      return ZC_ERR_CUDA;
    }
    S.ready = true;
  }
  *out = &S;
  return ZC_OK;
}

static zc_status static_prove(const zc_params* p, const void* const* cols,
                              const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                              StaticDev& S) {
  const uint32_t gate = p->gate, n = p->n, d = p->d;
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n;
  const bool plonk = gate == ZC_GATE_PLONK;
  int SMs = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&SMs, cudaDevAttrMultiProcessorCount, dev);
  const int grid_max_plonk = 2 * SMs / 8 * 8 > 0 ? 2 * SMs / 8 * 8 : 8;
  const int PP = 4;
  int G = 1;
  while (G * PP < (int)d + 1) G *= 2;
  const int grid_max_prod = 2 * SMs;
  const int npmax = (int)d + 1;
  uint32_t eq_total = 0;
  EqTask tasks[2 * kMaxN];
  uint32_t eq_off_hi[kMaxN], eq_off_lo[kMaxN], mlo_r[kMaxN];
  for (uint32_t i = 0; i < n; i++) {
    uint32_t mlo, mhi;
    eq_round_split((int)n, (int)i, &mlo, &mhi);
    mlo_r[i] = mlo;
    tasks[2 * i] = EqTask{eq_total, i + 1, mhi, plonk ? 1u : d};
    eq_off_hi[i] = eq_total;
    eq_total += 1u << mhi;
    tasks[2 * i + 1] = EqTask{eq_total, n - mlo, mlo, 1u};
    eq_off_lo[i] = eq_total;
    eq_total += 1u << mlo;
  }
  // carve the static array; reject instances that do not fit
  Arena ar;
  ar.base = static_cast<char*>(S.scratch);
  ar.cap = kStaticScratchBytes;
  fr* tab[kMaxCols];
  for (int j = 0; j < c; j++) tab[j] = ar.take<fr>(N);
  fr* partials = ar.take<fr>((size_t)std::max(grid_max_plonk, grid_max_prod) * (npmax + 1));
  fr* E = ar.take<fr>(eq_total);
  ScState* dst = ar.take<ScState>(1);
  uint8_t* droots = ar.take<uint8_t>(32 * (size_t)c);
  if (!tab[c - 1] || !partials || !E || !dst || !droots ||
      (!roots && ar.used + root_scratch_bytes(c, N) > ar.cap))
    return ZC_ERR_UNSUPPORTED;  // instance larger than the static scratch

  const fr* src[kMaxCols];
  for (int j = 0; j < c; j++) src[j] = reinterpret_cast<const fr*>(cols[j]);
  if (roots) {
    if (cudaMemcpyAsync(droots, roots, 32 * (size_t)c, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return ZC_ERR_CUDA;
  } else {
    // the root kernels take their node scratch from the rest of the static array
    zc_ctx tmp;
    tmp.arena = ar;
    zc_status rs = launch_roots(&tmp, src, c, N, droots, st);
    tmp.arena.base = nullptr;
    if (rs != ZC_OK) return rs;
  }
  ScSetupArgs sa{};
  sa.st = dst;
  sa.roots = droots;
  transcript_init_words(sa.S0, ZC_FORM_SUMCHECK, gate, n, d, 0);
  sa.c = c;
  sa.n = (int)n;
  sa.C = S.dconst;
  k_sc_setup<<<1, 32, 0, st>>>(sa);  // also clears the error flag and the claim
  ScEqArgs ea{};
  ea.st = dst;
  ea.E = E;
  for (uint32_t t = 0; t < 2 * n; t++) ea.task[t] = tasks[t];
  ea.ntask = 2 * n;
  ea.total = eq_total;
  ea.n = (int)n;
  ea.skip_point = 0;
  ea.C = S.dconst;
  k_sc_eq<<<1 + (eq_total + 255) / 256, 256, 0, st>>>(ea);
  const fr* cur[kMaxCols];
  for (int j = 0; j < c; j++) cur[j] = src[j];
  for (uint32_t i = 0; i < n; i++) {
    const uint64_t h = N >> (i + 1);
    int nblk, np;
    if (plonk) {
      ScPlonkArgs pa{};
      for (int j = 0; j < 8; j++) {
        pa.src[j] = cur[j];
        pa.dst[j] = tab[j];
      }
      pa.h = h;
      pa.ehi = E + eq_off_hi[i];
      pa.elo = E + eq_off_lo[i];
      pa.m_lo = mlo_r[i];
      pa.round = (int)i;
      pa.st = dst;
      pa.partials = partials;
      pa.C = S.dconst;
      nblk = (int)std::min<uint64_t>((h + 255) / 256, (uint64_t)grid_max_plonk);
      if (i == 0) {
        np = 4;
        k_sc_plonk_round<true><<<nblk, 256, 0, st>>>(pa);
        for (int j = 5; j < 8; j++) cur[j] = tab[j];
      } else {
        np = 3;
        k_sc_plonk_round<false><<<nblk, 256, 0, st>>>(pa);
        for (int j = 0; j < 8; j++) cur[j] = tab[j];
      }
    } else {
      if (i > 0) {
        ScFoldArgs fa{};
        for (int j = 0; j < c; j++) {
          fa.src[j] = cur[j];
          fa.dst[j] = tab[j];
        }
        fa.h = 2 * h;
        fa.c = c;
        fa.round = (int)i;
        fa.st = dst;
        uint64_t tot = 2 * h * (uint64_t)c;
        int fb = (int)std::min<uint64_t>((tot + 255) / 256, (uint64_t)SMs * 8);
        k_sc_fold<<<fb, 256, 0, st>>>(fa);
        for (int j = 0; j < c; j++) cur[j] = tab[j];
      }
      np = i == 0 ? (int)d + 1 : (int)d;
      ScProdArgs pa{};
      for (int j = 0; j < c; j++) pa.col[j] = cur[j];
      pa.h = h;
      pa.ehi = E + eq_off_hi[i];
      pa.elo = E + eq_off_lo[i];
      pa.m_lo = mlo_r[i];
      pa.d = (int)d;
      pa.np = np;
      pa.G = G;
      pa.round = (int)i;
      pa.st = dst;
      pa.partials = partials;
      pa.kcomp = S.hconst.rnegpow[d - 2];
      pa.C = S.dconst;
      uint64_t slots_per_blk = 256 / G;
      nblk = (int)std::min<uint64_t>((h + slots_per_blk - 1) / slots_per_blk, (uint64_t)grid_max_prod);
      k_sc_prod_eval<4><<<nblk, 256, 0, st>>>(pa);
    }
    ScChalArgs ca{};
    ca.partials = partials;
    ca.nblk = nblk;
    ca.np = np;
    ca.d = (int)d;
    ca.round = (int)i;
    ca.n = (int)n;
    ca.st = dst;
    ca.proof = proof;
    ca.C = S.dconst;
    ca.tabs = S.dtabs;
    k_sc_challenge<<<1, 256, 0, st>>>(ca);
  }
  ScFinalArgs fa{};
  for (int j = 0; j < c; j++) {
    fa.src[j] = cur[j];
    fa.level[j] = (plonk && j >= 5) ? 1u : 0u;
  }
  fa.c = c;
  fa.n = (int)n;
  fa.gate = gate;
  fa.d = d;
  fa.st = dst;
  fa.proof = proof;
  k_sc_final<<<1, 128, 0, st>>>(fa);
  return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

}  // namespace zc

extern "C" zc_status zc_prove_sumcheck_static(const zc_params* params, const void* const* cols,
                                              const uint8_t (*col_roots)[32], void* cuda_stream,
                                              uint8_t* proof, size_t cap, size_t* len) {
  using namespace zc;
  zc_status s = check_params(nullptr, params, ZC_FORM_SUMCHECK);
  if (s != ZC_OK) return s;
  if (!cols || !proof || !len) return ZC_ERR_ARG;
  const int c = gate_ncols(params->gate, params->d);
  for (int j = 0; j < c; j++)
    if (!cols[j]) return ZC_ERR_ARG;
  const size_t need = 16 + 32 * ((size_t)params->n * (params->d + 2) + c);
  *len = need;
  if (cap < need) return ZC_ERR_BUFFER_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
    cudaGetLastError();
    return ZC_ERR_CUDA;
  }
  StaticDev* S = nullptr;
  s = static_setup(dev, &S);
  if (s != ZC_OK) return s;
  return static_prove(params, cols, col_roots, static_cast<cudaStream_t>(cuda_stream), proof, *S);
}
