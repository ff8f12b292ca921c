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
// Scheduling: large rounds run on the whole GPU and the last CTA to finish
// (arrival counter) performs the challenge step in the same launch; once a
// round has at most kTailPairs pairs, one CTA runs all remaining rounds, the
// challenges and the final values in a single launch.
//
// Storage levels (see zc_field.cuh): Plonk selectors stay canonical (level
// 0), the wires a, b, c are converted once to level 1, so every gate term
// lands on level 0 and the sums need no conversion.  Product-gate tables stay
// at level 0; the product of d factors lands on level 1-d, which the eq
// weight (stored at level d) and a per-degree constant for o bring back to 0.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "zc_internal.cuh"
#include "zc_transcript.cuh"

namespace zc {

constexpr uint64_t kTailPairsPlonk = 32;
constexpr uint64_t kTailPairsProd = 32;
constexpr uint64_t kSmallPairsPlonk = 1ull << 14;  // rounds with at most this many pairs evaluate H(0) and H(1)
constexpr uint64_t kChunkPairsPlonk = 1ull << 14;  // Plonk rounds 2.. with at most this many: 16 threads per pair
constexpr uint64_t kQuadPairsPlonk = 1ull << 17;   // and up to this many: 4 threads per pair
constexpr uint64_t kFusePairsProd = 1ull << 16;    // product rounds 2.. with at most this many: fused update
constexpr int kPP = 3;  // product gate: points per thread
constexpr int kSmallPB = 16;  // pairs per chunk of the 16-threads-per-pair kernel (256 threads)
constexpr int kQuadPB = 32;   // pairs per chunk of the 4-threads-per-pair kernel (128 threads)
constexpr int kBigPB = 64;    // ... in the cooperative kernel's rounds above small_pairs (256 threads)
// From this n on the cooperative round kernel also takes the 4-threads-per-pair
// rounds (measured: n = 20 1.452 -> 1.430 ms, n = 22 3.601 -> 3.585 ms; at
// n = 18 their separate launches are faster, 0.795 against 0.805 ms).
constexpr uint32_t kCoopQuadMinN = 20;
constexpr int kTailPB = 32;   // pairs per chunk in the tail (512 threads)
constexpr int kTailThreads = 16 * kTailPB;

// ------------------------------------------------------------------ args --

struct ScSetupArgs {
  ScState* st;
  const uint8_t* roots;  // c x 32 bytes, device
  uint32_t S0[8];
  int c, n;
  const DevConst* C;
};

struct EqTask {        // one factor table
  uint32_t offset;     // into the E array
  uint32_t first_var;  // 0-based index of its most significant variable
  uint32_t nvars;
  uint32_t level;      // 1 or d
};

struct ScEqArgs {
  ScState* st;
  fr* E;
  EqTask task[2 * kMaxN];
  uint32_t ntask;
  uint32_t total;      // total entries
  int n;
  int skip_point;
  const DevConst* C;
};

// Everything one round (or the tail) needs.
struct ScRoundArgs {
  const fr* src[kMaxCols];
  fr* dst[kMaxCols];
  uint64_t h;          // pairs this round
  const fr* E;
  uint32_t eq_hi[kMaxN], eq_lo[kMaxN], m_lo[kMaxN];
  int round;           // 0-based; first round of the tail for k_sc_tail
  int n, c;
  uint32_t gate, d;
  int G;               // product gate: threads per pair
  uint32_t spb;        // product gate: pairs per CTA (at most 256 / threads per pair)
  uint32_t nwork;      // CTAs that evaluate pairs (round 1 may add one for the inverses)
  uint32_t full;       // evaluate H at all of 0..d-1 (no point derived from the claim)
  uint32_t next_derives;  // the next round derives a point: keep the claim
  uint32_t v2;         // eq-factored proof: rounds carry H_i(0..d), not G_i(0..d+1)
  int round_end;       // persistent round kernel: rounds [round, round_end)
  uint64_t small_pairs;  // ... rounds with more pairs derive a point, 4 threads per pair
  uint32_t spin_limit; // persistent round kernel: polls of a hand-off before giving up
  uint64_t k0, k1;     // round 1 in pair-range launches: pairs [k0, k1) (k1 = 0: all h)
  uint32_t cta0;       // ... this launch's first partial-sum slot
  uint32_t nwork_total;  // ... CTAs over all the launches of the round (0: nwork)
  ScState* st;
  fr* partials;
  uint8_t* proof;
  fr kcomp;            // product gate: R^(2-d) mod r
  const DevConst* C;
  const fr* tabs;
};

struct ScFoldArgs {
  const fr* src[kMaxCols];
  fr* dst[kMaxCols];
  uint64_t h;          // output size per column
  int c;
  int round;           // alpha index
  ScState* st;
};

// ----------------------------------------------------------- helpers --

// load through L2 only (data written earlier in the same launch)
__device__ __forceinline__ fr ld_fr_l2(const fr* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint4 a = __ldcg(q), b = __ldcg(q + 1);
  fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}

template <bool COHERENT>
__device__ __forceinline__ fr ldx(const fr* p) {
  return COHERENT ? ld_fr_l2(p) : ld_fr(p);
}

// table reads of a large round: each value is read once, so its lines are
// the first L2 evicts (ld.global.cs)
__device__ __forceinline__ fr ld_fr_cs(const fr* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint4 a = __ldcs(q), b = __ldcs(q + 1);
  fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}
template <bool COHERENT>
__device__ __forceinline__ fr ldt(const fr* p) {
  return COHERENT ? ld_fr_l2(p) : ld_fr_cs(p);
}

// small integer t times x by double-and-add, additions only.  The lanes of a
// warp may hold different t, so the loop starts at the highest bit set in
// any of them: a warp whose t are at most 6 runs two steps, not seven.
__device__ __forceinline__ fr fr_mul_small(const fr& x, uint32_t t) {
  const uint32_t any = __reduce_or_sync(__activemask(), t);
  if (any == 0) return fr_zero();
  const int top = 31 - __clz(any);
  fr acc = ((t >> top) & 1) ? x : fr_zero();
  for (int b = top - 1; b >= 0; b--) {
    acc = fr_add(acc, acc);
    if ((t >> b) & 1) acc = fr_add(acc, x);
  }
  return acc;
}

// Block-wide sum of NV values per thread, result to out[0..NV) (any memory),
// written by thread 0.  Ends with a barrier.
template <int NV>
__device__ void block_sum(fr (&v)[NV], fr* out) {
  __shared__ fr red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
  __syncthreads();
}

// ------------------------------------------------------------ challenge --

struct ChalSmem {
  fr Hc[kMaxPts];
  fr H[kMaxPts + 1];   // H(0..d+1)
  fr Hinf;
  fr tinf[2];          // Hinf times the two extrapolation weights
  fr hd[kMaxPts];      // H(t) times the Lagrange denominator's inverse
  fr tmp[2][kMaxPts];
  fr cl[kMaxPts];      // c_i l_i(t)
  fr alpha;
  uint32_t msg[8 + 8 * kMaxPts];
};
static_assert(2 * kMaxPts >= 32, "tmp holds one partial sum per warp of a 1024-thread CTA");

// Round i's value t (G_i(t), or H_i(t) for v2): into the transcript message
// (big-endian words) and the proof (little-endian bytes).
__device__ __forceinline__ void sc_put_value(ChalSmem& S, uint8_t* proof, int i, int per, int t, const fr& g) {
  uint8_t* pout = proof + 16 + 32 * ((size_t)i * per + t);
  for (int q = 0; q < 8; q++) {
    S.msg[8 + 8 * t + q] = sha_bswap(g.v[q]);
    for (int b = 0; b < 4; b++) pout[4 * q + b] = (uint8_t)(g.v[q] >> (8 * b));
  }
}

// Finish round `i` from the sums Hc (shared memory, np values): either all
// of H(0..d-1) and H(inf) (np = d + 1) or H(p0), H(2..d-1), H(inf) (np = d,
// the other of H(0), H(1) derived from the claim); extrapolate, G_i(t) =
// c_i l_i(t) H_i(t) into the proof (v2: H_i(0..d) itself, the eq-factored
// message), absorb, squeeze alpha_i, update c_i and, when the next round
// derives a point, the claim H_i(alpha_i).  All threads of the CTA (at least
// 128).  Independent steps run on different warps so the serial chain is
// four multiplications and the hash up to alpha (two or three more for c_i
// and the claim).  COLD: the hash uses the compact compression (a launch
// that runs one challenge).  release: a flag that receives i + 1 as soon as
// alpha_i is out (the persistent round kernel's hand-off).
template <bool COLD>
__device__ void sc_challenge(ChalSmem& S, int np, int d, int i, ScState* st, uint8_t* proof,
                             const DevConst* C, const fr* tabs, bool need_claim, bool v2,
                             uint32_t* release = nullptr) {
  const bool full = np == d + 1;
  const fr r = st->r[i];
  const fr two_r_m1 = fr_sub(fr_add(r, r), C->one);
  const fr one_m_r = fr_sub(C->one, r);
  const int t = threadIdx.x;
  const int hs = (d + 2 + 31) / 32 * 32;  // first thread of the warp after the c_i l_i(t) threads
  if (t < d + 2) {  // c_i l_i(t), l_i(t) = (1 - r) + t (2 r - 1): t times by additions
    if (!v2) S.cl[t] = fr_mul(st->ci, fr_add(one_m_r, fr_mul_small(two_r_m1, (uint32_t)t)));
  } else if (t == hs) {  // another warp: H(0..d-1), H(inf)
    S.Hinf = S.Hc[np - 1];
    if (full) {
      for (int q = 0; q < d; q++) S.H[q] = S.Hc[q];
    } else {
      const uint32_t p0 = st->p0[i];
      for (int q = 2; q < d; q++) S.H[q] = S.Hc[q - 1];
      const fr claim = st->claim;  // level 0
      if (p0 == 0) {
        S.H[0] = S.Hc[0];
        S.H[1] = fr_mul(fr_sub(claim, fr_mul(one_m_r, S.H[0])), st->rinv[i]);
      } else {
        S.H[1] = S.Hc[0];
        S.H[0] = fr_mul(fr_sub(claim, fr_mul(r, S.H[1])), st->r1inv[i]);
      }
    }
  }
  if (t < 8) S.msg[t] = st->S[t];
  __syncthreads();
  // extrapolate H(d), H(d+1) from H(0..d-1) and the leading coefficient:
  // every product in parallel, then two sums
  const fr* ext = tabs + C->ext_base[d];
  for (int k = t; k < 2 * d + 2; k += blockDim.x) {
    if (k < 2 * d) {
      const int which = k / d, q = k % d;
      S.tmp[which][q] = fr_mul(S.H[q], ext[2 + which * d + q]);
    } else {
      S.tinf[k - 2 * d] = fr_mul(S.Hinf, ext[k - 2 * d]);
    }
  }
  __syncthreads();
  if (t < 2) {
    fr v = S.tinf[t];
    for (int q = 0; q < d; q++) v = fr_add(v, S.tmp[t][q]);
    S.H[d + t] = v;
  }
  __syncthreads();
  // G(t) = c_i l_i(t) H(t) at t = 0..d+1, or (v2) H(t) at t = 0..d; H is
  // at level 0 = canonical.  Other threads: H(t) / prod_{q != t} (t - q)
  // for the next claim.
  const int per = v2 ? d + 1 : d + 2;
  if (t < per) sc_put_value(S, proof, i, per, t, v2 ? S.H[t] : fr_mul(S.H[t], S.cl[t]));
  const fr* dinv = tabs + C->lag_base[d];
  if (need_claim && t >= 32 && t - 32 <= d) S.hd[t - 32] = fr_mul(S.H[t - 32], dinv[t - 32]);
  __syncthreads();
  if (t == 0) {
    uint32_t Sn[8];
    sha256_words<COLD>(S.msg, 8 + 8 * per, Sn);
    const fr a = fr_mul(tr_squeeze<COLD>(Sn), C->r2);
    for (int q = 0; q < 8; q++) st->S[q] = Sn[q];
    st->alpha[i] = a;
    S.alpha = a;
    if (release) {  // the next round needs only alpha: hand it off before c_i and the claim
      __threadfence();
      atomicExch(release, (uint32_t)(i + 1));
    }
  }
  __syncthreads();
  const fr a = S.alpha;
  if (t == hs) st->ci = fr_mul(st->ci, fr_add(one_m_r, fr_mul(a, two_r_m1)));
  if (need_claim) {
    // next claim H_i(alpha) by Lagrange over the nodes 0..d
    if (t <= d) {
      const int q0 = t == 0 ? 1 : 0;
      fr num = fr_sub(a, C->small[q0]);
      for (int q = q0 + 1; q <= d; q++)
        if (q != t) num = fr_mul(num, fr_sub(a, C->small[q]));
      S.tmp[0][t] = fr_mul(S.hd[t], num);
    }
    __syncthreads();
    if (t == 0) {
      fr v = fr_zero();
      for (int q = 0; q <= d; q++) v = fr_add(v, S.tmp[0][q]);
      st->claim = v;
    }
  }
  __syncthreads();
}

// S.Hc[p] = sum of the np per-CTA partial sums of nwork CTAs.  G warps
// share each point; every lane issues its L2 loads four at a time, so the
// sum costs a few L2 round trips however many CTAs wrote partials.  All
// threads of the CTA.
__device__ void sc_sum_partials(ChalSmem& S, const fr* partials, uint32_t nwork, int np) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const int G = np < nw ? nw / np : 1, per_pass = nw / G;
  fr* W = &S.tmp[0][0];  // nw <= 2 kMaxPts partial sums, free until the challenge
  for (int base = 0; base < np; base += per_pass) {
    const int p = base + warp / G, g = warp % G;
    fr s = fr_zero();
    if (warp / G < per_pass && p < np) {
      const uint32_t stride = 32u * G;
      uint32_t b = lane + 32u * g;
      for (; b + 3 * stride < nwork; b += 4 * stride) {
        const fr x0 = ld_fr_l2(partials + (size_t)b * np + p);
        const fr x1 = ld_fr_l2(partials + (size_t)(b + stride) * np + p);
        const fr x2 = ld_fr_l2(partials + (size_t)(b + 2 * stride) * np + p);
        const fr x3 = ld_fr_l2(partials + (size_t)(b + 3 * stride) * np + p);
        s = fr_add(s, fr_add(fr_add(x0, x1), fr_add(x2, x3)));
      }
      for (; b < nwork; b += stride) s = fr_add(s, ld_fr_l2(partials + (size_t)b * np + p));
    }
    s = warp_sum(s);
    if (lane == 0) W[warp] = s;
    __syncthreads();
    if (t < per_pass && base + t < np) {
      fr v = W[t * G];
      for (int q = 1; q < G; q++) v = fr_add(v, W[t * G + q]);
      S.Hc[base + t] = v;
    }
    __syncthreads();
  }
}

// The last CTA to arrive reduces the per-CTA sums and runs the challenge.
__device__ void sc_finish_round(const ScRoundArgs& A, int np) {
  __shared__ bool am_last;
  __shared__ ChalSmem S;
  const uint32_t total = A.nwork_total ? A.nwork_total : A.nwork;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&A.st->counter[A.round], 1u);
    am_last = prev == total - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  sc_sum_partials(S, A.partials, total, np);
  sc_challenge<true>(S, np, (int)A.d, A.round, A.st, A.proof, A.C, A.tabs, A.next_derives != 0, A.v2 != 0);
}

// ------------------------------------------------------- per-pair work --

// Plonk gate, pair k of a round: loads (and, after round 1, folds by
// alpha) every column, evaluates at the finite points and infinity and adds
// eq-weighted values into acc.  Columns stream in the order b, qM, qL, a,
// qR, qO, c, qC so only the running gate value per point stays live:
//   f = a (qL + qM b) + qR b + qO c + qC.
template <bool FIRST, bool COHERENT>
__device__ __forceinline__ void plonk_pair(const fr* const* src, fr* const* dst, const DevConst* C,
                                           uint64_t k, uint64_t h, const fr& alpha, uint32_t p0,
                                           const fr& w, fr (&acc)[FIRST ? 4 : 3], uint32_t& bad) {
  constexpr int NF = FIRST ? 3 : 2;
  auto column = [&](int j, fr (&v)[NF], fr& dl) {
    fr lo, hi;
    if (FIRST) {
      lo = ldt<COHERENT>(src[j] + k);
      hi = ldt<COHERENT>(src[j] + k + h);
      bad |= (!fr_is_canonical(lo)) | (!fr_is_canonical(hi));
      if (j >= 5) {
        lo = to_mont(lo, C);
        hi = to_mont(hi, C);
        st_fr(dst[j] + k, lo);
        st_fr(dst[j] + k + h, hi);
      }
    } else {
      const fr x0 = ldt<COHERENT>(src[j] + k), x1 = ldt<COHERENT>(src[j] + k + 2 * h);
      const fr y0 = ldt<COHERENT>(src[j] + k + h), y1 = ldt<COHERENT>(src[j] + k + 3 * h);
      lo = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
      hi = fr_add(y0, fr_mul(alpha, fr_sub(y1, y0)));
      st_fr(dst[j] + k, lo);
      st_fr(dst[j] + k + h, hi);
    }
    dl = fr_sub(hi, lo);
    if (FIRST) {
      v[0] = lo;
      v[1] = hi;
    } else {
      v[0] = p0 ? hi : lo;
    }
    v[NF - 1] = fr_add(hi, dl);
  };
  fr bv[NF], s[NF], t[NF], u[NF], db, dt, dinf;
  column(6, bv, db);  // b
  column(2, t, dt);   // qM
  dinf = fr_mul(dt, db);
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_mul(t[p], bv[p]);
  column(0, t, dt);   // qL
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], t[p]);
  column(5, t, dt);   // a
  dinf = fr_mul(dinf, dt);
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_mul(t[p], s[p]);
  column(1, t, dt);   // qR
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], fr_mul(t[p], bv[p]));
  column(3, t, dt);   // qO
  column(7, u, db);   // c
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], fr_mul(t[p], u[p]));
  column(4, t, dt);   // qC
#pragma unroll
  for (int p = 0; p < NF; p++) s[p] = fr_add(s[p], t[p]);
#pragma unroll
  for (int p = 0; p < NF; p++) acc[p] = fr_add(acc[p], fr_mul(s[p], w));
  acc[NF] = fr_add(acc[NF], fr_mul(dinf, w));
}

// point index -> evaluation point (kInf for infinity)
constexpr uint32_t kInf = 0xffffffffu;
__device__ __forceinline__ uint32_t prod_point(int p, int np, bool full, uint32_t p0) {
  if (p == np - 1) return kInf;
  if (full) return (uint32_t)p;          // 0, 1, ..., d-1
  return p == 0 ? p0 : (uint32_t)p + 1;  // p0, 2, ..., d-1
}

// Product gate f = q w1 .. w_{d-1} - o, or sum gate f = g_1 .. g_d + g_{d+1}
// + .. + g_c, pair k: this thread's kPP points.  load(j, lo, hi) supplies
// column j of the pair (global memory or shared).  The degree-1 part (-o, or
// the sum of the single columns) is added up at level 0 over the pair's two
// ends first, then brought to the product's level 1-d by one kcomp
// multiplication per end (several points per thread) or per point.
template <int PP, class Load>
__device__ __forceinline__ void prod_pair_g(const ScRoundArgs& A, Load load, int pcnt,
                                            const uint32_t (&tpt)[PP], bool first, const fr& w,
                                            fr (&acc)[PP], uint32_t& bad) {
  const int d = (int)A.d, c = A.c;
  fr prod[PP];
  for (int j = 0; j < d; j++) {
    fr lo, hi;
    load(j, lo, hi);
    if (first) bad |= (!fr_is_canonical(lo)) | (!fr_is_canonical(hi));
    const fr dl = fr_sub(hi, lo);
    fr e = lo;
    uint32_t tcur = 0;
#pragma unroll
    for (int p = 0; p < PP; p++) {
      if (p >= pcnt) break;
      fr x;
      if (tpt[p] == kInf) {
        x = dl;
      } else {
        if (p == 0) e = fr_add(lo, fr_mul_small(dl, tpt[p]));
        else
          for (uint32_t s2 = tcur; s2 < tpt[p]; s2++) e = fr_add(e, dl);
        tcur = tpt[p];
        x = e;
      }
      prod[p] = j == 0 ? x : fr_mul(prod[p], x);
    }
  }
  if (c > d) {
    const bool minus = (A.gate & 0xffu) == ZC_GATE_PRODUCT;  // o is subtracted; sum-gate columns add
    fr lo = fr_zero(), hi = fr_zero();  // degree-1 part at the two ends, level 0
    for (int j = d; j < c; j++) {
      fr xl, xh;
      load(j, xl, xh);
      if (first) bad |= (!fr_is_canonical(xl)) | (!fr_is_canonical(xh));
      lo = minus ? fr_sub(lo, xl) : fr_add(lo, xl);
      hi = minus ? fr_sub(hi, xh) : fr_add(hi, xh);
    }
    const bool scale_ends = PP > 1 && pcnt >= 2;
    if (scale_ends) {
      lo = fr_mul(lo, A.kcomp);
      hi = fr_mul(hi, A.kcomp);
    }
    const fr dl = fr_sub(hi, lo);
    fr e = lo;
    uint32_t tcur = 0;
#pragma unroll
    for (int p = 0; p < PP; p++) {
      if (p >= pcnt) break;
      if (tpt[p] == kInf) continue;  // infinity has no degree-1 term
      if (p == 0) e = fr_add(lo, fr_mul_small(dl, tpt[p]));
      else
        for (uint32_t s2 = tcur; s2 < tpt[p]; s2++) e = fr_add(e, dl);
      tcur = tpt[p];
      prod[p] = fr_add(prod[p], scale_ends ? e : fr_mul(e, A.kcomp));
    }
  }
#pragma unroll
  for (int p = 0; p < PP; p++)
    if (p < pcnt) acc[p] = fr_add(acc[p], fr_mul(prod[p], w));
}

template <int PP, bool COHERENT>
__device__ __forceinline__ void prod_pair(const ScRoundArgs& A, const fr* const* col, uint64_t k,
                                          uint64_t h, int pcnt, const uint32_t (&tpt)[PP],
                                          bool first, const fr& w, fr (&acc)[PP], uint32_t& bad) {
  prod_pair_g<PP>(
      A,
      [&](int j, fr& lo, fr& hi) {
        lo = ldt<COHERENT>(col[j] + k);
        hi = ldt<COHERENT>(col[j] + k + h);
      },
      pcnt, tpt, first, w, acc, bad);
}

// Plonk round i >= 2 on a chunk of PB pairs, the work of each pair spread
// over TPP threads (blockDim.x == TPP PB), so a round is a few
// multiplications deep instead of ~30:
//   1. fold by alpha_{i-1}: 16 items per pair (column, half), store, keep in
//      smem; thread (slot, pair) takes items slot, slot + TPP, ...;
//   2. items per pair: qM b, qR b, qO c at each finite point, the slope
//      product dqM db, and the eq weight E_hi E_lo;
//   3. thread (point, pair): s = a (qL + qM b) + qR b + qO c + qC at a finite
//      point, dqM db da at infinity, times the eq weight.
// FULL: points 0, 1, 2, inf; otherwise p0, 2, inf.  Thread t = point * PB +
// pair (t < NPT PB) adds its value into acc.  Pairs are the fastest thread
// index, so every warp-wide load or store is contiguous.
template <int PB>
struct PlonkChunkSmem {
  fr V[8][2][PB];  // folded lo / hi per column
  fr U[12][PB];    // products and the eq weight
};

// column j of pair p at point pt: 0 -> lo, 1 -> hi, 2 -> 2 hi - lo, 3 -> slope
template <int PB>
__device__ __forceinline__ fr plonk_at(const PlonkChunkSmem<PB>& S, int j, int p, int pt) {
  const fr lo = S.V[j][0][p], hi = S.V[j][1][p];
  if (pt == 0) return lo;
  if (pt == 1) return hi;
  const fr dl = fr_sub(hi, lo);
  return pt == 2 ? fr_add(hi, dl) : dl;
}

template <int PB, int TPP, bool FULL, bool COHERENT>
__device__ __forceinline__ void plonk_chunk(PlonkChunkSmem<PB>& S, const fr* const* src, fr* const* dst,
                                            uint64_t h, uint64_t kbase, const fr& alpha, uint32_t p0,
                                            const fr* ehi, const fr* elo, uint32_t mlo, fr& acc) {
  constexpr int NPT = FULL ? 4 : 3, NF = NPT - 1, NITEM = 3 * NF + 2;
  static_assert(TPP >= NPT, "one point per thread in phase 3");
  const int t = threadIdx.x, p = t % PB, slot = t / PB;
  const uint64_t k = kbase + p;
  const bool live = k < h;
  auto point = [&](int f) { return FULL ? f : (f == 0 ? (int)p0 : 2); };  // finite point f
#pragma unroll
  for (int item = slot; item < 16; item += TPP) {
    const int j = item >> 1, half = item & 1;
    const uint64_t e = k + (half ? h : 0);
    if (live) {
      const fr x0 = ldt<COHERENT>(src[j] + e), x1 = ldt<COHERENT>(src[j] + e + 2 * h);
      const fr v = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
      st_fr(dst[j] + e, v);
      S.V[j][half][p] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = slot; q < NITEM; q += TPP) {
    if (live) {
      fr u;
      if (q == NITEM - 1) {
        u = fr_mul(ldx<COHERENT>(ehi + (k >> mlo)), ldx<COHERENT>(elo + (k & ((1ull << mlo) - 1))));
      } else if (q == NITEM - 2) {
        u = fr_mul(plonk_at(S, 2, p, 3), plonk_at(S, 6, p, 3));  // dqM db
      } else {
        const int pt = point(q / 3), term = q % 3;
        const int ja = term == 0 ? 2 : (term == 1 ? 1 : 3);  // qM, qR, qO
        const int jb = term == 2 ? 7 : 6;                    // b, b, c
        u = fr_mul(plonk_at(S, ja, p, pt), plonk_at(S, jb, p, pt));
      }
      S.U[q][p] = u;
    }
  }
  __syncthreads();
  if (slot < NPT && live) {
    const int f = slot;
    fr v;
    if (f < NF) {
      const int pt = point(f);
      v = fr_mul(plonk_at(S, 5, p, pt), fr_add(plonk_at(S, 0, p, pt), S.U[3 * f][p]));
      v = fr_add(v, fr_add(fr_add(S.U[3 * f + 1][p], S.U[3 * f + 2][p]), plonk_at(S, 4, p, pt)));
    } else {
      v = fr_mul(S.U[NITEM - 2][p], plonk_at(S, 5, p, 3));
    }
    acc = fr_add(acc, fr_mul(v, S.U[NITEM - 1][p]));
  }
  __syncthreads();
}

// Sum the per-thread values of plonk_chunk over pairs: out[q] for q < NPT.
// Warp q adds point q's PB values with shuffles.
template <int PB, int NPT>
__device__ __forceinline__ void plonk_chunk_reduce(const fr& acc, fr* out) {
  __shared__ fr R[NPT * PB];
  const int t = threadIdx.x;
  if (t < NPT * PB) R[t] = acc;
  __syncthreads();
  const int lane = t & 31, q = t >> 5;
  if (q < NPT) {
    fr s = fr_zero();
    for (int p = lane; p < PB; p += 32) s = fr_add(s, R[q * PB + p]);
    s = warp_sum(s);
    if (lane == 0) out[q] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- kernels --

// Transcript: absorb the column roots, squeeze r_1..r_n; reset per-proof state.
// The hash chain is serial (thread 0); the n conversions to Montgomery form
// run on n threads afterwards.  Launched with at least kMaxN threads.
__global__ void k_sc_setup(ScSetupArgs A) {
  __shared__ fr raw[kMaxN];
  if (threadIdx.x < kMaxN) A.st->counter[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    uint32_t S[8];
    for (int i = 0; i < 8; i++) S[i] = A.S0[i];
    for (int j = 0; j < A.c; j++) tr_absorb32(S, A.roots + 32 * j);
    for (int i = 0; i < A.n; i++) raw[i] = tr_squeeze(S);
    for (int i = 0; i < 8; i++) A.st->S[i] = S[i];
    A.st->claim = fr_zero();
    A.st->ci = A.C->one;
    A.st->err = 0;
    A.st->go = 0;
  }
  __syncthreads();
  if ((int)threadIdx.x < A.n) A.st->r[threadIdx.x] = fr_mul(raw[threadIdx.x], A.C->r2);
}

// Factor tables of eq_{>i} for every round, and the derived-point choice.
__global__ void k_sc_eq(ScEqArgs A) {
  const DevConst* C = A.C;
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (uint32_t)A.n) {
    const fr r = A.st->r[e];
    const bool rzero = fr_is_zero(r), rone = fr_equal(r, C->one);
    A.st->p0[e] = A.skip_point == 0 ? (rzero ? 1u : 0u) : (rone ? 0u : 1u);
  }
  if (e >= A.total) return;
  uint32_t ti = 0;
  while (ti + 1 < A.ntask && A.task[ti + 1].offset <= e) ti++;
  const EqTask& T = A.task[ti];
  const uint32_t x = e - T.offset;
  fr acc = C->one;
  for (uint32_t l = 0; l < T.nvars; l++) {
    const uint32_t bit = (x >> (T.nvars - 1 - l)) & 1;
    const fr r = A.st->r[T.first_var + l];
    acc = fr_mul(acc, bit ? r : fr_sub(C->one, r));
  }
  if (T.level > 1) acc = fr_mul(acc, C->rpow[T.level]);  // level 1 -> level L
  st_fr(A.E + e, acc);
}

// 1/r_i and 1/(1 - r_i) (level 1, 0 for a zero input) for i < n, by one
// batch inversion (Montgomery's trick): prefix and suffix products of the 2n
// values (Hillis-Steele scans in shared memory), a single binary-GCD
// inversion of their product, then inv_t = prefix_{t-1} suffix_{t+1} / P.
// All threads of the CTA (at least 64) reach every barrier.
__device__ void sc_inverses(ScState* st, int n, const DevConst* C) {
  __shared__ fr pre[2 * kMaxN], suf[2 * kMaxN];
  __shared__ fr total_inv;
  const int t = threadIdx.x, m = 2 * n;
  bool zero = false;
  fr x = C->one;
  if (t < m) {
    const fr r = st->r[t >> 1];
    x = (t & 1) ? fr_sub(C->one, r) : r;  // level 1
    zero = fr_is_zero(x);
    if (zero) x = C->one;  // leave it out of the product
    pre[t] = x;
    suf[t] = x;
  }
  __syncthreads();
  for (int off = 1; off < m; off <<= 1) {
    fr a, b;
    if (t < m) {
      a = t >= off ? fr_mul(pre[t - off], pre[t]) : pre[t];
      b = t + off < m ? fr_mul(suf[t], suf[t + off]) : suf[t];
    }
    __syncthreads();
    if (t < m) {
      pre[t] = a;
      suf[t] = b;
    }
    __syncthreads();
  }
  if (t == 0) {
    // pre[m-1] = P R (level 1); inv_binary gives P^-1 R^-1; times R^3 -> P^-1 R
    total_inv = fr_mul(fr_inv_binary(pre[m - 1]), C->rpow[3]);
  }
  __syncthreads();
  if (t < m) {
    fr inv = total_inv;
    if (t > 0) inv = fr_mul(inv, pre[t - 1]);
    if (t + 1 < m) inv = fr_mul(inv, suf[t + 1]);
    if (zero) inv = fr_zero();
    if (t & 1) st->r1inv[t >> 1] = inv;
    else st->rinv[t >> 1] = inv;
  }
}

// One large Plonk round on the whole GPU.  FIRST: round 1 (reads the input,
// converts a, b, c, evaluates t = 0, 1, 2, inf; the extra last CTA computes
// the inverses used from round 2 on).  Otherwise: folds by alpha_{i-1} and
// evaluates t = p0, 2, inf.  The last CTA to finish runs the challenge.
template <bool FIRST, int MINB>
__global__ void __launch_bounds__(256, MINB) k_sc_plonk_round(ScRoundArgs A) {
  constexpr int NP = FIRST ? 4 : 3;
  if (FIRST && blockIdx.x == A.nwork) {
    sc_inverses(A.st, A.n, A.C);
    return;
  }
  const int i = A.round;
  const uint64_t h = A.h;
  const uint32_t mlo = A.m_lo[i];
  const fr* ehi = A.E + A.eq_hi[i];
  const fr* elo = A.E + A.eq_lo[i];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t T = (uint64_t)A.nwork * blockDim.x;
  const uint64_t kend = A.k1 ? A.k1 : h;
  fr acc[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) acc[p] = fr_zero();
  const fr alpha = FIRST ? fr_zero() : A.st->alpha[i - 1];
  const uint32_t p0 = FIRST ? 0u : A.st->p0[i];
  uint32_t bad = 0;
  for (uint64_t k = A.k0 + tid; k < kend; k += T)
    plonk_pair<FIRST, false>(A.src, A.dst, A.C, k, h, alpha, p0, ld_fr(ehi + (k >> mlo)), acc, bad);
  if (FIRST && bad) atomicOr(&A.st->err, 1u);
  // each thread handled pairs with one fixed low part k_lo (k0 and T are
  // multiples of 2^mlo)
  const fr wl = ld_fr(elo + (tid & ((1ull << mlo) - 1)));
#pragma unroll
  for (int p = 0; p < NP; p++) acc[p] = fr_mul(acc[p], wl);
  block_sum<NP>(acc, A.partials + (size_t)(A.cta0 + blockIdx.x) * NP);
  sc_finish_round(A, NP);
}

// One Plonk round i >= 2 in chunks of PB pairs, each pair's work spread over
// TPP threads (plonk_chunk).  FULL: all of H(0), H(1), H(2),
// H(inf) (small rounds: no inverse needed); otherwise H(p0), H(2), H(inf).
// The last CTA to finish runs the challenge.
template <int TPP, int PB, bool FULL>
__global__ void __launch_bounds__(TPP * PB) k_sc_plonk_chunk(ScRoundArgs A) {
  constexpr int NPT = FULL ? 4 : 3;
  __shared__ PlonkChunkSmem<PB> S;
  __shared__ fr part[NPT];
  const int i = A.round;
  const fr alpha = A.st->alpha[i - 1];
  const uint32_t p0 = FULL ? 0u : A.st->p0[i];
  fr acc = fr_zero();
  for (uint64_t kb = (uint64_t)blockIdx.x * PB; kb < A.h; kb += (uint64_t)A.nwork * PB)
    plonk_chunk<PB, TPP, FULL, false>(S, A.src, A.dst, A.h, kb, alpha, p0, A.E + A.eq_hi[i],
                                      A.E + A.eq_lo[i], A.m_lo[i], acc);
  plonk_chunk_reduce<PB, NPT>(acc, part);
  if (threadIdx.x < NPT) st_fr(A.partials + (size_t)blockIdx.x * NPT + threadIdx.x, part[threadIdx.x]);
  __syncthreads();
  sc_finish_round(A, NPT);
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Plonk rounds [A.round, A.round_end) in one cooperative launch, so the
// latency-bound rounds pay no launch between them and their challenge code
// stays warm.  Rounds with more than A.small_pairs pairs take 4 threads per
// pair and derive one of H(0), H(1) from the claim (as k_sc_plonk_chunk<4,
// 32>); smaller ones take 16 threads per pair and evaluate every point.
// Each CTA folds and evaluates its chunks of a round and writes its partial
// sums; the last CTA to arrive sums them, runs the challenge and releases the
// next round through st->go.  The other CTAs poll st->go at most
// A.spin_limit times; a CTA that gives up sets bit 1 of st->err and returns,
// after which every later hand-off also gives up, so the launch always ends
// and the proof reports the timeout.  Tables are read through L2: other CTAs
// rewrote them in the previous round.  Dynamic shared memory: kRoundsDyn.
constexpr size_t kRoundsDyn = sizeof(PlonkChunkSmem<kBigPB>) > sizeof(PlonkChunkSmem<kSmallPB>)
                                  ? sizeof(PlonkChunkSmem<kBigPB>)
                                  : sizeof(PlonkChunkSmem<kSmallPB>);
__global__ void __launch_bounds__(16 * kSmallPB) k_sc_plonk_rounds(ScRoundArgs A) {
  static_assert(4 * kBigPB == 16 * kSmallPB, "both chunk shapes fill the CTA");
  extern __shared__ __align__(16) unsigned char rounds_smem[];
  auto& S = *reinterpret_cast<PlonkChunkSmem<kSmallPB>*>(rounds_smem);
  auto& SB = *reinterpret_cast<PlonkChunkSmem<kBigPB>*>(rounds_smem);
  __shared__ fr part[4];
  __shared__ ChalSmem CS;
  __shared__ int flag;  // 1: this CTA runs the challenge; 2: a wait gave up
  const uint32_t G = gridDim.x;
  const uint64_t N = 1ull << A.n;
  for (int i = A.round; i < A.round_end; i++) {
    const uint64_t h = N >> (i + 1);
    const bool big = h > A.small_pairs;
    const int np = big ? 3 : 4;
    const uint64_t pb = big ? kBigPB : kSmallPB;
    const uint32_t nwork = (uint32_t)min((h + pb - 1) / pb, (uint64_t)G);
    const fr alpha = ld_fr_l2(&A.st->alpha[i - 1]);
    const fr* const* src = i == A.round ? (const fr* const*)A.src : (const fr* const*)A.dst;
    fr acc = fr_zero();
    if (big) {
      const uint32_t p0 = A.st->p0[i];
      if (blockIdx.x < nwork)
        for (uint64_t kb = (uint64_t)blockIdx.x * kBigPB; kb < h; kb += (uint64_t)nwork * kBigPB)
          plonk_chunk<kBigPB, 4, false, true>(SB, src, A.dst, h, kb, alpha, p0, A.E + A.eq_hi[i],
                                               A.E + A.eq_lo[i], A.m_lo[i], acc);
      plonk_chunk_reduce<kBigPB, 3>(acc, part);
    } else {
      if (blockIdx.x < nwork)
        for (uint64_t kb = (uint64_t)blockIdx.x * kSmallPB; kb < h; kb += (uint64_t)nwork * kSmallPB)
          plonk_chunk<kSmallPB, 16, true, true>(S, src, A.dst, h, kb, alpha, 0u, A.E + A.eq_hi[i],
                                                A.E + A.eq_lo[i], A.m_lo[i], acc);
      plonk_chunk_reduce<kSmallPB, 4>(acc, part);
    }
    if (blockIdx.x < nwork && (int)threadIdx.x < np)
      st_fr(A.partials + (size_t)blockIdx.x * np + threadIdx.x, part[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&A.st->counter[i], 1u);
      flag = prev == G - 1 ? 1 : 0;
    }
    __syncthreads();
    if (flag == 1) {
      __threadfence();
      sc_sum_partials(CS, A.partials, nwork, np);
      // the next round needs the claim when it derives a point too
      sc_challenge<false>(CS, np, 3, i, A.st, A.proof, A.C, A.tabs, h / 2 > A.small_pairs, A.v2 != 0,
                          &A.st->go);
    } else {
      if (threadIdx.x == 0) {
        uint32_t polls = 0;
        while (ld_acquire_u32(&A.st->go) < (uint32_t)(i + 1)) {
          if (++polls > A.spin_limit) {
            atomicOr(&A.st->err, 2u);
            flag = 2;
            break;
          }
          __nanosleep(256);
        }
      }
      __syncthreads();
      if (flag == 2) return;
    }
    __syncthreads();
  }
}

// MLE update by alpha_{round-1}: dst[j][k] = src[j][k] + alpha (src[j][k+h] - src[j][k])
__global__ void __launch_bounds__(256) k_sc_fold(ScFoldArgs A) {
  const fr alpha = A.st->alpha[A.round - 1];
  const uint64_t total = A.h * (uint64_t)A.c;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / A.h);
    const uint64_t k = e - (uint64_t)j * A.h;
    const fr x0 = ld_fr_cs(A.src[j] + k), x1 = ld_fr_cs(A.src[j] + k + A.h);
    st_fr(A.dst[j] + k, fr_add(x0, fr_mul(alpha, fr_sub(x1, x0))));
  }
}

// A product CTA's partial sums: point q is the sum of red[sl G + q / PP][q % PP]
// over its spb pair slots.  Warps take points, lanes take slots.
template <int PP>
__device__ __forceinline__ void prod_cta_sums(const fr (&red)[256][PP], int np, int G, int spb, fr* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < np; q += nw) {
    const int gq = q / PP, pq = q % PP;
    fr v = fr_zero();
    for (int sl = lane; sl < spb; sl += 32) v = fr_add(v, red[sl * G + gq][pq]);
    v = warp_sum(v);
    if (lane == 0) st_fr(out + q, v);
  }
}

// Product-gate evaluation of one large round (columns already folded): G =
// ceil(np / PP) threads per pair, each evaluating up to PP consecutive
// points (the extensions lo + t (hi - lo) advance by one addition per
// point), floor(256 / G) pairs per CTA in flight.
template <int PP>
__global__ void __launch_bounds__(256, PP == 1 ? 3 : 2) k_sc_prod_round(ScRoundArgs A) {
  const int i = A.round;
  const bool first = i == 0;
  if (first && blockIdx.x == A.nwork) {
    sc_inverses(A.st, A.n, A.C);
    return;
  }
  const int d = (int)A.d;
  const bool full = first || A.full;
  const int np = full ? d + 1 : d;
  const uint32_t p0 = full ? 0u : A.st->p0[i];
  const int G = (np + PP - 1) / PP;
  const int spb = (int)A.spb;
  const int slot = (int)threadIdx.x / G, g = (int)threadIdx.x % G;
  const int pbeg = g * PP, pcnt = max(0, min(PP, np - pbeg));
  const uint32_t mlo = A.m_lo[i];
  const fr* ehi = A.E + A.eq_hi[i];
  const fr* elo = A.E + A.eq_lo[i];
  uint32_t bad = 0;
  fr acc[PP];
  uint32_t tpt[PP];
#pragma unroll
  for (int p = 0; p < PP; p++) {
    acc[p] = fr_zero();
    tpt[p] = p < pcnt ? prod_point(pbeg + p, np, full, p0) : 0u;
  }
  if (slot < spb) {
    const uint64_t kend = A.k1 ? A.k1 : A.h;
    for (uint64_t k = A.k0 + (uint64_t)blockIdx.x * spb + slot; k < kend; k += (uint64_t)A.nwork * spb) {
      const fr w = fr_mul(ld_fr(ehi + (k >> mlo)), ld_fr(elo + (k & ((1ull << mlo) - 1))));
      prod_pair<PP, false>(A, A.src, k, A.h, pcnt, tpt, first && g == 0, w, acc, bad);
    }
  }
  if (bad) atomicOr(&A.st->err, 1u);
  __shared__ fr red[256][PP];
#pragma unroll
  for (int p = 0; p < PP; p++) red[threadIdx.x][p] = acc[p];
  __syncthreads();
  prod_cta_sums<PP>(red, np, G, spb, A.partials + (size_t)(A.cta0 + blockIdx.x) * np);
  __syncthreads();
  sc_finish_round(A, np);
}

// Product-gate round i >= 2 with the MLE update fused: each CTA first
// folds the (d+1) columns of its spb pairs by alpha_{i-1} (all threads,
// coalesced; written back and kept in shared memory), then evaluates them
// from shared memory as k_sc_prod_round does.  Dynamic shared memory:
// (d+1) x 2 x spb elements.
template <int PP>
__global__ void __launch_bounds__(256, 2) k_sc_prod_fused(ScRoundArgs A) {
  extern __shared__ __align__(16) fr Vs[];
  const int i = A.round;
  const int d = (int)A.d, c = A.c;
  const bool full = A.full != 0;
  const int np = full ? d + 1 : d;
  const uint32_t p0 = full ? 0u : A.st->p0[i];
  const int G = (np + PP - 1) / PP;
  const int spb = (int)A.spb;
  const int slot = (int)threadIdx.x / G, g = (int)threadIdx.x % G;
  const int pbeg = g * PP, pcnt = max(0, min(PP, np - pbeg));
  const uint32_t mlo = A.m_lo[i];
  const fr* ehi = A.E + A.eq_hi[i];
  const fr* elo = A.E + A.eq_lo[i];
  const fr alpha = A.st->alpha[i - 1];
  const uint64_t h = A.h;
  uint32_t bad = 0;
  fr acc[PP];
  uint32_t tpt[PP];
#pragma unroll
  for (int p = 0; p < PP; p++) {
    acc[p] = fr_zero();
    tpt[p] = p < pcnt ? prod_point(pbeg + p, np, full, p0) : 0u;
  }
  for (uint64_t kb = (uint64_t)blockIdx.x * spb; kb < h; kb += (uint64_t)A.nwork * spb) {
    for (int e = threadIdx.x; e < c * 2 * spb; e += blockDim.x) {
      const int p = e % spb, rest = e / spb, half = rest & 1, j = rest >> 1;
      const uint64_t k = kb + p;
      if (k < h) {
        const uint64_t idx = k + (half ? h : 0);
        const fr x0 = ld_fr_cs(A.src[j] + idx), x1 = ld_fr_cs(A.src[j] + idx + 2 * h);
        const fr v = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
        st_fr(A.dst[j] + idx, v);
        Vs[(size_t)rest * spb + p] = v;
      }
    }
    __syncthreads();
    const uint64_t k = kb + slot;
    if (slot < spb && k < h) {
      const fr w = fr_mul(ld_fr(ehi + (k >> mlo)), ld_fr(elo + (k & ((1ull << mlo) - 1))));
      prod_pair_g<PP>(
          A,
          [&](int j, fr& lo, fr& hi) {
            lo = Vs[(size_t)(2 * j) * spb + slot];
            hi = Vs[(size_t)(2 * j + 1) * spb + slot];
          },
          pcnt, tpt, false, w, acc, bad);
    }
    __syncthreads();
  }
  __shared__ fr red[256][PP];
#pragma unroll
  for (int p = 0; p < PP; p++) red[threadIdx.x][p] = acc[p];
  __syncthreads();
  prod_cta_sums<PP>(red, np, G, spb, A.partials + (size_t)blockIdx.x * np);
  __syncthreads();
  sc_finish_round(A, np);
}

// All rounds from A.round on, their challenges and the final values, in one
// CTA of kTailThreads threads.  Tables are read with coherent loads: they
// are rewritten between rounds inside this launch.
template <bool PLONK>
__global__ void __launch_bounds__(PLONK ? kTailThreads : 256, 1) k_sc_tail(ScRoundArgs A) {
  __shared__ ChalSmem S;
  __shared__ fr pg[kMaxPts];
  const DevConst* C = A.C;
  const int n = A.n, c = A.c, d = (int)A.d;
  constexpr bool plonk = PLONK;
  const uint64_t N = 1ull << n;
  uint32_t bad = 0;
  // source of round i's pairs: the input for round 0, then the folded tables
  const fr* cur[kMaxCols];
  for (int j = 0; j < c; j++) cur[j] = A.src[j];
  for (int i = A.round; i < n; i++) {
    const uint64_t h = N >> (i + 1);
    const uint32_t mlo = A.m_lo[i];
    const fr* ehi = A.E + A.eq_hi[i];
    const fr* elo = A.E + A.eq_lo[i];
    int np;
    if constexpr (PLONK) {
      {  // i >= 1: round 1 never runs in the Plonk tail
        np = 4;
        fr acc = fr_zero();
        const fr alpha = A.st->alpha[i - 1];
        __shared__ PlonkChunkSmem<kTailPB> PS;
        for (uint64_t kb = 0; kb < h; kb += kTailPB)
          plonk_chunk<kTailPB, 16, true, true>(PS, cur, A.dst, h, kb, alpha, 0u, ehi, elo, mlo, acc);
        plonk_chunk_reduce<kTailPB, 4>(acc, pg);
      }
      for (int j = 0; j < c; j++) cur[j] = A.dst[j];
    } else {
      if (i > 0) {
        const fr alpha = A.st->alpha[i - 1];
        for (uint64_t e = threadIdx.x; e < 2 * h * (uint64_t)c; e += blockDim.x) {
          const int j = (int)(e / (2 * h));
          const uint64_t k = e - (uint64_t)j * 2 * h;
          const fr x0 = ld_fr_l2(cur[j] + k), x1 = ld_fr_l2(cur[j] + k + 2 * h);
          st_fr(A.dst[j] + k, fr_add(x0, fr_mul(alpha, fr_sub(x1, x0))));
        }
        __syncthreads();
        for (int j = 0; j < c; j++) cur[j] = A.dst[j];
      }
      // every tail round evaluates all of 0..d-1 and infinity (no derived point)
      const bool first = i == 0;
      np = d + 1;
      const int G = A.G;
      const int g = threadIdx.x % G;
      const uint64_t nslots = blockDim.x / G;
      const int pbeg = g * kPP, pcnt = max(0, min(kPP, np - pbeg));
      fr acc[kPP];
      uint32_t tpt[kPP];
#pragma unroll
      for (int p = 0; p < kPP; p++) {
        acc[p] = fr_zero();
        tpt[p] = p < pcnt ? prod_point(pbeg + p, np, true, 0u) : 0u;
      }
      for (uint64_t k = threadIdx.x / G; k < h && pcnt > 0; k += nslots) {
        const fr w = fr_mul(ld_fr_cg(ehi + (k >> mlo)), ld_fr_cg(elo + (k & ((1ull << mlo) - 1))));
        prod_pair<kPP, true>(A, cur, k, h, pcnt, tpt, first, w, acc, bad);
      }
      // sum each point over all threads (threads outside its group add zero)
      for (int p = 0; p < np; p++) {
        fr v[1] = {(p >= pbeg && p < pbeg + pcnt) ? acc[p - pbeg] : fr_zero()};
        block_sum<1>(v, pg + p);
      }
    }
    for (int p = threadIdx.x; p < np; p += blockDim.x) S.Hc[p] = pg[p];
    __syncthreads();
    sc_challenge<false>(S, np, d, i, A.st, A.proof, C, A.tabs, false, A.v2 != 0);
  }
  if (bad) atomicOr(&A.st->err, 1u);
  __syncthreads();
  // final values v_j = T_j[0] + alpha_n (T_j[1] - T_j[0]); Plonk wires are at level 1
  uint8_t* pv = A.proof + 16 + 32 * ((size_t)n * (A.v2 ? d + 1 : d + 2));
  if (threadIdx.x < (unsigned)c) {
    const int j = threadIdx.x;
    const fr alpha = A.st->alpha[n - 1];
    const fr x0 = ld_fr_l2(cur[j]), x1 = ld_fr_l2(cur[j] + 1);
    fr v = fr_add(x0, fr_mul(alpha, fr_sub(x1, x0)));
    if (plonk && j >= 5) v = from_mont(v);
    for (int q = 0; q < 8; q++)
      for (int b = 0; b < 4; b++) pv[32 * j + 4 * q + b] = (uint8_t)(v.v[q] >> (8 * b));
  }
  if (threadIdx.x == 0) {
    const uint32_t e = A.st->err;
    const char* mg = (e & 2u) ? "ZCT!" : (e ? "ZCE!" : (A.v2 ? "ZCS2" : "ZCS1"));
    for (int b = 0; b < 4; b++) A.proof[b] = (uint8_t)mg[b];
    const uint32_t hv[3] = {A.gate, (uint32_t)n, A.d};
    for (int q = 0; q < 3; q++)
      for (int b = 0; b < 4; b++) A.proof[4 + 4 * q + b] = (uint8_t)(hv[q] >> (8 * b));
  }
}

// ------------------------------------------------------------------ host --

static void eq_round_split(int n, int round, uint32_t* m_lo, uint32_t* m_hi) {
  const uint32_t m = (uint32_t)(n - 1 - round);  // variables after x_{round+1}
  uint32_t lo = m / 2;
  if (lo > 11) lo = 11;
  *m_lo = lo;
  *m_hi = m - lo;
}

// Buffers of one SumCheck proof (device).
struct ScBuffers {
  fr* tab[kMaxCols];
  fr* partials;
  fr* E;
  ScState* st;
  uint8_t* roots;
  uint8_t* proof;
};

struct ScPlan {
  int c, G, grid_plonk, grid_prod, npmax;
  uint64_t tail_pairs, small_pairs, chunk_pairs;
  int grid_chunk, grid_quad;
  int grid_rounds;      // co-resident CTAs of the persistent round kernel
  uint64_t quad_pairs;  // Plonk rounds 2.. in (chunk_pairs, quad_pairs]: 4 threads per pair
  int minb;  // Plonk round kernels: resident CTAs per SM they are compiled for
  int ppt;   // product round kernel: points per thread (1 or kPP; 0: by round, prod_ppt)
  uint64_t fuse_pairs;  // product rounds 2.. with at most this many pairs fold inside the evaluation
  int upload_chunks = 0;  // round 1 in this many pair-range launches (host columns), 0: one launch
  uint32_t eq_total, eq_hi[kMaxN], eq_lo[kMaxN], mlo[kMaxN];
  EqTask tasks[2 * kMaxN];
};

// grid: most CTAs per round kernel (0: two per SM); tail_log: the tail takes
// over at 2^tail_log pairs (0: the gate's default).
// The fused product kernel takes up to 48 KB of dynamic shared memory on top
// of its static arrays: opt in once per device.
static void ensure_prod_fused_attr() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_sc_prod_fused<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
  cudaFuncSetAttribute(k_sc_prod_fused<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 << 10);
  cudaFuncSetAttribute(k_sc_plonk_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRoundsDyn);
  done[dev] = true;
}

// Points per thread of a product round with np points over h pairs: one
// (np threads per pair, the shortest chain) in small rounds, which are
// latency-bound; in large rounds three when that is one thread per pair
// (d = 2), one for 4-5 points, else three (extensions by additions, fewer
// redundant loads).
static int prod_ppt(int forced, int np, uint64_t h) {
  if (forced) return forced;
  if (h <= (1ull << 16)) return 1;  // small rounds: shortest per-thread chain
  if (np <= 3) return 3;            // one thread per pair
  return np <= 5 ? 1 : 3;
}

// Resident CTAs per SM of a kernel on the current device (cached).
static int resident_ctas(const void* fn, int threads = 256, size_t dyn = 0) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : cache)
    if (e.first.first == dev && e.first.second == fn) return e.second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, dyn) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  cache.push_back({{dev, fn}, nb});
  return nb;
}

static const void* plonk_round_fn(int minb) {
  return minb == 2 ? reinterpret_cast<const void*>(k_sc_plonk_round<false, 2>)
                   : reinterpret_cast<const void*>(k_sc_plonk_round<false, 1>);
}

static ScPlan sc_plan(const zc_params* p, int SMs, int grid = 0, int tail_log = 0, int small_log = 0,
                      int minb = 0, int ppt = 0, int chunk_log = 0, int quad_log = 0, int fuse = 0) {
  ScPlan P{};
  const uint32_t n = p->n, d = p->d;
  const bool plonk = p->gate == ZC_GATE_PLONK;
  P.c = gate_ncols(p->gate, d);
  P.G = 1;
  while (P.G * kPP < (int)d + 1) P.G *= 2;
  // default: one wave of resident CTAs for the Plonk kernels (register bound,
  // one CTA per SM), two waves for the product kernel
  P.grid_plonk = grid > 0 ? grid : SMs * resident_ctas(plonk_round_fn(minb == 1 ? 1 : 2));
  P.ppt = ppt == 1 || ppt == 3 ? ppt : 0;  // 0: per round (see prod_ppt)
  P.fuse_pairs = fuse > 0 ? 1ull << fuse : kFusePairsProd;
  ensure_prod_fused_attr();
  P.grid_prod = grid > 0 ? grid
                         : 2 * SMs * std::max(resident_ctas(reinterpret_cast<const void*>(k_sc_prod_round<1>)),
                                              resident_ctas(reinterpret_cast<const void*>(k_sc_prod_round<3>)));
  P.tail_pairs = tail_log > 0 ? 1ull << tail_log : (plonk ? kTailPairsPlonk : kTailPairsProd);
  P.small_pairs = small_log > 0 ? 1ull << small_log : kSmallPairsPlonk;
  P.chunk_pairs = chunk_log > 0 ? 1ull << chunk_log : kChunkPairsPlonk;
  P.grid_chunk = SMs * resident_ctas(reinterpret_cast<const void*>(k_sc_plonk_chunk<16, kSmallPB, false>));
  P.grid_rounds = SMs * resident_ctas(reinterpret_cast<const void*>(k_sc_plonk_rounds), 16 * kSmallPB, kRoundsDyn);
  P.quad_pairs = quad_log > 0 ? 1ull << quad_log : kQuadPairsPlonk;
  P.grid_quad = SMs * resident_ctas(reinterpret_cast<const void*>(k_sc_plonk_chunk<4, kQuadPB, false>), 4 * kQuadPB);
  P.minb = minb == 1 ? 1 : 2;
  P.npmax = (int)d + 1;
  for (uint32_t i = 0; i < n; i++) {
    uint32_t mlo, mhi;
    eq_round_split((int)n, (int)i, &mlo, &mhi);
    P.mlo[i] = mlo;
    P.tasks[2 * i] = EqTask{P.eq_total, i + 1, mhi, plonk ? 1u : d};
    P.eq_hi[i] = P.eq_total;
    P.eq_total += 1u << mhi;
    P.tasks[2 * i + 1] = EqTask{P.eq_total, n - mlo, mlo, 1u};
    P.eq_lo[i] = P.eq_total;
    P.eq_total += 1u << mlo;
  }
  return P;
}

static size_t sc_partials_count(const ScPlan& P) {
  const size_t g = (size_t)std::max(std::max(P.grid_plonk, P.grid_prod), std::max(P.grid_chunk, P.grid_quad));
  return (g * (size_t)std::max(1, P.upload_chunks) + 1) * (P.npmax + 1);
}

// Host columns of a large instance are copied in kUploadChunks pair ranges
// (rows [a, a + h/K) and [h + a, h + a + h/K) of every column), and round 1
// runs on each range as soon as it has landed, so the copy overlaps it.
constexpr int kUploadChunks = 8;
constexpr uint32_t kUploadMinN = 18;

static bool sc_upload_chunkable(const zc_params* p) { return p->n >= kUploadMinN; }

struct ScUpload {
  const void* const* cols;  // host columns (canonical, N * 32 bytes each)
  int chunks;
  uint64_t hc;              // pairs per range
  cudaStream_t stream;
  cudaEvent_t fork;
  const cudaEvent_t* ev;    // one per range
};

// Carve the proof's buffers from an arena; false when it is too small.
static bool sc_carve(Arena& ar, const ScPlan& P, uint64_t N, size_t psize, ScBuffers& B) {
  for (int j = 0; j < P.c; j++) B.tab[j] = ar.take<fr>(N);
  B.partials = ar.take<fr>(sc_partials_count(P));
  B.E = ar.take<fr>(P.eq_total);
  B.st = ar.take<ScState>(1);
  B.roots = ar.take<uint8_t>(32 * (size_t)P.c);
  B.proof = ar.take<uint8_t>(psize);
  return B.tab[P.c - 1] && B.partials && B.E && B.st && B.roots && B.proof;
}

// Polls of a persistent round kernel's hand-off before it gives up (about a
// second); ZC_SPIN_LIMIT overrides it (tests make the wait run out).
static uint32_t persistent_spin_limit() {
  const char* e = std::getenv("ZC_SPIN_LIMIT");
  if (e && *e) return (uint32_t)std::strtoul(e, nullptr, 10);
  return 1u << 22;
}

// Whether a proof on this context may use the persistent round kernel: not
// on batch or serving lanes (their kernels share the GPU with other
// instances' kernels, and a batch is captured into a graph), and not when
// ZC_SC_PERSISTENT=0.
static bool persistent_allowed(const zc_ctx* ctx, cudaStream_t st) {
  const char* e = std::getenv("ZC_SC_PERSISTENT");
  if (e && e[0] == '0') return false;
  if (ctx->table_owner) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}

// Queue every kernel of one proof on st (B.roots must hold the column roots
// by the time the queue runs).  ev: optional events; [2] and [3] bracket the
// round-1 launch.
static zc_status sc_enqueue(const zc_params* p, const ScPlan& P, const fr* const* src,
                            const ScBuffers& B, const DevConst* dC, const fr* dtabs,
                            const DevConst& hC, int skip_point, cudaStream_t st,
                            uint32_t* launches, cudaEvent_t* ev, bool v2 = false,
                            bool persistent = false, const ScUpload* up = nullptr) {
  const uint32_t gate = p->gate, n = p->n, d = p->d;
  const int c = P.c;
  const uint64_t N = 1ull << n;
  const bool plonk = gate == ZC_GATE_PLONK;
  if (up) {  // the copies start at once, behind earlier work on st
    if (cudaEventRecord(up->fork, st) != cudaSuccess || cudaStreamWaitEvent(up->stream, up->fork, 0) != cudaSuccess)
      return ZC_ERR_CUDA;
  }
  // range q of the host columns to the tables, then st waits for it
  auto upload_range = [&](int q) -> bool {
    const uint64_t h0 = N / 2, a = (uint64_t)q * up->hc;
    for (int j = 0; j < c; j++) {
      const char* hs = static_cast<const char*>(up->cols[j]);
      if (cudaMemcpyAsync(B.tab[j] + a, hs + a * sizeof(fr), up->hc * sizeof(fr), cudaMemcpyHostToDevice,
                          up->stream) != cudaSuccess ||
          cudaMemcpyAsync(B.tab[j] + h0 + a, hs + (h0 + a) * sizeof(fr), up->hc * sizeof(fr),
                          cudaMemcpyHostToDevice, up->stream) != cudaSuccess)
        return false;
    }
    return cudaEventRecord(up->ev[q], up->stream) == cudaSuccess &&
           cudaStreamWaitEvent(st, up->ev[q], 0) == cudaSuccess;
  };
  ScSetupArgs sa{};
  sa.st = B.st;
  sa.roots = B.roots;
  transcript_init_words(sa.S0, v2 ? ZC_FORM_SUMCHECK_EQ : ZC_FORM_SUMCHECK, gate, n, d, 0);
  sa.c = c;
  sa.n = (int)n;
  sa.C = dC;
  k_sc_setup<<<1, 32, 0, st>>>(sa);
  ScEqArgs ea{};
  ea.st = B.st;
  ea.E = B.E;
  for (uint32_t t = 0; t < 2 * n; t++) ea.task[t] = P.tasks[t];
  ea.ntask = 2 * n;
  ea.total = P.eq_total;
  ea.n = (int)n;
  ea.skip_point = skip_point;
  ea.C = dC;
  k_sc_eq<<<(std::max<uint32_t>(P.eq_total, n) + 255) / 256, 256, 0, st>>>(ea);
  *launches += 2;
  if (ev) cudaEventRecord(ev[2], st);

  ScRoundArgs R{};
  R.E = B.E;
  for (uint32_t i = 0; i < n; i++) {
    R.eq_hi[i] = P.eq_hi[i];
    R.eq_lo[i] = P.eq_lo[i];
    R.m_lo[i] = P.mlo[i];
  }
  R.n = (int)n;
  R.c = c;
  R.gate = gate;
  R.d = d;
  R.G = P.G;
  R.st = B.st;
  R.partials = B.partials;
  R.proof = B.proof;
  R.kcomp = hC.rnegpow[d - 2];
  R.C = dC;
  R.tabs = dtabs;
  R.v2 = v2 ? 1u : 0u;
  const uint64_t tail_pairs = P.tail_pairs;
  const fr* cur[kMaxCols];
  for (int j = 0; j < c; j++) cur[j] = src[j];
  uint32_t i = 0;
  // Rounds i >= 2 with more than small_pairs pairs take one of H(0), H(1)
  // from the claim, which needs 1/r_i and 1/(1 - r_i): an extra CTA of round
  // 1 computes them, only when such a round exists.
  // Whether round i (h pairs, not in the tail) evaluates all points: round 1
  // always; later rounds when small, and for the Plonk gate only in the
  // chunk kernel (the pair kernel always derives a point).
  auto round_full = [&](uint32_t r, uint64_t hh) {
    if (r == 0) return true;
    if (hh > P.small_pairs) return false;
    return !plonk || hh <= std::max(P.chunk_pairs, P.quad_pairs);
  };
  bool need_inv = false;
  for (uint32_t r = 1; r < n && (N >> (r + 1)) > tail_pairs; r++) need_inv |= !round_full(r, N >> (r + 1));
  const uint32_t inv_cta = need_inv ? 1u : 0u;
  for (; i < n; i++) {
    const uint64_t h = N >> (i + 1);
    // the Plonk tail starts at round 2 at the earliest: round 1 always runs the
    // pair kernel, so the tail carries no round-1 code (fewer registers)
    if (h <= tail_pairs && !(plonk && i == 0)) break;
    R.round = (int)i;
    R.h = h;
    R.full = round_full(i, h) ? 1u : 0u;
    R.next_derives = (h / 2 > tail_pairs && !round_full(i + 1, h / 2)) ? 1u : 0u;
    for (int j = 0; j < c; j++) {
      R.src[j] = cur[j];
      R.dst[j] = B.tab[j];
    }
    const uint64_t coop_max = n >= kCoopQuadMinN ? std::max(P.chunk_pairs, P.quad_pairs) : P.chunk_pairs;
    if (plonk && i > 0 && h <= coop_max && persistent && (R.full || n >= kCoopQuadMinN) && h / 2 > tail_pairs) {
      // every remaining round before the tail in one cooperative launch
      // (those above small_pairs derive a point, the others evaluate every point)
      uint32_t end = i;
      while (end < n && (N >> (end + 1)) > tail_pairs) end++;
      R.round_end = (int)end;
      R.spin_limit = persistent_spin_limit();
      R.small_pairs = P.small_pairs;
      const uint64_t pb0 = h > P.small_pairs ? (uint64_t)kBigPB : (uint64_t)kSmallPB;
      const uint32_t G = (uint32_t)std::min<uint64_t>(
          std::min<uint64_t>((h + pb0 - 1) / pb0, (uint64_t)P.grid_chunk), (uint64_t)P.grid_rounds);
      R.nwork = G;
      void* kargs[] = {&R};
      if (G >= 2 && cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_sc_plonk_rounds), dim3(G),
                                                dim3(16 * kSmallPB), kargs, kRoundsDyn, st) == cudaSuccess) {
        for (int j = 0; j < 8; j++) cur[j] = B.tab[j];
        *launches += 1;
        i = end;
        break;
      }
      cudaGetLastError();  // not co-resident here: the per-round kernels below
    }
    if (plonk && i > 0 && h <= P.chunk_pairs) {
      R.nwork = (uint32_t)std::min<uint64_t>((h + kSmallPB - 1) / kSmallPB, (uint64_t)P.grid_chunk);
      if (R.full) k_sc_plonk_chunk<16, kSmallPB, true><<<R.nwork, 16 * kSmallPB, 0, st>>>(R);
      else k_sc_plonk_chunk<16, kSmallPB, false><<<R.nwork, 16 * kSmallPB, 0, st>>>(R);
      for (int j = 0; j < 8; j++) cur[j] = B.tab[j];
      *launches += 1;
    } else if (plonk && i > 0 && h <= P.quad_pairs) {
      R.nwork = (uint32_t)std::min<uint64_t>((h + kQuadPB - 1) / kQuadPB, (uint64_t)P.grid_quad);
      if (R.full) k_sc_plonk_chunk<4, kQuadPB, true><<<R.nwork, 4 * kQuadPB, 0, st>>>(R);
      else k_sc_plonk_chunk<4, kQuadPB, false><<<R.nwork, 4 * kQuadPB, 0, st>>>(R);
      for (int j = 0; j < 8; j++) cur[j] = B.tab[j];
      *launches += 1;
    } else if (plonk) {
      R.nwork = (uint32_t)std::min<uint64_t>((h + 255) / 256, (uint64_t)P.grid_plonk);
      if (i == 0 && up) {
        const uint32_t nwc = (uint32_t)std::min<uint64_t>((up->hc + 255) / 256, (uint64_t)P.grid_plonk);
        R.nwork = nwc;
        R.nwork_total = nwc * (uint32_t)up->chunks;
        for (int q = 0; q < up->chunks; q++) {
          if (!upload_range(q)) return ZC_ERR_CUDA;
          R.k0 = (uint64_t)q * up->hc;
          R.k1 = R.k0 + up->hc;
          R.cta0 = (uint32_t)q * nwc;
          const uint32_t g = nwc + (q == 0 ? inv_cta : 0u);
          if (P.minb == 2) k_sc_plonk_round<true, 2><<<g, 256, 0, st>>>(R);
          else k_sc_plonk_round<true, 1><<<g, 256, 0, st>>>(R);
          *launches += 1;
        }
        *launches -= 1;  // counted once below
        R.k0 = R.k1 = 0;
        R.cta0 = R.nwork_total = 0;
        for (int j = 5; j < 8; j++) cur[j] = B.tab[j];
      } else if (i == 0) {
        if (P.minb == 2) k_sc_plonk_round<true, 2><<<R.nwork + inv_cta, 256, 0, st>>>(R);
        else k_sc_plonk_round<true, 1><<<R.nwork + inv_cta, 256, 0, st>>>(R);
        for (int j = 5; j < 8; j++) cur[j] = B.tab[j];
      } else {
        if (P.minb == 2) k_sc_plonk_round<false, 2><<<R.nwork, 256, 0, st>>>(R);
        else k_sc_plonk_round<false, 1><<<R.nwork, 256, 0, st>>>(R);
        for (int j = 0; j < 8; j++) cur[j] = B.tab[j];
      }
      *launches += 1;
    } else {
      if (i > 0 && h <= P.fuse_pairs) {
        // fold fused into the evaluation (rounds 2..)
        const int npr = R.full ? (int)d + 1 : (int)d;
        const int ppt = prod_ppt(P.ppt, npr, h);
        // at most two fold items per thread: the round is latency-bound
        const int G = (npr + ppt - 1) / ppt, spb = std::max(1, std::min(256 / G, 256 / c));
        R.spb = (uint32_t)spb;
        R.nwork = (uint32_t)std::min<uint64_t>((h + spb - 1) / spb, (uint64_t)P.grid_prod);
        const size_t dyn = sizeof(fr) * (size_t)c * 2 * spb;
        if (ppt == 1) k_sc_prod_fused<1><<<R.nwork, 256, dyn, st>>>(R);
        else k_sc_prod_fused<3><<<R.nwork, 256, dyn, st>>>(R);
        for (int j = 0; j < c; j++) cur[j] = B.tab[j];
        *launches += 1;
        if (i == 0 && ev) cudaEventRecord(ev[3], st);
        continue;
      }
      if (i > 0) {
        ScFoldArgs fa{};
        for (int j = 0; j < c; j++) {
          fa.src[j] = cur[j];
          fa.dst[j] = B.tab[j];
        }
        fa.h = 2 * h;
        fa.c = c;
        fa.round = (int)i;
        fa.st = B.st;
        const uint64_t tot = 2 * h * (uint64_t)c;
        k_sc_fold<<<(unsigned)std::min<uint64_t>((tot + 255) / 256, (uint64_t)P.grid_prod * 4), 256, 0,
                    st>>>(fa);
        for (int j = 0; j < c; j++) cur[j] = B.tab[j];
        for (int j = 0; j < c; j++) R.src[j] = cur[j];
        *launches += 1;
      }
      const int npr = R.full ? (int)d + 1 : (int)d;
      const int ppt = prod_ppt(P.ppt, npr, h);
      const uint64_t slots_per_blk = 256 / ((npr + ppt - 1) / ppt);
      R.spb = (uint32_t)slots_per_blk;
      R.nwork = (uint32_t)std::min<uint64_t>((h + slots_per_blk - 1) / slots_per_blk, (uint64_t)P.grid_prod);
      if (i == 0 && up) {
        const uint32_t nwc =
            (uint32_t)std::min<uint64_t>((up->hc + slots_per_blk - 1) / slots_per_blk, (uint64_t)P.grid_prod);
        R.nwork = nwc;
        R.nwork_total = nwc * (uint32_t)up->chunks;
        for (int q = 0; q < up->chunks; q++) {
          if (!upload_range(q)) return ZC_ERR_CUDA;
          R.k0 = (uint64_t)q * up->hc;
          R.k1 = R.k0 + up->hc;
          R.cta0 = (uint32_t)q * nwc;
          const uint32_t g = nwc + (q == 0 ? inv_cta : 0u);
          if (ppt == 1) k_sc_prod_round<1><<<g, 256, 0, st>>>(R);
          else k_sc_prod_round<3><<<g, 256, 0, st>>>(R);
          *launches += 1;
        }
        R.k0 = R.k1 = 0;
        R.cta0 = R.nwork_total = 0;
      } else {
        const uint32_t ctas = R.nwork + (i == 0 ? inv_cta : 0u);
        if (ppt == 1) k_sc_prod_round<1><<<ctas, 256, 0, st>>>(R);
        else k_sc_prod_round<3><<<ctas, 256, 0, st>>>(R);
        *launches += 1;
      }
    }
    if (i == 0 && ev) cudaEventRecord(ev[3], st);
  }
  if (i == 0 && ev) cudaEventRecord(ev[3], st);
  // the tail: remaining rounds, challenges and final values in one CTA
  R.round = (int)i;
  for (int j = 0; j < c; j++) {
    R.src[j] = cur[j];
    R.dst[j] = B.tab[j];
  }
  R.nwork = 1;
  if (plonk)
    k_sc_tail<true><<<1, kTailThreads, 0, st>>>(R);
  else
    k_sc_tail<false><<<1, 256, 0, st>>>(R);
  *launches += 1;
  return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

size_t sumcheck_scratch_bytes(const zc_ctx* ctx, const zc_params* p) {
  const ScPlan P = sc_plan(p, ctx->sm_count, ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_GRID),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_TAIL_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_SMALL_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_MINB),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_PROD_PPT),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_CHUNK_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_QUAD_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_PROD_FUSE));
  const uint64_t N = 1ull << p->n;
  const size_t psize = 16 + 32 * ((size_t)p->n * (p->d + 2) + P.c);
  ScPlan Pc = P;
  if (sc_upload_chunkable(p)) Pc.upload_chunks = kUploadChunks;  // host columns may come in ranges
  return align_up(sizeof(fr) * N, 256) * P.c + align_up(sizeof(fr) * sc_partials_count(Pc), 256) +
         align_up(sizeof(fr) * P.eq_total, 256) + align_up(sizeof(ScState), 256) + align_up(psize, 256) +
         align_up(32 * (size_t)P.c, 256) + 4096 + root_scratch_bytes(P.c, N);
}

zc_status sumcheck_prove(zc_ctx* ctx, const zc_params* p, const void* const* cols, int on_dev,
                         const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                         bool proof_on_dev, bool v2) {
  const uint32_t n = p->n, d = p->d;
  const ScPlan P = sc_plan(p, ctx->sm_count, ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_GRID),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_TAIL_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_SMALL_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_MINB),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_PROD_PPT),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_CHUNK_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_QUAD_LOG),
                           ctx->tuned(ZC_FORM_SUMCHECK, p->n, ZC_TUNE_SC_PROD_FUSE));
  const int c = P.c;
  const uint64_t N = 1ull << n;
  const size_t psize = 16 + 32 * ((size_t)n * (v2 ? d + 1 : d + 2) + c);
  // Host columns with their roots given: copied in pair ranges beside round 1.
  // The Plonk round kernel takes a pair's low eq factor from its thread
  // index, so a range start and the launch's thread count must be multiples
  // of the low table's length.
  const uint64_t hc = (N / 2) / kUploadChunks;
  bool chunked = !on_dev && roots && sc_upload_chunkable(p);
  if (chunked && p->gate == ZC_GATE_PLONK) {
    const uint64_t nwc = std::min<uint64_t>((hc + 255) / 256, (uint64_t)P.grid_plonk), m = 1ull << P.mlo[0];
    chunked = (nwc * 256) % m == 0 && hc % m == 0;
  }
  ScPlan Pm = P;
  if (chunked) Pm.upload_chunks = kUploadChunks;
  zc_status s = ensure_arena(ctx, sumcheck_scratch_bytes(ctx, p));
  if (s != ZC_OK) return s;
  Arena& ar = ctx->arena;
  ar.reset();
  ScBuffers B{};
  if (!sc_carve(ar, Pm, N, psize, B)) {
    ctx->err = "scratch arena too small";
    return ZC_ERR_OOM;
  }
  const fr* src[kMaxCols];
  ScUpload up{};
  if (on_dev) {
    for (int j = 0; j < c; j++) src[j] = reinterpret_cast<const fr*>(cols[j]);
  } else if (chunked) {
    s = ensure_upload_stream(ctx, kUploadChunks);
    if (s != ZC_OK) return s;
    up.cols = cols;
    up.chunks = kUploadChunks;
    up.hc = hc;
    up.stream = ctx->up_stream;
    up.fork = ctx->up_fork;
    up.ev = ctx->up_ev.data();
    for (int j = 0; j < c; j++) src[j] = B.tab[j];
  } else {
    for (int j = 0; j < c; j++) {
      ZC_CUDA_TRY(ctx, cudaMemcpyAsync(B.tab[j], cols[j], N * sizeof(fr), cudaMemcpyHostToDevice, st));
      src[j] = B.tab[j];
    }
  }
  ctx->launches = 0;
  ctx->nev = 6;
  ctx->dom_a = 2;
  ctx->dom_b = 3;
  // round-1 evaluation: per pair (d+1)(g+1)+1 mulmods, reads c*N*32 bytes
  const double g_mul = p->gate == ZC_GATE_PLONK ? 5.0 : (double)(d - 1);
  ctx->dom_mulmods = (double)(N / 2) * ((d + 1) * (g_mul + 1) + 1);
  ctx->dom_bytes = 32.0 * (double)c * (double)N;
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], st));
  if (roots) {
    std::memcpy(ctx->pinned, roots, 32 * (size_t)c);
    ZC_CUDA_TRY(ctx, cudaMemcpyAsync(B.roots, ctx->pinned, 32 * (size_t)c, cudaMemcpyHostToDevice, st));
  } else {
    s = launch_roots(ctx, src, c, N, B.roots, st);
    if (s != ZC_OK) return s;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1], st));
  uint32_t launches = 0;
  s = sc_enqueue(p, Pm, src, B, ctx->dconst, ctx->dtabs, ctx->hconst, ctx->skip_point, st, &launches,
                 ctx->ev, v2, persistent_allowed(ctx, st), chunked ? &up : nullptr);
  ctx->launches += launches;
  if (s != ZC_OK) {
    ctx->err = "kernel launch failed";
    return s;
  }
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[4], st));
  ZC_CUDA_TRY(ctx, cudaMemcpyAsync(proof, B.proof, psize,
                                   proof_on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev[5], st));
  if (!proof_on_dev || !on_dev) {
    ZC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (std::memcmp(proof, "ZCE!", 4) == 0) {
      ctx->err = "column value >= r";
      return ZC_ERR_ARG;
    }
    if (std::memcmp(proof, "ZCT!", 4) == 0) {
      ctx->err = "a bounded device wait gave up (persistent round kernel)";
      return ZC_ERR_TIMEOUT;
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
  unsigned long long ctx_id = 0;  // the CUDA context the addresses belong to
  void* scratch = nullptr;
  DevConst* dconst = nullptr;
  fr* dtabs = nullptr;
  DevConst hconst;
};
static StaticDev g_static_dev[kStaticMaxDevices];
static std::mutex g_static_mu;

// Unique id of the current CUDA context (0 if the driver cannot say).  A
// cudaDeviceReset followed by new work creates a new primary context in
// which the static arrays are fresh, so set-up must run again there.
static unsigned long long current_context_id() {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_cur = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {  // called under g_static_mu
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess || q1 != cudaDriverEntryPointSuccess)
      get_cur = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess || q2 != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    cudaGetLastError();
    looked = true;
  }
  void* cu = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&cu) == 0 && cu && get_id(cu, &id) == 0) return id;
  return 0;
}

// Set-up for the current device: look up the device addresses of the static
// arrays and copy the field constants into them.  Runs on the first call per
// device and context (synchronous copies), so that first call must not be
// inside a stream capture.
static zc_status static_setup(int dev, StaticDev** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticDev& S = g_static_dev[dev];
  // the symbol lookup makes the device's context current (creating it if
  // needed) and is cheap once the module is loaded
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_static_scratch) != cudaSuccess) {
    cudaGetLastError();
    return ZC_ERR_CUDA;
  }
  const unsigned long long id = current_context_id();
  if (S.ready && (id != S.ctx_id || scratch != S.scratch)) S.ready = false;  // a new context
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
    S.ctx_id = id;
    S.ready = true;
  }
  *out = &S;
  return ZC_OK;
}

// Usable bytes of the static scratch: all of it, or less when the
// environment variable ZC_STATIC_SCRATCH_BYTES asks for a smaller limit
// (tests use it to reach the size checks with small instances).
static size_t static_scratch_limit() {
  const char* e = std::getenv("ZC_STATIC_SCRATCH_BYTES");
  if (!e || !*e) return kStaticScratchBytes;
  const unsigned long long v = std::strtoull(e, nullptr, 10);
  return v < kStaticScratchBytes ? (size_t)v : kStaticScratchBytes;
}

static zc_status static_prove(const zc_params* p, const void* const* cols,
                              const uint8_t (*roots)[32], cudaStream_t st, uint8_t* proof,
                              StaticDev& S) {
  const uint32_t n = p->n, d = p->d;
  int SMs = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&SMs, cudaDevAttrMultiProcessorCount, dev);
  const ScPlan P = sc_plan(p, SMs);
  const int c = P.c;
  const uint64_t N = 1ull << n;
  const size_t psize = 16 + 32 * ((size_t)n * (d + 2) + c);
  // carve the static array; reject instances that do not fit
  Arena ar;
  ar.base = static_cast<char*>(S.scratch);
  ar.cap = static_scratch_limit();
  ScBuffers B{};
  if (!sc_carve(ar, P, N, psize, B) || (!roots && ar.used + root_scratch_bytes(c, N) > ar.cap))
    return ZC_ERR_UNSUPPORTED;  // instance larger than the static scratch
  B.proof = proof;              // kernels write the caller's device buffer directly
  const fr* src[kMaxCols];
  for (int j = 0; j < c; j++) src[j] = reinterpret_cast<const fr*>(cols[j]);
  if (roots) {
    if (cudaMemcpyAsync(B.roots, roots, 32 * (size_t)c, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return ZC_ERR_CUDA;
  } else {
    // the root kernels take their node scratch from the rest of the static array
    zc_ctx tmp;
    tmp.arena = ar;
    const zc_status rs = launch_roots(&tmp, src, c, N, B.roots, st);
    tmp.arena.base = nullptr;
    if (rs != ZC_OK) return rs;
  }
  uint32_t launches = 0;
  return sc_enqueue(p, P, src, B, S.dconst, S.dtabs, S.hconst, 0, st, &launches, nullptr);
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
