// zc_api.cu -- C ABI entry points, context set-up, host-side verifier.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>

#include "zc_internal.cuh"

namespace zc {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int gate_ncols(uint32_t gate, uint32_t d) {
  const uint32_t base = gate & 0xffu, m = gate >> 8;
  if (base == ZC_GATE_PLONK) return (m == 0 && d == 3) ? 8 : -1;
  if (base == ZC_GATE_PRODUCT) return (m == 0 && d >= 2 && d <= (uint32_t)kMaxDeg) ? (int)d + 1 : -1;
  if (base == ZC_GATE_SUM)
    return (m <= 0xffu && d >= 2 && d <= (uint32_t)kMaxDeg && d + m <= (uint32_t)kMaxCols) ? (int)(d + m) : -1;
  return -1;
}

static uint32_t default_log_blowup(uint32_t d) {
  uint32_t l = 0;
  while ((1u << l) < d) l++;
  return l;
}

bool ntt_domain(uint32_t n, uint32_t d, uint32_t w, NttDomain* D) {
  if (w >> 16) return false;
  const uint32_t sp1 = (w >> 8) & 0xffu;
  D->step = sp1 != 0;
  D->k = w & 0xffu;
  if (!D->step && D->k == 0) D->k = default_log_blowup(d);
  D->s = D->step ? sp1 - 1 : 0;
  if (D->step && (D->k == 0 || D->s >= D->k)) return false;
  if (n + D->k > 32) return false;
  D->N = 1ull << n;
  D->Mb = D->N << D->k;
  D->Ms = D->step ? D->N << D->s : 0;
  D->M = D->Mb + D->Ms;
  // |D| must hold the quotient's (d-1) N - d + 1 coefficients
  if (D->M + d < (uint64_t)(d - 1) * D->N + 1) return false;
  D->word = D->step ? (n + D->k) | ((n + D->s + 1) << 8) : n + D->k;
  return true;
}

zc_status check_params(zc_ctx* ctx, const zc_params* p, zc_form form) {
  if (!p) {
    if (ctx) ctx->err = "null params";
    return ZC_ERR_ARG;
  }
  if (gate_ncols(p->gate, p->d) < 0 || p->n < 1 || p->n > (uint32_t)kMaxN) {
    if (ctx) ctx->err = "unsupported gate / degree / n";
    return ZC_ERR_ARG;
  }
  if (form == ZC_FORM_NTT) {
    NttDomain D;
    if (!ntt_domain(p->n, p->d, p->log_blowup, &D) || p->n + D.k > (uint32_t)kMaxN + 2) {
      if (ctx) ctx->err = "domain word malformed, too small for the degree, or domain too large";
      return ZC_ERR_ARG;
    }
  } else if (form != ZC_FORM_SUMCHECK && form != ZC_FORM_SUMCHECK_EQ) {
    if (ctx) ctx->err = "unknown form";
    return ZC_ERR_ARG;
  }
  if (ctx && (p->n > ctx->max_n || p->d > ctx->max_d)) {
    ctx->err = "instance larger than the context's max_n / max_d";
    return ZC_ERR_UNSUPPORTED;
  }
  return ZC_OK;
}

zc_status ensure_arena(zc_ctx* ctx, size_t bytes) {
  if (ctx->arena.cap >= bytes) return ZC_OK;
  if (ctx->arena_borrowed) {
    ctx->err = "scratch block smaller than the proof needs";
    return ZC_ERR_OOM;
  }
  if (ctx->budget && bytes > ctx->budget) {
    ctx->err = "scratch need exceeds the memory budget";
    return ZC_ERR_OOM;
  }
  if (ctx->arena.base) {
    cudaDeviceSynchronize();
    cudaFree(ctx->arena.base);
    ctx->arena.base = nullptr;
    ctx->arena.cap = 0;
  }
  size_t want = align_up(bytes, 1 << 20);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string("cudaMalloc scratch: ") + cudaGetErrorString(e);
    return ZC_ERR_OOM;
  }
  ctx->arena.base = static_cast<char*>(p);
  ctx->arena.cap = want;
  ctx->arena.used = 0;
  return ZC_OK;
}

// ------------------------------------------------------------ host field --

fr h_from_u64(uint64_t x) {
  fr z = fr_zero();
  z.v[0] = (uint32_t)x;
  z.v[1] = (uint32_t)(x >> 32);
  return z;
}

fr h_canon_mul(const fr& a, const fr& b, const DevConst& C) {
  return fr_mul_g(fr_mul_g(a, b), C.r2);
}

static fr h_pow_limbs(const fr& a, const uint32_t e[8], const DevConst& C) {
  fr acc = h_from_u64(1);
  for (int i = 7; i >= 0; i--)
    for (int b = 31; b >= 0; b--) {
      acc = h_canon_mul(acc, acc, C);
      if ((e[i] >> b) & 1) acc = h_canon_mul(acc, a, C);
    }
  return acc;
}

fr h_pow(const fr& a, uint64_t e, const DevConst& C) {
  fr acc = h_from_u64(1), base = a;
  while (e) {
    if (e & 1) acc = h_canon_mul(acc, base, C);
    base = h_canon_mul(base, base, C);
    e >>= 1;
  }
  return acc;
}

fr h_root_of_unity(uint32_t logn, const DevConst& C) {
  // 7^((r-1) / 2^32) generates the 2^32-element subgroup; square down to 2^logn
  uint32_t sh[8];
  for (int i = 0; i < 8; i++) sh[i] = i < 7 ? p_limb(i + 1) : 0;
  fr w = h_pow_limbs(h_from_u64(7), sh, C);
  for (uint32_t i = logn; i < 32; i++) w = h_canon_mul(w, w, C);
  return w;
}

fr h_inv(const fr& a, const DevConst& C) {
  uint32_t e[8];  // r - 2 (r's low limb is 1, so the subtraction borrows)
  uint64_t br = 2;
  for (int i = 0; i < 8; i++) {
    uint64_t x = (uint64_t)p_limb(i) - br;
    e[i] = (uint32_t)x;
    br = (x >> 63) & 1;
  }
  return h_pow_limbs(a, e, C);
}

void h_to_bytes(const fr& a, uint8_t* out) {
  for (int i = 0; i < 8; i++)
    for (int b = 0; b < 4; b++) out[4 * i + b] = (uint8_t)(a.v[i] >> (8 * b));
}

bool h_from_bytes(const uint8_t* in, fr* out) {
  for (int i = 0; i < 8; i++)
    out->v[i] = (uint32_t)in[4 * i] | ((uint32_t)in[4 * i + 1] << 8) |
                ((uint32_t)in[4 * i + 2] << 16) | ((uint32_t)in[4 * i + 3] << 24);
  return fr_is_canonical(*out);
}

static fr h_signed(int64_t x) {  // canonical residue of a small signed integer
  if (x >= 0) return h_from_u64((uint64_t)x);
  return fr_sub_g(fr_zero(), h_from_u64((uint64_t)(-x)));
}

void transcript_init_words(uint32_t S[8], uint32_t form, uint32_t gate, uint32_t n, uint32_t d,
                           uint32_t logm) {
  // the eq-factored SumCheck has its own transcript version
  const char* tag = form == ZC_FORM_SUMCHECK_EQ ? "zerocheck-gb300/v2" : "zerocheck-gb300/v1";
  uint8_t msg[64];
  size_t tl = std::strlen(tag);
  std::memcpy(msg, tag, tl);
  uint32_t v[5] = {form, gate, n, d, logm};
  for (int i = 0; i < 5; i++)
    for (int b = 0; b < 4; b++) msg[tl + 4 * i + b] = (uint8_t)(v[i] >> (8 * b));
  uint8_t out[32];
  sha256_bytes(msg, tl + 20, out);
  for (int i = 0; i < 8; i++)
    S[i] = ((uint32_t)out[4 * i] << 24) | ((uint32_t)out[4 * i + 1] << 16) |
           ((uint32_t)out[4 * i + 2] << 8) | out[4 * i + 3];
}

static void build_constants(zc_ctx* ctx) {
  DevConst& C = ctx->hconst;
  std::memset(&C, 0, sizeof C);
  fr x = h_from_u64(1);
  for (int i = 1; i <= 512; i++) {
    x = fr_add_g(x, x);
    if (i == 256) C.one = x;
  }
  C.r2 = x;
  C.rpow[0] = h_from_u64(1);
  for (int k = 1; k < kMaxDeg + 2; k++) C.rpow[k] = h_canon_mul(C.rpow[k - 1], C.one, C);
  fr rinv = h_inv(C.one, C);
  C.rnegpow[0] = h_from_u64(1);
  for (int k = 1; k < kMaxDeg + 2; k++) C.rnegpow[k] = h_canon_mul(C.rnegpow[k - 1], rinv, C);
  auto lvl1 = [&](const fr& a) { return h_canon_mul(a, C.one, C); };
  for (int t = 0; t < kMaxPts + 2; t++) C.small[t] = lvl1(h_from_u64((uint64_t)t));
  // per-degree extrapolation and Lagrange tables
  std::vector<fr>& T = ctx->htabs;
  T.clear();
  for (int d = 0; d <= kMaxDeg; d++) {
    C.ext_base[d] = (uint32_t)T.size();
    if (d < 2) {
      C.lag_base[d] = (uint32_t)T.size();
      continue;
    }
    // pinf(t) = prod_{s<d} (t - s); lext(t)[s] = prod_{s' != s, s' < d} (t - s')/(s - s')
    for (int t = d; t <= d + 1; t++) {
      fr pr = h_from_u64(1);
      for (int s = 0; s < d; s++) pr = h_canon_mul(pr, h_signed(t - s), C);
      T.push_back(lvl1(pr));
    }
    for (int t = d; t <= d + 1; t++) {
      for (int s = 0; s < d; s++) {
        fr num = h_from_u64(1), den = h_from_u64(1);
        for (int q = 0; q < d; q++) {
          if (q == s) continue;
          num = h_canon_mul(num, h_signed(t - q), C);
          den = h_canon_mul(den, h_signed(s - q), C);
        }
        T.push_back(lvl1(h_canon_mul(num, h_inv(den, C), C)));
      }
    }
    C.lag_base[d] = (uint32_t)T.size();
    for (int s = 0; s <= d; s++) {
      fr den = h_from_u64(1);
      for (int q = 0; q <= d; q++)
        if (q != s) den = h_canon_mul(den, h_signed(s - q), C);
      T.push_back(lvl1(h_inv(den, C)));
    }
  }
}

// ------------------------------------------------------ host SHA helpers --

static void sha256_host_mem(const uint8_t* p, size_t len, uint32_t h[8]) {
  sha256_init(h);
  size_t nfull = len / 64;
  uint32_t w[16];
  for (size_t b = 0; b < nfull; b++) {
    for (int i = 0; i < 16; i++) {
      const uint8_t* q = p + 64 * b + 4 * i;
      w[i] = ((uint32_t)q[0] << 24) | ((uint32_t)q[1] << 16) | ((uint32_t)q[2] << 8) | q[3];
    }
    sha256_compress(h, w);
  }
  Sha256 s;
  s.init();
  for (int i = 0; i < 8; i++) s.h[i] = h[i];
  s.total = nfull * 64;
  s.update(p + nfull * 64, len - nfull * 64);
  uint8_t out[32];
  s.final(out);
  for (int i = 0; i < 8; i++)
    h[i] = ((uint32_t)out[4 * i] << 24) | ((uint32_t)out[4 * i + 1] << 16) |
           ((uint32_t)out[4 * i + 2] << 8) | out[4 * i + 3];
}

template <class F>
static void parallel_for(size_t n, F f) {
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < 4096 || nt == 1) {
    f(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  size_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; t++) {
    size_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back(f, lo, hi, t);
  }
  for (auto& x : th) x.join();
}

// root(v) on the host (same definition as the device kernels): leaves of
// 64 elements (the last may be shorter), node = SHA-256(l | r), the odd last
// node of a level moves up unchanged, root = SHA-256(le64(L) | top).
static bool host_root(const uint8_t* v, uint64_t L, uint8_t out[32]) {
  if (L == 0) return false;
  const uint64_t nl = (L + 63) / 64;
  std::vector<uint32_t> nodes(nl * 8);
  parallel_for(nl, [&](size_t lo, size_t hi, unsigned) {
    for (size_t t = lo; t < hi; t++) {
      const uint64_t cnt = std::min<uint64_t>(64, L - 64 * t);
      sha256_host_mem(v + t * 64 * 32, (uint32_t)(cnt * 32), &nodes[8 * t]);
    }
  });
  for (uint64_t cnt = nl; cnt > 1; cnt = (cnt + 1) / 2) {
    for (uint64_t i = 0; i < cnt / 2; i++) {
      uint32_t w[16], h[8];
      for (int k = 0; k < 16; k++) w[k] = nodes[16 * i + k];
      sha256_init(h);
      sha256_compress(h, w);
      for (int k = 0; k < 16; k++) w[k] = 0;
      w[0] = 0x80000000u;
      w[15] = 512;
      sha256_compress(h, w);
      for (int k = 0; k < 8; k++) nodes[8 * i + k] = h[k];
    }
    if (cnt & 1)
      for (int k = 0; k < 8; k++) nodes[8 * (cnt / 2) + k] = nodes[8 * (cnt - 1) + k];
  }
  uint8_t msg[40];
  for (int i = 0; i < 8; i++) msg[i] = (uint8_t)(L >> (8 * i));
  for (int i = 0; i < 8; i++) {
    msg[8 + 4 * i] = (uint8_t)(nodes[i] >> 24);
    msg[9 + 4 * i] = (uint8_t)(nodes[i] >> 16);
    msg[10 + 4 * i] = (uint8_t)(nodes[i] >> 8);
    msg[11 + 4 * i] = (uint8_t)nodes[i];
  }
  sha256_bytes(msg, 40, out);
  return true;
}

struct HostTranscript {
  uint8_t s[32];
  void init(uint32_t form, uint32_t gate, uint32_t n, uint32_t d, uint32_t logm) {
    uint32_t S[8];
    transcript_init_words(S, form, gate, n, d, logm);
    for (int i = 0; i < 8; i++) {
      s[4 * i] = (uint8_t)(S[i] >> 24);
      s[4 * i + 1] = (uint8_t)(S[i] >> 16);
      s[4 * i + 2] = (uint8_t)(S[i] >> 8);
      s[4 * i + 3] = (uint8_t)S[i];
    }
  }
  void absorb(const uint8_t* m, size_t len) {
    Sha256 h;
    h.init();
    h.update(s, 32);
    h.update(m, len);
    h.final(s);
  }
  fr squeeze() {  // canonical
    uint8_t m[33];
    std::memcpy(m, s, 32);
    m[32] = 0x43;
    sha256_bytes(m, 33, s);
    fr x;
    for (int i = 0; i < 8; i++)
      x.v[i] = (uint32_t)s[4 * i] | ((uint32_t)s[4 * i + 1] << 8) | ((uint32_t)s[4 * i + 2] << 16) |
               ((uint32_t)s[4 * i + 3] << 24);
    for (int k = 0; k < 2; k++)
      if (!fr_is_canonical(x)) {
        int64_t br = 0;
        for (int i = 0; i < 8; i++) {
          int64_t dd = (int64_t)x.v[i] - p_limb(i) + br;
          x.v[i] = (uint32_t)dd;
          br = dd >> 32;
        }
      }
    return x;
  }
};

// canonical gate evaluation
static fr host_gate(uint32_t gate, uint32_t d, const fr* x, const DevConst& C) {
  if (gate == ZC_GATE_PLONK) {
    fr s = h_canon_mul(x[0], x[5], C);
    s = fr_add_g(s, h_canon_mul(x[1], x[6], C));
    s = fr_add_g(s, h_canon_mul(h_canon_mul(x[2], x[5], C), x[6], C));
    s = fr_add_g(s, h_canon_mul(x[3], x[7], C));
    return fr_add_g(s, x[4]);
  }
  fr pr = x[0];
  for (uint32_t j = 1; j < d; j++) pr = h_canon_mul(pr, x[j], C);
  if (gate == ZC_GATE_PRODUCT) return fr_sub_g(pr, x[d]);
  for (uint32_t j = d; j < d + (gate >> 8); j++) pr = fr_add_g(pr, x[j]);  // sum gate
  return pr;
}

static fr host_lagrange(const fr* y, int m, const fr& x, const DevConst& C) {
  fr acc = fr_zero();
  for (int t = 0; t < m; t++) {
    fr num = h_from_u64(1), den = h_from_u64(1);
    for (int s = 0; s < m; s++) {
      if (s == t) continue;
      num = h_canon_mul(num, fr_sub_g(x, h_from_u64((uint64_t)s)), C);
      den = h_canon_mul(den, h_signed(t - s), C);
    }
    acc = fr_add_g(acc, h_canon_mul(y[t], h_canon_mul(num, h_inv(den, C), C), C));
  }
  return acc;
}

// SumCheck proofs: v1 rounds carry G_i(0..d+1) (check G(0) + G(1) = claim,
// claim <- G(alpha)); eq-factored v2 rounds carry H_i(0..d) with G_i =
// c_i l_i H_i (check c_i ((1 - r_i) H(0) + r_i H(1)) = claim, then
// c_{i+1} = c_i l_i(alpha), claim <- c_{i+1} H(alpha)).  Both end with
// claim = gate(v) eq(r, alpha) and v_j = MLE_j(alpha).
// Replay a SumCheck proof: the transcript (column roots given, or computed
// from host columns), every round's check and the final check of the claim
// against gate(v) eq(r, alpha).  Out: alpha (canonical), v (the final
// values), ok.  ZC_ERR_ARG if the proof is malformed.
static zc_status sumcheck_replay(const zc_params* p, const void* const* cols, const uint8_t (*roots)[32],
                                 const uint8_t* proof, size_t len, const DevConst& C, bool v2,
                                 std::vector<fr>& al, std::vector<fr>& v, bool& ok) {
  const uint32_t n = p->n, d = p->d, gate = p->gate;
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n;
  const uint32_t per = v2 ? d + 1 : d + 2;  // values per round
  size_t need = 16 + 32 * ((size_t)n * per + c);
  if (len != need || std::memcmp(proof, v2 ? "ZCS2" : "ZCS1", 4) != 0) return ZC_ERR_ARG;
  uint32_t hdr[3];
  for (int q = 0; q < 3; q++) std::memcpy(&hdr[q], proof + 4 + 4 * q, 4);
  if (hdr[0] != gate || hdr[1] != n || hdr[2] != d) return ZC_ERR_ARG;
  HostTranscript tr;
  tr.init(v2 ? ZC_FORM_SUMCHECK_EQ : ZC_FORM_SUMCHECK, gate, n, d, 0);
  for (int j = 0; j < c; j++) {
    uint8_t rt[32];
    if (roots) std::memcpy(rt, roots[j], 32);
    else if (!host_root(static_cast<const uint8_t*>(cols[j]), N, rt)) return ZC_ERR_ARG;
    tr.absorb(rt, 32);
  }
  std::vector<fr> r(n);
  al.assign(n, fr_zero());
  for (uint32_t i = 0; i < n; i++) r[i] = tr.squeeze();
  ok = true;
  fr claim = fr_zero(), ci = h_from_u64(1);
  const fr one1 = h_from_u64(1);
  const uint8_t* pp = proof + 16;
  std::vector<fr> G(per);
  for (uint32_t i = 0; i < n; i++) {
    for (uint32_t t = 0; t < per; t++)
      if (!h_from_bytes(pp + 32 * t, &G[t])) return ZC_ERR_ARG;
    if (v2) {
      const fr s = fr_add_g(h_canon_mul(fr_sub_g(one1, r[i]), G[0], C), h_canon_mul(r[i], G[1], C));
      if (!fr_equal(h_canon_mul(ci, s, C), claim)) ok = false;
    } else if (!fr_equal(fr_add_g(G[0], G[1]), claim)) {
      ok = false;
    }
    tr.absorb(pp, 32 * (size_t)per);
    pp += 32 * (size_t)per;
    al[i] = tr.squeeze();
    claim = host_lagrange(G.data(), (int)per, al[i], C);
    if (v2) {
      const fr li = fr_add_g(h_canon_mul(fr_sub_g(one1, r[i]), fr_sub_g(one1, al[i]), C),
                             h_canon_mul(r[i], al[i], C));
      ci = h_canon_mul(ci, li, C);
      claim = h_canon_mul(ci, claim, C);
    }
  }
  v.assign(c, fr_zero());
  for (int j = 0; j < c; j++)
    if (!h_from_bytes(pp + 32 * j, &v[j])) return ZC_ERR_ARG;
  fr eqra = h_from_u64(1);
  fr one = h_from_u64(1);
  for (uint32_t i = 0; i < n; i++) {
    fr e = fr_add_g(h_canon_mul(r[i], al[i], C),
                    h_canon_mul(fr_sub_g(one, r[i]), fr_sub_g(one, al[i]), C));
    eqra = h_canon_mul(eqra, e, C);
  }
  if (!fr_equal(claim, h_canon_mul(host_gate(gate, d, v.data(), C), eqra, C))) ok = false;
  return ZC_OK;
}

static zc_status verify_sumcheck(const zc_params* p, const void* const* cols,
                                 const uint8_t (*roots)[32], const uint8_t* proof, size_t len,
                                 int* accept, const DevConst& C, bool v2) {
  const uint32_t n = p->n, d = p->d, gate = p->gate;
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n;
  std::vector<fr> al, v;
  bool ok = true;
  zc_status rs = sumcheck_replay(p, cols, roots, proof, len, C, v2, al, v, ok);
  if (rs != ZC_OK) return rs;
  (void)gate;
  // v_j = sum_b col_j[b] eq_alpha(b): eq table at level 1, columns canonical
  std::vector<fr> E(1, C.one);
  E.reserve(N);
  for (uint32_t i = 0; i < n; i++) {
    fr ai = fr_mul_g(al[i], C.r2), bi = fr_sub_g(C.one, ai);
    std::vector<fr> E2(E.size() * 2);
    for (size_t k = 0; k < E.size(); k++) {
      E2[2 * k] = fr_mul_g(E[k], bi);
      E2[2 * k + 1] = fr_mul_g(E[k], ai);
    }
    E.swap(E2);
  }
  for (int j = 0; j < c && ok; j++) {
    const uint8_t* col = static_cast<const uint8_t*>(cols[j]);
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<fr> part(nt, fr_zero());
    std::vector<int> good(nt, 1);
    parallel_for(N, [&](size_t lo, size_t hi, unsigned t) {
      fr s = fr_zero();
      for (size_t k = lo; k < hi; k++) {
        fr x;
        if (!h_from_bytes(col + 32 * k, &x)) good[t] = 0;
        s = fr_add_g(s, fr_mul_g(x, E[k]));
      }
      part[t] = s;
    });
    fr tot = fr_zero();
    for (unsigned t = 0; t < nt; t++) {
      if (!good[t]) return ZC_ERR_ARG;
      tot = fr_add_g(tot, part[t]);
    }
    if (!fr_equal(tot, v[j])) ok = false;
  }
  *accept = ok ? 1 : 0;
  return ZC_OK;
}

static zc_status verify_ntt(const zc_params* p, const void* const* cols, const uint8_t (*roots)[32],
                            const uint8_t* proof, size_t len, const void* qv, int* accept,
                            const DevConst& C) {
  const uint32_t n = p->n, d = p->d, gate = p->gate;
  const int c = gate_ncols(gate, d);
  const uint64_t N = 1ull << n;
  size_t need = 20 + 32 + 32 * ((size_t)c + 1);
  if (len != need || std::memcmp(proof, "ZCN1", 4) != 0 || !qv) return ZC_ERR_ARG;
  uint32_t hdr[4];
  for (int q = 0; q < 4; q++) std::memcpy(&hdr[q], proof + 4 + 4 * q, 4);
  NttDomain D;
  if (!ntt_domain(n, d, p->log_blowup, &D)) return ZC_ERR_ARG;
  if (hdr[0] != gate || hdr[1] != n || hdr[2] != d || hdr[3] != D.word) return ZC_ERR_ARG;
  const uint32_t logm = D.word;
  const uint64_t M = D.M;
  const uint8_t* q = static_cast<const uint8_t*>(qv);
  bool ok = true;
  uint8_t qroot[32];
  host_root(q, M, qroot);
  if (std::memcmp(qroot, proof + 20, 32) != 0) ok = false;
  HostTranscript tr;
  tr.init(ZC_FORM_NTT, gate, n, d, logm);
  for (int j = 0; j < c; j++) {
    uint8_t rt[32];
    if (roots) std::memcpy(rt, roots[j], 32);
    else if (!host_root(static_cast<const uint8_t*>(cols[j]), N, rt)) return ZC_ERR_ARG;
    tr.absorb(rt, 32);
  }
  tr.absorb(proof + 20, 32);
  fr z, zn;
  const fr one = h_from_u64(1);
  do {
    z = tr.squeeze();
    zn = h_pow(z, N, C);
  } while (fr_equal(zn, one));
  // t = q(z) by Horner (level 1 z, canonical q -> canonical), degree bound
  const uint64_t qlen = (uint64_t)(d - 1) * N - d + 1;
  fr zm = fr_mul_g(z, C.r2), tq = fr_zero();
  for (uint64_t k = M; k-- > 0;) {
    fr qk;
    if (!h_from_bytes(q + 32 * k, &qk)) return ZC_ERR_ARG;
    if (k >= qlen && !fr_is_zero(qk)) ok = false;
    tq = fr_add_g(fr_mul_g(tq, zm), qk);
  }
  std::vector<fr> y(c);
  fr tclaim;
  for (int j = 0; j < c; j++)
    if (!h_from_bytes(proof + 52 + 32 * j, &y[j])) return ZC_ERR_ARG;
  if (!h_from_bytes(proof + 52 + 32 * c, &tclaim)) return ZC_ERR_ARG;
  if (!fr_equal(tq, tclaim)) ok = false;
  // barycentric g_j(z) = (z^N - 1)/N sum_i e_i w^i/(z - w^i)
  uint32_t e[8];
  for (int i = 0; i < 8; i++) e[i] = p_limb(i);
  // w_N = 7^((r-1)/2^32) squared (32-n) times
  uint32_t sh[8];
  for (int i = 0; i < 8; i++) sh[i] = (i < 7 ? e[i + 1] : 0);  // (r-1) >> 32 = limbs 1..7
  fr w = h_pow_limbs(h_from_u64(7), sh, C);
  for (uint32_t i = n; i < 32; i++) w = h_canon_mul(w, w, C);
  // level-1 copies for fast products
  fr wm = fr_mul_g(w, C.r2);
  std::vector<fr> wi(N), den(N);
  {
    // powers in parallel chunks
    parallel_for(N, [&](size_t lo, size_t hi, unsigned) {
      fr x = fr_mul_g(h_pow(w, lo, C), C.r2);
      for (size_t k = lo; k < hi; k++) {
        wi[k] = x;  // level 1
        x = fr_mul_g(x, wm);
      }
    });
  }
  parallel_for(N, [&](size_t lo, size_t hi, unsigned) {
    for (size_t k = lo; k < hi; k++) den[k] = fr_sub_g(zm, wi[k]);  // level 1
  });
  // batch inversion (level 1): prefix products
  {
    std::vector<fr> pre(N);
    fr acc = C.one;
    for (uint64_t k = 0; k < N; k++) {
      pre[k] = acc;
      acc = fr_mul_g(acc, den[k]);
    }
    // inverse of acc (level 1): canonical inverse then back to level 1 twice
    fr accc = fr_mul_g(acc, h_from_u64(1));
    fr inv = fr_mul_g(h_inv(accc, C), C.r2);
    for (uint64_t k = N; k-- > 0;) {
      fr dk = den[k];
      den[k] = fr_mul_g(inv, pre[k]);
      inv = fr_mul_g(inv, dk);
    }
  }
  fr zn1 = fr_sub_g(zn, one);
  fr scale = h_canon_mul(zn1, h_inv(h_from_u64(N), C), C);
  for (int j = 0; j < c && ok; j++) {
    const uint8_t* col = static_cast<const uint8_t*>(cols[j]);
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<fr> part(nt, fr_zero());
    std::vector<int> good(nt, 1);
    parallel_for(N, [&](size_t lo, size_t hi, unsigned t) {
      fr s = fr_zero();
      for (size_t k = lo; k < hi; k++) {
        fr x;
        if (!h_from_bytes(col + 32 * k, &x)) good[t] = 0;
        s = fr_add_g(s, fr_mul_g(x, fr_mul_g(wi[k], den[k])));  // canonical
      }
      part[t] = s;
    });
    fr tot = fr_zero();
    for (unsigned t = 0; t < nt; t++) {
      if (!good[t]) return ZC_ERR_ARG;
      tot = fr_add_g(tot, part[t]);
    }
    if (!fr_equal(h_canon_mul(tot, scale, C), y[j])) ok = false;
  }
  if (!fr_equal(host_gate(gate, d, y.data(), C), h_canon_mul(zn1, tq, C))) ok = false;
  *accept = ok ? 1 : 0;
  return ZC_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const DevConst& host_constants() {
  static DevConst C;
  static std::once_flag once;
  std::call_once(once, [] {
    zc_ctx tmp;
    build_constants(&tmp);
    C = tmp.hconst;
  });
  return C;
}

// Field constants and per-degree tables as plain host values (used by the
// static-scratch entry point, which has no context).
void static_constants(DevConst* C, std::vector<fr>* tabs) {
  zc_ctx tmp;
  build_constants(&tmp);
  *C = tmp.hconst;
  *tabs = tmp.htabs;
}

}  // namespace zc

using namespace zc;

extern "C" {

zc_status zc_setup(const zc_setup_opts* opts, zc_ctx** out) {
  if (!opts || !out) return ZC_ERR_ARG;
  *out = nullptr;
  if (opts->max_n < 1 || opts->max_n > (uint32_t)kMaxN) return ZC_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || opts->device < 0 || opts->device >= ndev) {
    cudaGetLastError();
    return ZC_ERR_CUDA;
  }
  zc_ctx* ctx = new zc_ctx();
  ctx->device = opts->device;
  ctx->max_n = opts->max_n;
  ctx->max_d = opts->max_d ? std::min<uint32_t>(opts->max_d, kMaxDeg) : 3;
  if (ctx->max_d < 3) ctx->max_d = 3;
  ctx->budget = opts->mem_budget_bytes;
  const char* sp = std::getenv("ZC_SUMCHECK_DERIVED_POINT");
  ctx->skip_point = (sp && sp[0] == '0') ? 1 : 0;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete ctx;
    return ZC_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
  build_constants(ctx);
  if (cudaMalloc(&ctx->dconst, sizeof(DevConst)) != cudaSuccess ||
      cudaMalloc(&ctx->dtabs, sizeof(fr) * std::max<size_t>(1, ctx->htabs.size())) != cudaSuccess ||
      cudaMallocHost(&ctx->pinned, 1 << 16) != cudaSuccess) {
    cudaGetLastError();
    zc_destroy(ctx);
    return ZC_ERR_OOM;
  }
  ctx->pinned_cap = 1 << 16;
  cudaMemcpy(ctx->dconst, &ctx->hconst, sizeof(DevConst), cudaMemcpyHostToDevice);
  cudaMemcpy(ctx->dtabs, ctx->htabs.data(), sizeof(fr) * ctx->htabs.size(), cudaMemcpyHostToDevice);
  for (int i = 0; i < 8; i++) cudaEventCreate(&ctx->ev[i]);
  if (cudaGetLastError() != cudaSuccess) {
    zc_destroy(ctx);
    return ZC_ERR_CUDA;
  }
  *out = ctx;
  return ZC_OK;
}

void zc_destroy(zc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  destroy_lanes(ctx);
  destroy_serve_pool(ctx);
  for (cudaEvent_t e : ctx->up_ev) cudaEventDestroy(e);
  if (ctx->up_fork) cudaEventDestroy(ctx->up_fork);
  if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
  if (ctx->arena.base) cudaFree(ctx->arena.base);
  for (auto& t : ctx->ntt_cache) {
    if (t.mem) cudaFree(t.mem);
    if (t.step_mem) cudaFree(t.step_mem);
  }
  if (ctx->dconst) cudaFree(ctx->dconst);
  if (ctx->dtabs) cudaFree(ctx->dtabs);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (int i = 0; i < 8; i++)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  delete ctx;
}

zc_status zc_proof_size(const zc_params* params, zc_form form, size_t* bytes) {
  if (!bytes) return ZC_ERR_ARG;
  zc_status s = check_params(nullptr, params, form);
  if (s != ZC_OK) return s;
  int c = gate_ncols(params->gate, params->d);
  if (form == ZC_FORM_SUMCHECK) *bytes = 16 + 32 * ((size_t)params->n * (params->d + 2) + c);
  else if (form == ZC_FORM_SUMCHECK_EQ) *bytes = 16 + 32 * ((size_t)params->n * (params->d + 1) + c);
  else *bytes = 20 + 32 + 32 * ((size_t)c + 1);
  return ZC_OK;
}

static zc_status prove_sumcheck_form(zc_ctx* ctx, zc_form form, const zc_params* params,
                                     const void* const* cols, int cols_on_device,
                                     const uint8_t (*col_roots)[32], void* cuda_stream, uint8_t* proof,
                                     size_t cap, size_t* len) {
  if (!ctx) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  zc_status s = check_params(ctx, params, form);
  if (s != ZC_OK) return s;
  if (!cols || !proof || !len) {
    ctx->err = "null argument";
    return ZC_ERR_ARG;
  }
  int c = gate_ncols(params->gate, params->d);
  for (int j = 0; j < c; j++)
    if (!cols[j]) {
      ctx->err = "null column pointer";
      return ZC_ERR_ARG;
    }
  size_t need;
  zc_proof_size(params, form, &need);
  *len = need;
  if (cap < need) {
    ctx->err = "proof buffer too small";
    return ZC_ERR_BUFFER_TOO_SMALL;
  }
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  bool pdev = is_device_ptr(proof);
  return sumcheck_prove(ctx, params, cols, cols_on_device, col_roots,
                        static_cast<cudaStream_t>(cuda_stream), proof, pdev, form == ZC_FORM_SUMCHECK_EQ);
}

zc_status zc_prove_sumcheck(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                            int cols_on_device, const uint8_t (*col_roots)[32], void* cuda_stream,
                            uint8_t* proof, size_t cap, size_t* len) {
  return prove_sumcheck_form(ctx, ZC_FORM_SUMCHECK, params, cols, cols_on_device, col_roots, cuda_stream,
                             proof, cap, len);
}

zc_status zc_prove_sumcheck_eq(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                               int cols_on_device, const uint8_t (*col_roots)[32], void* cuda_stream,
                               uint8_t* proof, size_t cap, size_t* len) {
  return prove_sumcheck_form(ctx, ZC_FORM_SUMCHECK_EQ, params, cols, cols_on_device, col_roots, cuda_stream,
                             proof, cap, len);
}

zc_status zc_prove_ntt(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                       int cols_on_device, const uint8_t (*col_roots)[32], void* cuda_stream,
                       uint8_t* proof, size_t cap, size_t* len, void* q_out, int q_on_device) {
  if (!ctx) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  zc_status s = check_params(ctx, params, ZC_FORM_NTT);
  if (s != ZC_OK) return s;
  if (!cols || !proof || !len) {
    ctx->err = "null argument";
    return ZC_ERR_ARG;
  }
  int c = gate_ncols(params->gate, params->d);
  for (int j = 0; j < c; j++)
    if (!cols[j]) {
      ctx->err = "null column pointer";
      return ZC_ERR_ARG;
    }
  size_t need;
  zc_proof_size(params, ZC_FORM_NTT, &need);
  *len = need;
  if (cap < need) {
    ctx->err = "proof buffer too small";
    return ZC_ERR_BUFFER_TOO_SMALL;
  }
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  bool pdev = is_device_ptr(proof);
  return ntt_prove(ctx, params, cols, cols_on_device, col_roots,
                   static_cast<cudaStream_t>(cuda_stream), proof, pdev, q_out, q_on_device);
}

zc_status zc_verify(const zc_params* params, zc_form form, const void* const* cols,
                    const uint8_t (*col_roots)[32], const uint8_t* proof, size_t len, const void* q,
                    int* accept) {
  if (!accept) return ZC_ERR_ARG;
  *accept = 0;
  zc_status s = check_params(nullptr, params, form);
  if (s != ZC_OK) return s;
  if (!cols || !proof) return ZC_ERR_ARG;
  int c = gate_ncols(params->gate, params->d);
  for (int j = 0; j < c; j++)
    if (!cols[j]) return ZC_ERR_ARG;
  const DevConst& C = host_constants();
  if (form == ZC_FORM_SUMCHECK || form == ZC_FORM_SUMCHECK_EQ)
    return verify_sumcheck(params, cols, col_roots, proof, len, accept, C, form == ZC_FORM_SUMCHECK_EQ);
  return verify_ntt(params, cols, col_roots, proof, len, q, accept, C);
}

zc_status zc_sumcheck_point(const zc_params* params, zc_form form, const uint8_t (*col_roots)[32],
                            const uint8_t* proof, size_t len, uint8_t (*alpha_out)[32],
                            uint8_t (*values_out)[32], int* rounds_ok) {
  if (!col_roots || !proof || !alpha_out || !values_out || !rounds_ok) return ZC_ERR_ARG;
  *rounds_ok = 0;
  if (form != ZC_FORM_SUMCHECK && form != ZC_FORM_SUMCHECK_EQ) return ZC_ERR_ARG;
  zc_status s = check_params(nullptr, params, form);
  if (s != ZC_OK) return s;
  std::vector<fr> al, v;
  bool ok = false;
  s = sumcheck_replay(params, nullptr, col_roots, proof, len, host_constants(), form == ZC_FORM_SUMCHECK_EQ,
                      al, v, ok);
  if (s != ZC_OK) return s;
  for (uint32_t i = 0; i < params->n; i++) h_to_bytes(al[i], alpha_out[i]);
  for (size_t j = 0; j < v.size(); j++) h_to_bytes(v[j], values_out[j]);
  *rounds_ok = ok ? 1 : 0;
  return ZC_OK;
}

zc_status zc_roots(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                   int cols_on_device, void* cuda_stream, uint8_t (*roots_out)[32]) {
  if (!ctx) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  zc_status s = check_params(ctx, params, ZC_FORM_SUMCHECK);
  if (s != ZC_OK) return s;
  if (!cols || !roots_out) return ZC_ERR_ARG;
  int c = gate_ncols(params->gate, params->d);
  uint64_t N = 1ull << params->n;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  size_t need = root_scratch_bytes(c, N) + 32 * (size_t)c + 1024;
  if (!cols_on_device) need += align_up(N * 32, 256) * c;
  s = ensure_arena(ctx, need);
  if (s != ZC_OK) return s;
  ctx->arena.reset();
  const fr* dcols[kMaxCols];
  for (int j = 0; j < c; j++) {
    if (cols_on_device) {
      dcols[j] = static_cast<const fr*>(cols[j]);
    } else {
      fr* t = ctx->arena.take<fr>(N);
      ZC_CUDA_TRY(ctx, cudaMemcpyAsync(t, cols[j], N * 32, cudaMemcpyHostToDevice, st));
      dcols[j] = t;
    }
  }
  uint8_t* dr = ctx->arena.take<uint8_t>(32 * (size_t)c);
  s = launch_roots(ctx, dcols, c, N, dr, st);
  if (s != ZC_OK) return s;
  ZC_CUDA_TRY(ctx, cudaMemcpyAsync(roots_out, dr, 32 * (size_t)c, cudaMemcpyDeviceToHost, st));
  ZC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return ZC_OK;
}

zc_status zc_stats(zc_ctx* ctx, double* phase_ms, uint32_t cap) {
  if (!ctx || !phase_ms) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  double out[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i + 1 < ctx->nev && i < 6; i++) {
    float ms = 0;
    if (cudaEventSynchronize(ctx->ev[i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0;
    }
    out[i] = ms;
  }
  {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ctx->ev[ctx->dom_a], ctx->ev[ctx->dom_b]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0;
    }
    out[6] = ms;
  }
  out[7] = ctx->dom_mulmods;
  out[8] = ctx->dom_bytes;
  out[9] = ctx->launches;
  for (uint32_t i = 0; i < cap && i < 10; i++) phase_ms[i] = out[i];
  return ZC_OK;
}

static bool tune_value_ok(zc_tune_key key, int32_t v) {
  if (v == 0) return true;
  switch (key) {
    case ZC_TUNE_SC_GRID: return v >= 1 && v <= 4096;
    case ZC_TUNE_SC_TAIL_LOG: return v >= 1 && v <= 24;
    case ZC_TUNE_NTT_TILE_LOG: return v >= 10 && v <= 12;
    case ZC_TUNE_NTT_MINB: return v == 1 || v == 2;
    case ZC_TUNE_SC_SMALL_LOG: return v >= 1 && v <= 24;
    case ZC_TUNE_SC_MINB: return v == 1 || v == 2;
    case ZC_TUNE_SC_PROD_PPT: return v == 1 || v == 3;
    case ZC_TUNE_SC_CHUNK_LOG: return v >= 1 && v <= 24;
    case ZC_TUNE_BATCH_LANES: return v >= 1 && v <= 64;
    case ZC_TUNE_SC_QUAD_LOG: return v >= 1 && v <= 24;
    case ZC_TUNE_SC_PROD_FUSE: return v >= 1 && v <= 24;
    case ZC_TUNE_NTT_TWO_LOG: return v >= 2 && v <= 24;
  }
  return false;
}

static bool tune_form_ok(zc_form form, zc_tune_key key) {
  if (key == ZC_TUNE_BATCH_LANES) return form == ZC_FORM_SUMCHECK || form == ZC_FORM_NTT;
  if (form == ZC_FORM_SUMCHECK)
    return key == ZC_TUNE_SC_GRID || key == ZC_TUNE_SC_TAIL_LOG || key == ZC_TUNE_SC_SMALL_LOG ||
           key == ZC_TUNE_SC_MINB || key == ZC_TUNE_SC_PROD_PPT || key == ZC_TUNE_SC_CHUNK_LOG ||
           key == ZC_TUNE_SC_QUAD_LOG || key == ZC_TUNE_SC_PROD_FUSE;
  if (form == ZC_FORM_NTT)
    return key == ZC_TUNE_NTT_TILE_LOG || key == ZC_TUNE_NTT_MINB || key == ZC_TUNE_NTT_TWO_LOG;
  return false;
}

zc_status zc_tune_set(zc_ctx* ctx, zc_form form, uint32_t n, zc_tune_key key, int32_t value) {
  if (!ctx || n > (uint32_t)kMaxN || !tune_form_ok(form, key) || !tune_value_ok(key, value))
    return ZC_ERR_ARG;
  if (key == ZC_TUNE_BATCH_LANES && n != 0) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (key == ZC_TUNE_BATCH_LANES) {  // one value for the context, kept under the SumCheck form
    ctx->tune[0][0][(int)key - 1] = value;
    return ZC_OK;
  }
  ctx->tune[(int)form - 1][n][(int)key - 1] = value;
  return ZC_OK;
}

zc_status zc_tune_get(zc_ctx* ctx, zc_form form, uint32_t n, zc_tune_key key, int32_t* value) {
  if (!ctx || !value || n > (uint32_t)kMaxN || !tune_form_ok(form, key)) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  *value = key == ZC_TUNE_BATCH_LANES ? ctx->tuned(ZC_FORM_SUMCHECK, 0, key) : ctx->tuned(form, n, key);
  return ZC_OK;
}

const char* zc_last_error(zc_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

}  // extern "C"
