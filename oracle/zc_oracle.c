/*
 * zc_oracle.c -- CPU oracle for the ZeroCheck prover (both forms).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the GPU
 * path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant or table with the CUDA library: every constant below is derived
 * here at start-up from the modulus alone.
 *
 * Paper: "When Proofs Meet Hardware: Comparing NTT and SumCheck in
 * Zero-Knowledge Systems".  Each routine cites the passage it follows:
 *   - Fig. side-by-side-zc (left)  : univariate (NTT) ZeroCheck
 *   - Fig. side-by-side-zc (right) : multilinear (SumCheck) ZeroCheck
 *   - Sec. 3.2 (Univariate ZeroCheck): z_H = x^N - 1, y = z_H(r) t, deg q
 *   - Sec. 3.3 (Multilinear ZeroCheck): MLE, eq, Eq. (multilinear_zc_sc)
 *   - Sec. 3.4: per-round check G_i(0) + G_i(1) = G_{i-1}(alpha_{i-1})
 * Conventions the paper leaves open (variable order, transcript bytes,
 * commitment stand-in, round-polynomial representation) are the readings
 * listed in the project's design notes; they are restated where used.
 *
 * Arithmetic: BLS12-381 scalar field r, 4 x 64-bit limbs, Montgomery form
 * (CIOS, Koc-Acar-Kaliski 1996) with unsigned __int128.  SHA-256 follows
 * FIPS 180-4.  Loops over independent elements carry an OpenMP pragma; the
 * arithmetic order inside each element is the textbook one.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef struct { uint64_t w[4]; } fe;          /* Montgomery form */

/* r = 0x73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001 */
static const uint64_t P[4] = {0xffffffff00000001ULL, 0x53bda402fffe5bfeULL,
                              0x3339d80809a1d805ULL, 0x73eda753299d7d48ULL};
static uint64_t PINV;      /* -r^{-1} mod 2^64 */
static fe R1;              /* 2^256 mod r  (Montgomery 1) */
static fe R2;              /* 2^512 mod r */
static int g_init = 0;

/* ------------------------------------------------------------ field ---- */

static int geq_p(const uint64_t t[4]) {
    for (int i = 3; i >= 0; i--) {
        if (t[i] > P[i]) return 1;
        if (t[i] < P[i]) return 0;
    }
    return 1;
}

static void sub_p(uint64_t t[4]) {
    uint64_t borrow = 0;
    for (int i = 0; i < 4; i++) {
        u128 d = (u128)t[i] - P[i] - borrow;
        t[i] = (uint64_t)d;
        borrow = (uint64_t)(d >> 64) ? 1 : 0;
    }
}

static fe f_add(fe a, fe b) {
    fe t; uint64_t c = 0;
    for (int i = 0; i < 4; i++) {
        u128 s = (u128)a.w[i] + b.w[i] + c;
        t.w[i] = (uint64_t)s; c = (uint64_t)(s >> 64);
    }
    if (c || geq_p(t.w)) sub_p(t.w);
    return t;
}

static fe f_sub(fe a, fe b) {
    fe t; uint64_t borrow = 0;
    for (int i = 0; i < 4; i++) {
        u128 d = (u128)a.w[i] - b.w[i] - borrow;
        t.w[i] = (uint64_t)d; borrow = (uint64_t)(d >> 64) ? 1 : 0;
    }
    if (borrow) {
        uint64_t c = 0;
        for (int i = 0; i < 4; i++) {
            u128 s = (u128)t.w[i] + P[i] + c;
            t.w[i] = (uint64_t)s; c = (uint64_t)(s >> 64);
        }
    }
    return t;
}

/* CIOS Montgomery product a*b*2^-256 mod r. */
static fe f_mul(fe a, fe b) {
    uint64_t t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        uint64_t C = 0;
        for (int j = 0; j < 4; j++) {
            u128 s = (u128)a.w[j] * b.w[i] + t[j] + C;
            t[j] = (uint64_t)s; C = (uint64_t)(s >> 64);
        }
        u128 s = (u128)t[4] + C;
        t[4] = (uint64_t)s; t[5] = (uint64_t)(s >> 64);
        uint64_t m = t[0] * PINV;
        s = (u128)m * P[0] + t[0];
        C = (uint64_t)(s >> 64);
        for (int j = 1; j < 4; j++) {
            s = (u128)m * P[j] + t[j] + C;
            t[j - 1] = (uint64_t)s; C = (uint64_t)(s >> 64);
        }
        s = (u128)t[4] + C;
        t[3] = (uint64_t)s;
        t[4] = t[5] + (uint64_t)(s >> 64);
    }
    fe r; memcpy(r.w, t, 32);
    if (t[4] || geq_p(r.w)) sub_p(r.w);
    return r;
}

static fe f_zero(void) { fe z; memset(&z, 0, sizeof z); return z; }
static fe f_one(void) { return R1; }
static int f_eq(fe a, fe b) { return memcmp(a.w, b.w, 32) == 0; }
static int f_is_zero(fe a) { return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) == 0; }
static fe f_neg(fe a) { return f_sub(f_zero(), a); }

static fe f_from_u64(uint64_t x) {
    fe t = f_zero(); t.w[0] = x;         /* x < r */
    return f_mul(t, R2);
}

/* canonical little-endian 32 bytes -> Montgomery; returns 0 if >= r */
static int f_from_bytes(const uint8_t *b, fe *out) {
    fe t;
    for (int i = 0; i < 4; i++) {
        uint64_t v = 0;
        for (int k = 7; k >= 0; k--) v = (v << 8) | b[8 * i + k];
        t.w[i] = v;
    }
    if (geq_p(t.w)) return 0;
    *out = f_mul(t, R2);
    return 1;
}

static void f_to_bytes(fe a, uint8_t *b) {
    fe one = f_zero(); one.w[0] = 1;
    fe c = f_mul(a, one);                 /* leave Montgomery form */
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 8; k++) b[8 * i + k] = (uint8_t)(c.w[i] >> (8 * k));
}

/* x^e, e given as 4 little-endian 64-bit words (square and multiply) */
static fe f_pow(fe x, const uint64_t e[4]) {
    fe acc = f_one();
    for (int i = 3; i >= 0; i--)
        for (int b = 63; b >= 0; b--) {
            acc = f_mul(acc, acc);
            if ((e[i] >> b) & 1) acc = f_mul(acc, x);
        }
    return acc;
}

static fe f_pow_u64(fe x, uint64_t e) {
    uint64_t ee[4] = {e, 0, 0, 0};
    return f_pow(x, ee);
}

/* Fermat inverse x^(r-2); x must be nonzero */
static fe f_inv(fe x) {
    uint64_t e[4]; memcpy(e, P, 32);
    e[0] -= 2;                           /* r - 2 (no borrow: low word ends in 1) */
    return f_pow(x, e);
}

/* Montgomery's batch inversion of n nonzero elements, in place. */
static int f_batch_inv(fe *v, size_t n) {
    if (n == 0) return 1;
    fe *pre = (fe *)malloc(n * sizeof(fe));
    if (!pre) return 0;
    fe acc = f_one();
    for (size_t i = 0; i < n; i++) { pre[i] = acc; acc = f_mul(acc, v[i]); }
    fe inv = f_inv(acc);
    for (size_t i = n; i-- > 0;) {
        fe vi = v[i];
        v[i] = f_mul(inv, pre[i]);
        inv = f_mul(inv, vi);
    }
    free(pre);
    return 1;
}

static void field_init(void) {
    if (g_init) return;
    /* -r^{-1} mod 2^64 by Newton iteration on the low word */
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - P[0] * inv;
    PINV = (uint64_t)0 - inv;
    /* 2^256 mod r and 2^512 mod r by repeated doubling of 1 */
    fe x = f_zero(); x.w[0] = 1;
    for (int i = 0; i < 512; i++) {
        x = f_add(x, x);               /* f_add works on any residues < r */
        if (i == 255) R1 = x;
    }
    R2 = x;
    g_init = 1;
}

/* generator of the 2^32 subgroup: 7^((r-1)/2^32); 2^k-th root by squaring */
static fe root_of_unity(unsigned logn) {
    uint64_t e[4];                        /* (r-1) >> 32 */
    e[0] = (P[0] >> 32) | (P[1] << 32);
    e[1] = (P[1] >> 32) | (P[2] << 32);
    e[2] = (P[2] >> 32) | (P[3] << 32);
    e[3] = (P[3] >> 32);
    fe w = f_pow(f_from_u64(7), e);
    for (unsigned i = logn; i < 32; i++) w = f_mul(w, w);
    return w;
}

/* out[k] = base^k for k < count (each thread starts its chunk with a pow) */
static void powers(fe base, size_t count, fe *out) {
    #pragma omp parallel
    {
        size_t nt = 1, id = 0;
#ifdef _OPENMP
        nt = (size_t)omp_get_num_threads(); id = (size_t)omp_get_thread_num();
#endif
        size_t chunk = (count + nt - 1) / nt, lo = id * chunk;
        size_t hi = lo + chunk < count ? lo + chunk : count;
        if (lo < hi) {
            fe x = f_pow_u64(base, (uint64_t)lo);
            for (size_t k = lo; k < hi; k++) { out[k] = x; x = f_mul(x, base); }
        }
    }
}

/* ------------------------------------------------------------ SHA-256 -- */
/* FIPS 180-4, section 6.2 */

typedef struct { uint32_t h[8]; uint8_t buf[64]; size_t nbuf; uint64_t total; } sha_ctx;

static const uint32_t SHA_K[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};

static uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

static void sha_block(uint32_t h[8], const uint8_t *p) {
    uint32_t W[64];
    for (int t = 0; t < 16; t++)
        W[t] = ((uint32_t)p[4 * t] << 24) | ((uint32_t)p[4 * t + 1] << 16) |
               ((uint32_t)p[4 * t + 2] << 8) | (uint32_t)p[4 * t + 3];
    for (int t = 16; t < 64; t++) {
        uint32_t s0 = rotr(W[t - 15], 7) ^ rotr(W[t - 15], 18) ^ (W[t - 15] >> 3);
        uint32_t s1 = rotr(W[t - 2], 17) ^ rotr(W[t - 2], 19) ^ (W[t - 2] >> 10);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
    for (int t = 0; t < 64; t++) {
        uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t T1 = hh + S1 + ch + SHA_K[t] + W[t];
        uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
        uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t T2 = S0 + mj;
        hh = g; g = f; f = e; e = d + T1; d = c; c = b; b = a; a = T1 + T2;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

static void sha_init(sha_ctx *s) {
    static const uint32_t H0[8] = {0x6a09e667, 0xbb67ae85, 0x3c6ef372, 0xa54ff53a,
                                   0x510e527f, 0x9b05688c, 0x1f83d9ab, 0x5be0cd19};
    memcpy(s->h, H0, sizeof H0);
    s->nbuf = 0; s->total = 0;
}

static void sha_update(sha_ctx *s, const uint8_t *m, size_t len) {
    s->total += len;
    while (len > 0) {
        size_t take = 64 - s->nbuf;
        if (take > len) take = len;
        memcpy(s->buf + s->nbuf, m, take);
        s->nbuf += take; m += take; len -= take;
        if (s->nbuf == 64) { sha_block(s->h, s->buf); s->nbuf = 0; }
    }
}

static void sha_final(sha_ctx *s, uint8_t out[32]) {
    uint64_t bits = s->total * 8;
    uint8_t pad = 0x80;
    sha_update(s, &pad, 1);
    uint8_t z = 0;
    while (s->nbuf != 56) sha_update(s, &z, 1);
    uint8_t L[8];
    for (int i = 0; i < 8; i++) L[i] = (uint8_t)(bits >> (56 - 8 * i));
    sha_update(s, L, 8);
    for (int i = 0; i < 8; i++) {
        out[4 * i] = (uint8_t)(s->h[i] >> 24); out[4 * i + 1] = (uint8_t)(s->h[i] >> 16);
        out[4 * i + 2] = (uint8_t)(s->h[i] >> 8); out[4 * i + 3] = (uint8_t)s->h[i];
    }
}

static void sha256(const uint8_t *m, size_t len, uint8_t out[32]) {
    sha_ctx s; sha_init(&s); sha_update(&s, m, len); sha_final(&s, out);
}

/* ------------------------------------------------ commitment stand-in -- */
/* The paper's commitments [g], [q] (Fig. side-by-side-zc, "Commit") are
 * stood in by a binary SHA-256 Merkle root over chunks of 64 canonical
 * elements: leaf t = SHA-256(enc(v[64t]) || ... || enc(v[min(64t+63, L-1)]))
 * (the last leaf may be shorter), node = SHA-256(l || r), and at a level
 * with an odd count the last node moves up unchanged; root =
 * SHA-256(le64(L) || top).  For a power-of-two L every level is even. */
#define LEAF_ELEMS 64

static int root_of(const uint8_t *canon, size_t L, uint8_t out[32]) {
    if (L == 0) return 0;
    size_t nl = (L + LEAF_ELEMS - 1) / LEAF_ELEMS;
    uint8_t *nodes = (uint8_t *)malloc(nl * 32);
    if (!nodes) return 0;
    #pragma omp parallel for schedule(static)
    for (long t = 0; t < (long)nl; t++) {
        size_t first = (size_t)t * LEAF_ELEMS;
        size_t cnt = L - first < LEAF_ELEMS ? L - first : LEAF_ELEMS;
        sha256(canon + first * 32, cnt * 32, nodes + (size_t)t * 32);
    }
    /* each level is written to a fresh buffer: a parallel in-place update
     * would let node i be overwritten while node i/2 is still reading it */
    uint8_t *next = (uint8_t *)malloc((nl / 2 + 1) * 32);
    if (!next) { free(nodes); return 0; }
    for (size_t cnt = nl; cnt > 1; cnt = (cnt + 1) / 2) {
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)(cnt / 2); i++)
            sha256(nodes + (size_t)(2 * i) * 32, 64, next + (size_t)i * 32);
        if (cnt & 1) memcpy(next + (cnt / 2) * 32, nodes + (cnt - 1) * 32, 32);
        memcpy(nodes, next, ((cnt + 1) / 2) * 32);
    }
    free(next);
    uint8_t msg[40];
    for (int i = 0; i < 8; i++) msg[i] = (uint8_t)((uint64_t)L >> (8 * i));
    memcpy(msg + 8, nodes, 32);
    sha256(msg, 40, out);
    free(nodes);
    return 1;
}

/* --------------------------------------------------------- transcript -- */
/* Fiat-Shamir: "alpha_i <- Hash(G_i)", "r <- Hash([g])" (Fig.
 * side-by-side-zc).  State S; absorb(m): S = H(S||m); squeeze: S =
 * H(S||0x43), output int_le(S) mod r. */
typedef struct { uint8_t s[32]; } transcript;

static void le32(uint8_t *b, uint32_t v) { for (int i = 0; i < 4; i++) b[i] = (uint8_t)(v >> (8 * i)); }

static void tr_init_tag(transcript *t, const char *tag, uint32_t form, uint32_t gate, uint32_t n,
                        uint32_t d, uint32_t logm) {
    uint8_t msg[64]; size_t tl = strlen(tag);
    memcpy(msg, tag, tl);
    le32(msg + tl, form); le32(msg + tl + 4, gate); le32(msg + tl + 8, n);
    le32(msg + tl + 12, d); le32(msg + tl + 16, logm);
    sha256(msg, tl + 20, t->s);
}

static void tr_init(transcript *t, uint32_t form, uint32_t gate, uint32_t n, uint32_t d, uint32_t logm) {
    tr_init_tag(t, "zerocheck-gb300/v1", form, gate, n, d, logm);
}

static void tr_absorb(transcript *t, const uint8_t *m, size_t len) {
    sha_ctx s; sha_init(&s); sha_update(&s, t->s, 32); sha_update(&s, m, len); sha_final(&s, t->s);
}

static fe tr_squeeze(transcript *t) {
    uint8_t msg[33]; memcpy(msg, t->s, 32); msg[32] = 0x43;
    sha256(msg, 33, t->s);
    fe x;
    for (int i = 0; i < 4; i++) {
        uint64_t v = 0;
        for (int k = 7; k >= 0; k--) v = (v << 8) | t->s[8 * i + k];
        x.w[i] = v;
    }
    while (geq_p(x.w)) sub_p(x.w);       /* at most twice: 2^256 < 3r */
    return f_mul(x, R2);
}

/* ------------------------------------------------------------- gates --- */
/* Plonk gate (columns qL,qR,qM,qO,qC,a,b,c):  qL a + qR b + qM a b + qO c + qC
 * Product gate (columns q,w1..w_{d-1},o):     q w1 ... w_{d-1} - o
 * Sum gate (columns g_1..g_{d+m}):            g_1 ... g_d + g_{d+1} + ... + g_{d+m}
 * The sum gate is the paper's workload family (Table poly_examples: g1 g2,
 * g1 g2 + g3, ..., g1 g2 g3 g4): one product of d columns plus m single
 * columns.  Its gate word carries m in bits 8..15 (GATE_SUM | m << 8). */
enum { GATE_PLONK = 1, GATE_PRODUCT = 2, GATE_SUM = 3 };

static int gate_cols(uint32_t gate, uint32_t d) {
    const uint32_t base = gate & 0xff, m = gate >> 8;
    if (base == GATE_PLONK) return (m == 0 && d == 3) ? 8 : -1;
    if (base == GATE_PRODUCT) return (m == 0 && d >= 2 && d <= 64) ? (int)d + 1 : -1;
    if (base == GATE_SUM) return (m <= 63 && d >= 2 && d <= 64 && d + m <= 65) ? (int)(d + m) : -1;
    return -1;
}

static fe gate_eval(uint32_t gate, uint32_t d, const fe *x) {
    if (gate == GATE_PLONK) {
        fe qL = x[0], qR = x[1], qM = x[2], qO = x[3], qC = x[4], a = x[5], b = x[6], c = x[7];
        fe s = f_mul(qL, a);
        s = f_add(s, f_mul(qR, b));
        s = f_add(s, f_mul(f_mul(qM, a), b));
        s = f_add(s, f_mul(qO, c));
        return f_add(s, qC);
    }
    fe p = x[0];
    for (uint32_t i = 1; i < d; i++) p = f_mul(p, x[i]);
    if ((gate & 0xff) == GATE_PRODUCT) return f_sub(p, x[d]);
    for (uint32_t i = d; i < d + (gate >> 8); i++) p = f_add(p, x[i]);
    return p;
}

/* ------------------------------------------------------------ NTT ------ */
/* Textbook iterative radix-2 transform A[i] = sum_k a[k] w^(ik) for a
 * primitive 2^logn-th root w: bit-reversal permutation, then log n stages
 * of butterflies (Sec. 2, "NTT"). */
static void ntt_inplace(fe *a, unsigned logn, fe w) {
    size_t N = (size_t)1 << logn;
    if (N == 1) return;
    for (size_t i = 0, j = 0; i < N; i++) {
        if (i < j) { fe t = a[i]; a[i] = a[j]; a[j] = t; }
        size_t bit = N >> 1;
        while (j & bit) { j ^= bit; bit >>= 1; }
        j |= bit;
    }
    fe *pw = (fe *)malloc((N / 2) * sizeof(fe));          /* w^k, k < N/2 */
    powers(w, N / 2, pw);
    for (size_t len = 2; len <= N; len <<= 1) {
        size_t half = len / 2, step = N / len;
        #pragma omp parallel for schedule(static)
        for (long bfly = 0; bfly < (long)(N / 2); bfly++) {
            size_t blk = (size_t)bfly / half, j = (size_t)bfly % half;
            size_t i0 = blk * len + j, i1 = i0 + half;
            fe u = a[i0], v = f_mul(a[i1], pw[j * step]);
            a[i0] = f_add(u, v);
            a[i1] = f_sub(u, v);
        }
    }
    free(pw);
}

/* ------------------------------------------------------------- helpers -- */

static unsigned ilog2(uint64_t x) { unsigned l = 0; while ((1ULL << l) < x) l++; return l; }

static int load_cols(const uint8_t *const *cols, int c, size_t N, fe **T) {
    for (int j = 0; j < c; j++) {
        T[j] = (fe *)malloc(N * sizeof(fe));
        if (!T[j]) return 0;
    }
    int ok = 1;
    for (int j = 0; j < c; j++) {
        #pragma omp parallel for schedule(static) reduction(&:ok)
        for (long k = 0; k < (long)N; k++)
            ok &= f_from_bytes(cols[j] + (size_t)k * 32, &T[j][k]);
    }
    return ok;
}

static void free_cols(fe **T, int c) { for (int j = 0; j < c; j++) free(T[j]); }

static int col_roots(const uint8_t *const *cols, int c, size_t N, const uint8_t *given, uint8_t *roots) {
    for (int j = 0; j < c; j++) {
        if (given) memcpy(roots + 32 * j, given + 32 * j, 32);
        else if (!root_of(cols[j], N, roots + 32 * j)) return 0;
    }
    return 1;
}

/* ---------------------------------------------- SumCheck ZeroCheck ----- */
/* Fig. side-by-side-zc (right), Sec. 3.3.  Variable x_1 is the most
 * significant bit of the table index, so round i pairs entries k and k+h
 * with h half the current table size.  G_i is sent as its values at
 * t = 0..d+1.  Proof = "ZCS1" | gate | n | d | G_1..G_n | v_1..v_c. */
int zo_proof_size(uint32_t form, uint32_t gate, uint32_t n, uint32_t d, size_t *bytes) {
    int c = gate_cols(gate, d);
    if (c < 0) return 1;
    if (form == 1) *bytes = 16 + 32 * ((size_t)n * (d + 2) + c);
    else *bytes = 20 + 32 + 32 * ((size_t)c + 1);
    return 0;
}

int zo_prove_sumcheck(uint32_t gate, uint32_t n, uint32_t d, const uint8_t *const *cols,
                      const uint8_t *roots_in, uint8_t *proof, size_t cap, size_t *len,
                      uint8_t *r_out, uint8_t *alpha_out) {
    field_init();
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 30) return 1;
    size_t need; zo_proof_size(1, gate, n, d, &need);
    if (cap < need) return 6;
    size_t N = (size_t)1 << n;
    fe *T[65];
    if (!load_cols(cols, c, N, T)) { free_cols(T, c); return 1; }
    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);

    transcript tr; tr_init(&tr, 1, gate, n, d, 0);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    fe r[64];
    for (uint32_t i = 0; i < n; i++) r[i] = tr_squeeze(&tr);

    /* Build MLE: E[k] = prod_i ((1-b_i)(1-r_i) + b_i r_i), b_i = bit (n-i) of k */
    fe *E = (fe *)malloc(N * sizeof(fe));
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)N; k++) {
        fe e = f_one();
        for (uint32_t i = 0; i < n; i++) {
            int b = (int)(((size_t)k >> (n - 1 - i)) & 1);
            e = f_mul(e, b ? r[i] : f_sub(f_one(), r[i]));
        }
        E[k] = e;
    }

    memcpy(proof, "ZCS1", 4);
    le32(proof + 4, gate); le32(proof + 8, n); le32(proof + 12, d);
    uint8_t *pp = proof + 16;
    size_t size = N;
    fe tpt[70];
    for (uint32_t t = 0; t <= d + 1; t++) tpt[t] = f_from_u64(t);
    for (uint32_t i = 0; i < n; i++) {
        size_t h = size / 2;
        fe G[70];
        for (uint32_t t = 0; t <= d + 1; t++) {
            fe tot = f_zero();
            #pragma omp parallel
            {
                fe part = f_zero();
                fe x[65];
                #pragma omp for schedule(static)
                for (long k = 0; k < (long)h; k++) {
                    for (int j = 0; j < c; j++)
                        x[j] = f_add(T[j][k], f_mul(tpt[t], f_sub(T[j][k + h], T[j][k])));
                    fe e = f_add(E[k], f_mul(tpt[t], f_sub(E[k + h], E[k])));
                    part = f_add(part, f_mul(gate_eval(gate, d, x), e));
                }
                #pragma omp critical
                tot = f_add(tot, part);
            }
            G[t] = tot;
        }
        uint8_t msg[70 * 32];
        for (uint32_t t = 0; t <= d + 1; t++) f_to_bytes(G[t], msg + 32 * t);
        memcpy(pp, msg, 32 * (size_t)(d + 2)); pp += 32 * (size_t)(d + 2);
        tr_absorb(&tr, msg, 32 * (size_t)(d + 2));
        fe alpha = tr_squeeze(&tr);
        if (alpha_out) f_to_bytes(alpha, alpha_out + 32 * i);
        /* MLE update: T[k] <- T[k] + alpha (T[k+h] - T[k]) */
        for (int j = 0; j < c; j++) {
            fe *Tj = T[j];
            #pragma omp parallel for schedule(static)
            for (long k = 0; k < (long)h; k++)
                Tj[k] = f_add(Tj[k], f_mul(alpha, f_sub(Tj[k + h], Tj[k])));
        }
        #pragma omp parallel for schedule(static)
        for (long k = 0; k < (long)h; k++)
            E[k] = f_add(E[k], f_mul(alpha, f_sub(E[k + h], E[k])));
        size = h;
    }
    for (int j = 0; j < c; j++) { f_to_bytes(T[j][0], pp); pp += 32; }
    if (r_out) for (uint32_t i = 0; i < n; i++) f_to_bytes(r[i], r_out + 32 * i);
    *len = need;
    free(E); free(roots); free_cols(T, c);
    return 0;
}

/* Lagrange interpolation of the values y[0..m-1] at points 0..m-1, at x. */
static fe lagrange_at(const fe *y, uint32_t m, fe x) {
    fe acc = f_zero();
    for (uint32_t t = 0; t < m; t++) {
        fe num = f_one(), den = f_one();
        for (uint32_t s = 0; s < m; s++) {
            if (s == t) continue;
            num = f_mul(num, f_sub(x, f_from_u64(s)));
            den = f_mul(den, f_sub(f_from_u64(t), f_from_u64(s)));
        }
        acc = f_add(acc, f_mul(y[t], f_mul(num, f_inv(den))));
    }
    return acc;
}

/* SumCheck verifier (Sec. 3.4 round check; final check; MLE openings by
 * direct evaluation f~(x) = sum_b f(b) eq_x(b), Sec. 3.3). */
int zo_verify_sumcheck(uint32_t gate, uint32_t n, uint32_t d, const uint8_t *const *cols,
                       const uint8_t *roots_in, const uint8_t *proof, size_t len, int *accept) {
    field_init();
    *accept = 0;
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 30) return 1;
    size_t need; zo_proof_size(1, gate, n, d, &need);
    if (len != need || memcmp(proof, "ZCS1", 4) != 0) return 1;
    uint8_t hdr[16]; memcpy(hdr, "ZCS1", 4); le32(hdr + 4, gate); le32(hdr + 8, n); le32(hdr + 12, d);
    if (memcmp(hdr, proof, 16) != 0) return 1;
    size_t N = (size_t)1 << n;
    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);
    transcript tr; tr_init(&tr, 1, gate, n, d, 0);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    free(roots);
    fe r[64], alpha[64];
    for (uint32_t i = 0; i < n; i++) r[i] = tr_squeeze(&tr);
    const uint8_t *pp = proof + 16;
    fe claim = f_zero();
    int ok = 1;
    for (uint32_t i = 0; i < n; i++) {
        fe G[70];
        for (uint32_t t = 0; t <= d + 1; t++)
            if (!f_from_bytes(pp + 32 * t, &G[t])) return 1;
        if (!f_eq(f_add(G[0], G[1]), claim)) ok = 0;
        tr_absorb(&tr, pp, 32 * (size_t)(d + 2));
        pp += 32 * (size_t)(d + 2);
        alpha[i] = tr_squeeze(&tr);
        claim = lagrange_at(G, d + 2, alpha[i]);
    }
    fe v[65];
    for (int j = 0; j < c; j++) if (!f_from_bytes(pp + 32 * j, &v[j])) return 1;
    fe eqra = f_one();
    for (uint32_t i = 0; i < n; i++)
        eqra = f_mul(eqra, f_add(f_mul(r[i], alpha[i]),
                                 f_mul(f_sub(f_one(), r[i]), f_sub(f_one(), alpha[i]))));
    if (!f_eq(claim, f_mul(gate_eval(gate, d, v), eqra))) ok = 0;
    /* oracle access to the columns: v_j = sum_b col_j[b] eq_alpha(b) */
    fe *T[65];
    if (!load_cols(cols, c, N, T)) { free_cols(T, c); return 1; }
    for (int j = 0; j < c && ok; j++) {
        fe tot = f_zero();
        #pragma omp parallel
        {
            fe part = f_zero();
            #pragma omp for schedule(static)
            for (long k = 0; k < (long)N; k++) {
                fe e = f_one();
                for (uint32_t i = 0; i < n; i++) {
                    int b = (int)(((size_t)k >> (n - 1 - i)) & 1);
                    e = f_mul(e, b ? alpha[i] : f_sub(f_one(), alpha[i]));
                }
                part = f_add(part, f_mul(T[j][k], e));
            }
            #pragma omp critical
            tot = f_add(tot, part);
        }
        if (!f_eq(tot, v[j])) ok = 0;
    }
    free_cols(T, c);
    *accept = ok;
    return 0;
}

/* ------------------------------- eq-factored SumCheck (transcript v2) -- */
/* Sec. 3.3 with the eq factor split off, as in the faster SumCheck provers
 * the paper cites for Build MLE: G_i(X) = c_i l_i(X) H_i(X), where
 *   c_i = prod_{j<i} eq(alpha_j, r_j),  l_i(X) = (1 - r_i)(1 - X) + r_i X,
 *   H_i(X) = sum over x in {0,1}^{n-i} of f_M(alpha_<i, X, x) eq_{r_>i}(x).
 * c_i and l_i are known to the verifier, so a round sends H_i, of degree d,
 * at X = 0..d (d + 1 values instead of G_i's d + 2).  The verifier checks
 * c_i ((1 - r_i) H_i(0) + r_i H_i(1)) = claim, then claim <- c_i l_i(alpha_i)
 * H_i(alpha_i) and c_{i+1} = c_i l_i(alpha_i).  Transcript tag
 * "zerocheck-gb300/v2" (form word 3); absorbs enc(H_i(0..d)).
 * Proof = "ZCS2" | gate | n | d | H_1..H_n | v_1..v_c. */
int zo_proof_size_eq(uint32_t gate, uint32_t n, uint32_t d, size_t *bytes) {
    int c = gate_cols(gate, d);
    if (c < 0) return 1;
    *bytes = 16 + 32 * ((size_t)n * (d + 1) + c);
    return 0;
}

int zo_prove_sumcheck_eq(uint32_t gate, uint32_t n, uint32_t d, const uint8_t *const *cols,
                         const uint8_t *roots_in, uint8_t *proof, size_t cap, size_t *len,
                         uint8_t *r_out, uint8_t *alpha_out) {
    field_init();
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 30) return 1;
    size_t need; zo_proof_size_eq(gate, n, d, &need);
    if (cap < need) return 6;
    size_t N = (size_t)1 << n;
    fe *T[65];
    if (!load_cols(cols, c, N, T)) { free_cols(T, c); return 1; }
    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);

    transcript tr; tr_init_tag(&tr, "zerocheck-gb300/v2", 3, gate, n, d, 0);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    fe r[64];
    for (uint32_t i = 0; i < n; i++) r[i] = tr_squeeze(&tr);

    memcpy(proof, "ZCS2", 4);
    le32(proof + 4, gate); le32(proof + 8, n); le32(proof + 12, d);
    uint8_t *pp = proof + 16;
    fe *E = (fe *)malloc((N / 2 + 1) * sizeof(fe));
    fe tpt[70];
    for (uint32_t t = 0; t <= d; t++) tpt[t] = f_from_u64(t);
    size_t size = N;
    for (uint32_t i = 0; i < n; i++) {
        size_t h = size / 2;
        /* eq_{r_>i}(x) over the remaining n - i - 1 variables, x MSB first */
        const uint32_t m = n - i - 1;
        #pragma omp parallel for schedule(static)
        for (long k = 0; k < (long)h; k++) {
            fe e = f_one();
            for (uint32_t l = 0; l < m; l++) {
                int b = (int)(((size_t)k >> (m - 1 - l)) & 1);
                fe rl = r[i + 1 + l];
                e = f_mul(e, b ? rl : f_sub(f_one(), rl));
            }
            E[k] = e;
        }
        fe H[70];
        for (uint32_t t = 0; t <= d; t++) {
            fe tot = f_zero();
            #pragma omp parallel
            {
                fe part = f_zero();
                fe x[65];
                #pragma omp for schedule(static)
                for (long k = 0; k < (long)h; k++) {
                    for (int j = 0; j < c; j++)
                        x[j] = f_add(T[j][k], f_mul(tpt[t], f_sub(T[j][k + h], T[j][k])));
                    part = f_add(part, f_mul(gate_eval(gate, d, x), E[k]));
                }
                #pragma omp critical
                tot = f_add(tot, part);
            }
            H[t] = tot;
        }
        uint8_t msg[70 * 32];
        for (uint32_t t = 0; t <= d; t++) f_to_bytes(H[t], msg + 32 * t);
        memcpy(pp, msg, 32 * (size_t)(d + 1)); pp += 32 * (size_t)(d + 1);
        tr_absorb(&tr, msg, 32 * (size_t)(d + 1));
        fe alpha = tr_squeeze(&tr);
        if (alpha_out) f_to_bytes(alpha, alpha_out + 32 * i);
        for (int j = 0; j < c; j++) {
            fe *Tj = T[j];
            #pragma omp parallel for schedule(static)
            for (long k = 0; k < (long)h; k++)
                Tj[k] = f_add(Tj[k], f_mul(alpha, f_sub(Tj[k + h], Tj[k])));
        }
        size = h;
    }
    for (int j = 0; j < c; j++) { f_to_bytes(T[j][0], pp); pp += 32; }
    if (r_out) for (uint32_t i = 0; i < n; i++) f_to_bytes(r[i], r_out + 32 * i);
    *len = need;
    free(E); free(roots); free_cols(T, c);
    return 0;
}

int zo_verify_sumcheck_eq(uint32_t gate, uint32_t n, uint32_t d, const uint8_t *const *cols,
                          const uint8_t *roots_in, const uint8_t *proof, size_t len, int *accept) {
    field_init();
    *accept = 0;
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 30) return 1;
    size_t need; zo_proof_size_eq(gate, n, d, &need);
    if (len != need) return 1;
    uint8_t hdr[16]; memcpy(hdr, "ZCS2", 4); le32(hdr + 4, gate); le32(hdr + 8, n); le32(hdr + 12, d);
    if (memcmp(hdr, proof, 16) != 0) return 1;
    size_t N = (size_t)1 << n;
    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);
    transcript tr; tr_init_tag(&tr, "zerocheck-gb300/v2", 3, gate, n, d, 0);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    free(roots);
    fe r[64], alpha[64];
    for (uint32_t i = 0; i < n; i++) r[i] = tr_squeeze(&tr);
    const uint8_t *pp = proof + 16;
    fe claim = f_zero(), ci = f_one();
    int ok = 1;
    for (uint32_t i = 0; i < n; i++) {
        fe H[70];
        for (uint32_t t = 0; t <= d; t++)
            if (!f_from_bytes(pp + 32 * t, &H[t])) return 1;
        fe sum = f_add(f_mul(f_sub(f_one(), r[i]), H[0]), f_mul(r[i], H[1]));
        if (!f_eq(f_mul(ci, sum), claim)) ok = 0;
        tr_absorb(&tr, pp, 32 * (size_t)(d + 1));
        pp += 32 * (size_t)(d + 1);
        alpha[i] = tr_squeeze(&tr);
        fe li = f_add(f_mul(f_sub(f_one(), r[i]), f_sub(f_one(), alpha[i])), f_mul(r[i], alpha[i]));
        ci = f_mul(ci, li);
        claim = f_mul(ci, lagrange_at(H, d + 1, alpha[i]));
    }
    fe v[65];
    for (int j = 0; j < c; j++) if (!f_from_bytes(pp + 32 * j, &v[j])) return 1;
    if (!f_eq(claim, f_mul(gate_eval(gate, d, v), ci))) ok = 0;
    fe *T[65];
    if (!load_cols(cols, c, N, T)) { free_cols(T, c); return 1; }
    for (int j = 0; j < c && ok; j++) {
        fe tot = f_zero();
        #pragma omp parallel
        {
            fe part = f_zero();
            #pragma omp for schedule(static)
            for (long k = 0; k < (long)N; k++) {
                fe e = f_one();
                for (uint32_t i = 0; i < n; i++) {
                    int b = (int)(((size_t)k >> (n - 1 - i)) & 1);
                    e = f_mul(e, b ? alpha[i] : f_sub(f_one(), alpha[i]));
                }
                part = f_add(part, f_mul(T[j][k], e));
            }
            #pragma omp critical
            tot = f_add(tot, part);
        }
        if (!f_eq(tot, v[j])) ok = 0;
    }
    free_cols(T, c);
    *accept = ok;
    return 0;
}

/* ------------------------------------------------- NTT ZeroCheck ------- */
/* Fig. side-by-side-zc (left), Sec. 3.2.  Column j holds g_j(w_N^i) at
 * index i.  The domain D is given by a domain word w:
 *   - power of two (w < 256): D = {7 w_M^i}, M = 2^k N with k = w (0: the
 *     default log2(next_pow2(d)));
 *   - step radix (w = k | (s+1) << 8, s < k): D = D_big u D_small with
 *     D_big = {7 w_Mb^i}, Mb = 2^k N, and D_small = {sigma w_Ms^i},
 *     Ms = 2^s N, sigma = 7 w_{2 Mb}; M = Mb + Ms (Sec. 4, "Degree
 *     scaling": a non-power-of-two transform, e.g. 3N = 2N + N, built from
 *     power-of-two transforms plus element-wise work).
 * Any M >= (d-1)N holds the quotient.  The header and the transcript carry
 * log2 M (power of two) or log2 Mb | (log2 Ms + 1) << 8 (step radix).
 * Proof = "ZCN1" | gate | n | d | domain | root(q) | g_j(z) ... | q(z). */

static uint32_t default_blowup(uint32_t d) { return ilog2(d); }

typedef struct { unsigned k, s; int step; size_t N, Mb, Ms, M; uint32_t word; } ntt_domain;

/* The domain with big part 2^k N and, if step, small part 2^s N (s < k),
 * for size n and degree d; 0 if it is invalid or cannot hold the quotient. */
static int domain_make(uint32_t n, uint32_t d, unsigned k, int step, unsigned s, ntt_domain *D) {
    D->k = k; D->s = step ? s : 0; D->step = step;
    if (n + k > 32 || (step && s >= k)) return 0;
    D->N = (size_t)1 << n;
    D->Mb = D->N << k;
    D->Ms = step ? D->N << s : 0;
    D->M = D->Mb + D->Ms;
    /* |D| must hold the quotient's (d-1)N - d + 1 coefficients (Sec. 4,
     * degree scaling: the NTT size follows the degree of q) */
    if (D->M < (size_t)(d - 1) * D->N - d + 1) return 0;
    D->word = step ? (n + k) | ((n + s + 1) << 8) : n + k;
    return 1;
}

/* From the caller's domain word (0: the default 2^log2(next_pow2(d)) N). */
static int domain_of(uint32_t n, uint32_t d, uint32_t w, ntt_domain *D) {
    if (w >> 16) return 0;
    const unsigned k = w & 0xff, sp1 = (w >> 8) & 0xff;
    if (sp1) return k > 0 && domain_make(n, d, k, 1, sp1 - 1, D);
    return domain_make(n, d, k ? k : default_blowup(d), 0, 0, D);
}

/* From the proof header's word (log2 M, or log2 Mb | (log2 Ms + 1) << 8). */
static int domain_of_header(uint32_t n, uint32_t d, uint32_t W, ntt_domain *D) {
    if (W >> 16) return 0;
    const unsigned lb = W & 0xff, sl = (W >> 8) & 0xff;
    if (lb < n) return 0;
    if (!sl) return domain_make(n, d, lb - n, 0, 0, D);
    if (sl < n + 1) return 0;
    return domain_make(n, d, lb - n, 1, sl - 1 - n, D);
}

/* coefficients of g from its values on H: N^{-1} sum_i e_i w_N^{-ik} */
static void intt_h(fe *a, unsigned n) {
    size_t N = (size_t)1 << n;
    ntt_inplace(a, n, f_inv(root_of_unity(n)));
    fe ninv = f_inv(f_from_u64(N));
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)N; k++) a[k] = f_mul(a[k], ninv);
}

/* evaluations of the coefficient vector c (length N) on the coset
 * shift <w_M>: out[i] = sum_k c[k] (shift w_M^i)^k */
static void coset_lde_at(const fe *coef, unsigned n, unsigned logm, fe shift, fe *out) {
    size_t N = (size_t)1 << n, M = (size_t)1 << logm;
    /* out[k] = coef[k] * shift^k for k < N, zero above */
    powers(shift, N, out);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)M; k++)
        out[k] = (size_t)k < N ? f_mul(coef[k], out[k]) : f_zero();
    ntt_inplace(out, logm, root_of_unity(logm));
}

static void coset_lde(const fe *coef, unsigned n, unsigned logm, fe *out) {
    coset_lde_at(coef, n, logm, f_from_u64(7), out);
}

/* f-hat / z_H at the M = 2^logm points x_i = shift w_M^i of a coset:
 * evaluations of the g_j there (coset LDE), the gate pointwise, then the
 * element-wise division by z_H(x_i) = x_i^N - 1.  fh, tmp: M entries. */
static void quotient_evals(uint32_t gate, uint32_t d, int c, fe *const *G, unsigned n, unsigned logm,
                           fe shift, fe *fh, fe *tmp) {
    size_t N = (size_t)1 << n, M = (size_t)1 << logm;
    if (gate == GATE_PLONK) {
        fe *L[8];
        for (int j = 0; j < 8; j++) { L[j] = (fe *)malloc(M * sizeof(fe)); coset_lde_at(G[j], n, logm, shift, L[j]); }
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)M; i++) {
            fe x[8];
            for (int j = 0; j < 8; j++) x[j] = L[j][i];
            fh[i] = gate_eval(gate, d, x);
        }
        for (int j = 0; j < 8; j++) free(L[j]);
    } else {
        /* running product of the first d columns, then minus o (product gate)
         * or plus the single columns (sum gate) */
        coset_lde_at(G[0], n, logm, shift, fh);
        for (uint32_t j = 1; j < d; j++) {
            coset_lde_at(G[j], n, logm, shift, tmp);
            #pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)M; i++) fh[i] = f_mul(fh[i], tmp[i]);
        }
        if ((gate & 0xff) == GATE_PRODUCT) {
            coset_lde_at(G[d], n, logm, shift, tmp);
            #pragma omp parallel for schedule(static)
            for (long i = 0; i < (long)M; i++) fh[i] = f_sub(fh[i], tmp[i]);
        } else {
            for (int j = (int)d; j < c; j++) {
                coset_lde_at(G[j], n, logm, shift, tmp);
                #pragma omp parallel for schedule(static)
                for (long i = 0; i < (long)M; i++) fh[i] = f_add(fh[i], tmp[i]);
            }
        }
    }
    /* evals of z_H = x^N - 1 at x_i = shift w_M^i, then element-wise division */
    powers(root_of_unity(logm), M, tmp);                  /* w_M^i */
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)M; i++) {
        fe xi = f_mul(shift, tmp[i]);
        tmp[i] = f_sub(f_pow_u64(xi, N), f_one());
    }
    f_batch_inv(tmp, M);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)M; i++) fh[i] = f_mul(fh[i], tmp[i]);
}

/* INTT on a coset, in place: v[k] <- M^{-1} shift^{-k} sum_i v[i] w_M^{-ik},
 * the coefficients of the degree < M polynomial with those values at the
 * points shift w_M^i.  tmp: M entries. */
static void coset_intt(fe *v, unsigned logm, fe shift, fe *tmp) {
    size_t M = (size_t)1 << logm;
    ntt_inplace(v, logm, f_inv(root_of_unity(logm)));
    fe minv = f_inv(f_from_u64(M));
    powers(f_inv(shift), M, tmp);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)M; k++) v[k] = f_mul(v[k], f_mul(minv, tmp[k]));
}

int zo_prove_ntt(uint32_t gate, uint32_t n, uint32_t d, uint32_t log_blowup,
                 const uint8_t *const *cols, const uint8_t *roots_in,
                 uint8_t *proof, size_t cap, size_t *len, uint8_t *q_out) {
    field_init();
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 28) return 1;
    ntt_domain D;
    if (!domain_of(n, d, log_blowup, &D)) return 1;
    size_t need; zo_proof_size(2, gate, n, d, &need);
    if (cap < need) return 6;
    size_t N = D.N, M = D.M, Mb = D.Mb, Ms = D.Ms;

    fe *G[65];
    if (!load_cols(cols, c, N, G)) { free_cols(G, c); return 1; }
    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);

    /* 1. g_j <- INTT_H(evals g_j) */
    for (int j = 0; j < c; j++) intt_h(G[j], n);

    /* 2-5 on D_big: qhat = gate(ghat) / z_H, then q_big <- INTT_D_big(qhat):
     * the degree < Mb polynomial that matches q on D_big */
    const fe seven = f_from_u64(7);
    fe *q = (fe *)malloc(M * sizeof(fe));
    fe *tmp = (fe *)malloc(Mb * sizeof(fe));
    quotient_evals(gate, d, c, G, n, n + D.k, seven, q, tmp);
    coset_intt(q, n + D.k, seven, tmp);
    if (D.step) {
        /* step radix: q = q_big + (x^Mb - 7^Mb) q_small with deg q_small < Ms.
         * On D_small x^Mb = sigma^Mb, so q_small there is
         * (qhat - q_big) / (sigma^Mb - 7^Mb): evaluate q_big on D_small
         * (reduce it modulo x^Ms - sigma^Ms, then a coset NTT of Ms points),
         * subtract, scale, and interpolate with a coset INTT of Ms points. */
        const fe sigma = f_mul(seven, root_of_unity(n + D.k + 1));
        fe *hs = (fe *)malloc(Ms * sizeof(fe)), *vs = (fe *)malloc(Ms * sizeof(fe));
        fe *t2 = (fe *)malloc(Ms * sizeof(fe));
        quotient_evals(gate, d, c, G, n, n + D.s, sigma, hs, t2);
        const fe sms = f_pow_u64(sigma, Ms);
        const size_t parts = Mb / Ms;
        #pragma omp parallel for schedule(static)
        for (long kk = 0; kk < (long)Ms; kk++) {
            fe acc = f_zero();                            /* Horner in sigma^Ms */
            for (size_t m = parts; m-- > 0;) acc = f_add(f_mul(acc, sms), q[(size_t)kk + m * Ms]);
            t2[kk] = acc;
        }
        coset_lde_at(t2, n + D.s, n + D.s, sigma, vs);   /* q_big on D_small */
        const fe s7mb = f_pow_u64(seven, Mb);
        const fe kinv = f_inv(f_sub(f_pow_u64(sigma, Mb), s7mb));
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < (long)Ms; i++) hs[i] = f_mul(f_sub(hs[i], vs[i]), kinv);
        coset_intt(hs, n + D.s, sigma, t2);               /* q_small */
        #pragma omp parallel for schedule(static)
        for (long kk = 0; kk < (long)Ms; kk++) {
            q[kk] = f_sub(q[kk], f_mul(s7mb, hs[kk]));
            q[Mb + (size_t)kk] = hs[kk];
        }
        free(hs); free(vs); free(t2);
    }

    uint8_t *qb = q_out ? q_out : (uint8_t *)malloc(M * 32);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < (long)M; k++) f_to_bytes(q[k], qb + (size_t)k * 32);
    uint8_t qroot[32];
    root_of(qb, M, qroot);

    /* 6. r <- Hash([g], [q]); re-squeeze while z lies in H */
    transcript tr; tr_init(&tr, 2, gate, n, d, D.word);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    tr_absorb(&tr, qroot, 32);
    fe z;
    do { z = tr_squeeze(&tr); } while (f_eq(f_pow_u64(z, N), f_one()));

    /* 7. open g_j(z), q(z) by Horner */
    memcpy(proof, "ZCN1", 4);
    le32(proof + 4, gate); le32(proof + 8, n); le32(proof + 12, d); le32(proof + 16, D.word);
    memcpy(proof + 20, qroot, 32);
    uint8_t *pp = proof + 52;
    for (int j = 0; j < c; j++) {
        fe y = f_zero();
        for (size_t k = N; k-- > 0;) y = f_add(f_mul(y, z), G[j][k]);
        f_to_bytes(y, pp); pp += 32;
    }
    fe tq = f_zero();
    for (size_t k = M; k-- > 0;) tq = f_add(f_mul(tq, z), q[k]);
    f_to_bytes(tq, pp);
    *len = need;
    if (!q_out) free(qb);
    free(q); free(tmp); free(roots); free_cols(G, c);
    return 0;
}

/* NTT verifier: root(q), degree bound deg q <= deg f - N (Sec. 3.2),
 * t = q(z), g_j(z) from the evaluations on H by the barycentric formula
 * (oracle access), and gate(g(z)) = z_H(z) t (Sec. 3.2). */
int zo_verify_ntt(uint32_t gate, uint32_t n, uint32_t d, const uint8_t *const *cols,
                  const uint8_t *roots_in, const uint8_t *proof, size_t len,
                  const uint8_t *q, int *accept) {
    field_init();
    *accept = 0;
    int c = gate_cols(gate, d);
    if (c < 0 || n < 1 || n > 28) return 1;
    size_t need; zo_proof_size(2, gate, n, d, &need);
    if (len != need || memcmp(proof, "ZCN1", 4) != 0) return 1;
    uint32_t word = 0;
    for (int i = 3; i >= 0; i--) word = (word << 8) | proof[16 + i];
    ntt_domain D;
    if (!domain_of_header(n, d, word, &D)) return 1;
    uint8_t hdr[20]; memcpy(hdr, "ZCN1", 4);
    le32(hdr + 4, gate); le32(hdr + 8, n); le32(hdr + 12, d); le32(hdr + 16, word);
    if (memcmp(hdr, proof, 20) != 0) return 1;
    size_t N = (size_t)1 << n, M = D.M;
    int ok = 1;

    uint8_t qroot[32];
    if (!root_of(q, M, qroot)) return 1;
    if (memcmp(qroot, proof + 20, 32) != 0) ok = 0;

    uint8_t *roots = (uint8_t *)malloc(32 * (size_t)c);
    col_roots(cols, c, N, roots_in, roots);
    transcript tr; tr_init(&tr, 2, gate, n, d, word);
    for (int j = 0; j < c; j++) tr_absorb(&tr, roots + 32 * j, 32);
    free(roots);
    tr_absorb(&tr, proof + 20, 32);
    fe z;
    do { z = tr_squeeze(&tr); } while (f_eq(f_pow_u64(z, N), f_one()));

    /* degree bound and t = q(z) */
    size_t qlen = (size_t)(d - 1) * N - d + 1;
    fe tq = f_zero();
    for (size_t k = M; k-- > 0;) {
        fe qk;
        if (!f_from_bytes(q + k * 32, &qk)) return 1;
        if (k >= qlen && !f_is_zero(qk)) ok = 0;
        tq = f_add(f_mul(tq, z), qk);
    }
    fe t_claim, y[65];
    const uint8_t *pp = proof + 52;
    for (int j = 0; j < c; j++) if (!f_from_bytes(pp + 32 * j, &y[j])) return 1;
    if (!f_from_bytes(pp + 32 * c, &t_claim)) return 1;
    if (!f_eq(tq, t_claim)) ok = 0;

    /* barycentric g_j(z) = (z^N - 1)/N sum_i e_i w^i / (z - w^i) */
    fe wN = root_of_unity(n);
    fe *den = (fe *)malloc(N * sizeof(fe)), *wi = (fe *)malloc(N * sizeof(fe));
    powers(wN, N, wi);
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)N; i++) den[i] = f_sub(z, wi[i]);
    f_batch_inv(den, N);
    fe zn1 = f_sub(f_pow_u64(z, N), f_one());
    fe scale = f_mul(zn1, f_inv(f_from_u64(N)));
    for (int j = 0; j < c; j++) {
        fe tot = f_zero();
        int okj = 1;
        #pragma omp parallel
        {
            fe part = f_zero();
            #pragma omp for schedule(static) reduction(&:okj)
            for (long i = 0; i < (long)N; i++) {
                fe e;
                okj &= f_from_bytes(cols[j] + (size_t)i * 32, &e);
                part = f_add(part, f_mul(e, f_mul(wi[i], den[i])));
            }
            #pragma omp critical
            tot = f_add(tot, part);
        }
        if (!okj) { free(den); free(wi); return 1; }
        if (!f_eq(f_mul(tot, scale), y[j])) ok = 0;
    }
    free(den); free(wi);
    if (!f_eq(gate_eval(gate, d, y), f_mul(zn1, tq))) ok = 0;
    *accept = ok;
    return 0;
}

/* ------------------------------- hash-based PCS around the ZeroCheck -- */
/* Stages (1) and (3) of the prover workflow (Sec. 3.1): commit to the
 * witness columns, then open them at the point the ZeroCheck's SumCheck
 * ends in, with the lightweight hash-based commitment the paper points to
 * (Ligero, Sec. 3.1).  The c columns (MLE tables of N = 2^n values, x_1 the
 * most significant index bit) are m x w matrices, w = 2^nc (1 <= nc <= n;
 * the library's default is min(n, 12)), m = 2^(n - nc), row i holding
 * entries i w .. i w + w - 1.
 *   Commit: every row is Reed-Solomon encoded at rate 1/4, as the values of
 *   the polynomial with the row as coefficients at the W = 4w points
 *   x_k = 7 w_W^k: E[i][k] = sum_l M[i][l] x_k^l.  Column digest
 *   D_kj = SHA-256(enc(E_j[0][k]) | ... | enc(E_j[m-1][k])), leaf
 *   L_k = SHA-256(D_k0 | ... | D_k,c-1), binary Merkle tree over the W
 *   leaves, root = SHA-256(le64(W) | top).
 *   Open at alpha with values v_j: transcript S = SHA-256(
 *   "zerocheck-gb300/pcs-v1" | u32 n | u32 nc | u32 c | u32 t | root | enc(alpha_i)
 *   | enc(v_j)); u_j = sum_i eq(alpha_1..nr, i) M_j[i] (so that
 *   v_j = <u_j, eq(alpha_nr+1..n, .)>); absorb enc(u_0..u_c-1); gamma =
 *   squeeze; u' = sum_j,i gamma^(j m + i) M_j[i] (proximity); absorb
 *   enc(u'); t queries k_s = squeeze mod W.  Proof = "ZCP1" | u32 n | u32 nc
 *   | u32 c | u32 t | u_j | u' | per query: enc(E_j[i][k_s]) for j, i, then the
 *   log2 W sibling digests from the leaf up.
 *   Verify: <u_j, eq_lo> = v_j; each queried column hashes up to the root;
 *   its entries combine to the encodings of u_j (with eq_hi) and of u'
 *   (with the gamma powers) at x_k. */
typedef struct { unsigned n, nc, nr; size_t m, w, W; unsigned logW; } pcs_shape;

static int pcs_shape_of(unsigned n, unsigned nc, pcs_shape *P) {
    if (n < 1 || n > 24 || nc < 1 || nc > n) return 0;
    P->n = n; P->nc = nc; P->nr = n - P->nc;
    P->m = (size_t)1 << P->nr; P->w = (size_t)1 << P->nc; P->W = P->w * 4; P->logW = P->nc + 2;
    return 1;
}

int zo_pcs_proof_size(uint32_t n, uint32_t nc, uint32_t c, uint32_t t, size_t *bytes) {
    pcs_shape P;
    if (!pcs_shape_of(n, nc, &P) || c < 1 || c > 65 || t < 1) return 1;
    *bytes = 20 + 32 * (c * P.w + P.w + (size_t)t * c * P.m + (size_t)t * P.logW);
    return 0;
}

/* E_j[i][k] for all i < m, k < W (row-major by i), canonical fe */
static void pcs_encode(const fe *M, const pcs_shape *P, fe *E) {
    fe *row = (fe *)malloc(P->W * sizeof(fe));
    for (size_t i = 0; i < P->m; i++) {
        coset_lde(M + i * P->w, P->nc, P->logW, row);          /* values at 7 w_W^k */
        memcpy(E + i * P->W, row, P->W * sizeof(fe));
    }
    free(row);
}

/* leaf digests of all W columns of the c encoded matrices */
static void pcs_leaves(fe *const *E, uint32_t c, const pcs_shape *P, uint8_t *leaves) {
    #pragma omp parallel
    {
        uint8_t *buf = (uint8_t *)malloc(P->m * 32), *dg = (uint8_t *)malloc(32 * (size_t)c);
        #pragma omp for schedule(static)
        for (long k = 0; k < (long)P->W; k++) {
            for (uint32_t j = 0; j < c; j++) {
                for (size_t i = 0; i < P->m; i++) f_to_bytes(E[j][i * P->W + (size_t)k], buf + 32 * i);
                sha256(buf, P->m * 32, dg + 32 * j);
            }
            sha256(dg, 32 * (size_t)c, leaves + 32 * (size_t)k);
        }
        free(buf); free(dg);
    }
}

/* all levels of the tree: level 0 = leaves (W), level l has W >> l nodes */
static uint8_t *pcs_tree(const uint8_t *leaves, const pcs_shape *P, uint8_t root[32]) {
    uint8_t *T = (uint8_t *)malloc(2 * P->W * 32);
    memcpy(T, leaves, P->W * 32);
    size_t off = 0, cnt = P->W;
    while (cnt > 1) {
        for (size_t u = 0; u < cnt / 2; u++) sha256(T + (off + 2 * u) * 32, 64, T + (off + cnt + u) * 32);
        off += cnt; cnt /= 2;
    }
    uint8_t msg[40];
    for (int i = 0; i < 8; i++) msg[i] = (uint8_t)((uint64_t)P->W >> (8 * i));
    memcpy(msg + 8, T + off * 32, 32);
    sha256(msg, 40, root);
    return T;
}

static int pcs_load(const uint8_t *const *cols, uint32_t c, const pcs_shape *P, fe **M, fe **E) {
    if (!load_cols(cols, (int)c, P->m * P->w, M)) return 0;
    for (uint32_t j = 0; j < c; j++) {
        E[j] = (fe *)malloc(P->m * P->W * sizeof(fe));
        pcs_encode(M[j], P, E[j]);
    }
    return 1;
}

int zo_pcs_commit(uint32_t n, uint32_t nc, uint32_t c, const uint8_t *const *cols, uint8_t *root) {
    field_init();
    pcs_shape P;
    if (!pcs_shape_of(n, nc, &P) || c < 1 || c > 65) return 1;
    fe *M[65], *E[65];
    if (!pcs_load(cols, c, &P, M, E)) { free_cols(M, (int)c); return 1; }
    uint8_t *leaves = (uint8_t *)malloc(P.W * 32);
    pcs_leaves(E, c, &P, leaves);
    free(pcs_tree(leaves, &P, root));
    free(leaves); free_cols(M, (int)c); free_cols(E, (int)c);
    return 0;
}

/* eq(x, b) over the variables x[0..k) for every b < 2^k, b_1 the MSB */
static void eq_table(const fe *x, unsigned k, fe *out) {
    for (size_t b = 0; b < ((size_t)1 << k); b++) {
        fe e = f_one();
        for (unsigned l = 0; l < k; l++) {
            int bit = (int)((b >> (k - 1 - l)) & 1);
            e = f_mul(e, bit ? x[l] : f_sub(f_one(), x[l]));
        }
        out[b] = e;
    }
}

static void pcs_transcript(transcript *tr, uint32_t n, uint32_t nc, uint32_t c, uint32_t t,
                           const uint8_t root[32], const fe *alpha, const fe *v) {
    sha_ctx s; sha_init(&s);
    const char *tag = "zerocheck-gb300/pcs-v1";
    sha_update(&s, (const uint8_t *)tag, strlen(tag));
    uint8_t b4[4], b32[32];
    le32(b4, n); sha_update(&s, b4, 4);
    le32(b4, nc); sha_update(&s, b4, 4);
    le32(b4, c); sha_update(&s, b4, 4);
    le32(b4, t); sha_update(&s, b4, 4);
    sha_update(&s, root, 32);
    for (uint32_t i = 0; i < n; i++) { f_to_bytes(alpha[i], b32); sha_update(&s, b32, 32); }
    for (uint32_t j = 0; j < c; j++) { f_to_bytes(v[j], b32); sha_update(&s, b32, 32); }
    sha_final(&s, tr->s);
}

static int load_fes(const uint8_t *b, size_t cnt, fe *out) {
    for (size_t i = 0; i < cnt; i++) if (!f_from_bytes(b + 32 * i, &out[i])) return 0;
    return 1;
}

static size_t query_index(transcript *tr, const pcs_shape *P) {
    fe q = tr_squeeze(tr);
    uint8_t b[32]; f_to_bytes(q, b);
    uint64_t x = 0;
    for (int i = 7; i >= 0; i--) x = (x << 8) | b[i];
    return (size_t)(x & (P->W - 1));
}

int zo_pcs_open(uint32_t n, uint32_t nc, uint32_t c, uint32_t t, const uint8_t *const *cols,
                const uint8_t *alpha_b, const uint8_t *values_b, uint8_t *proof, size_t cap, size_t *len) {
    field_init();
    size_t need;
    if (zo_pcs_proof_size(n, nc, c, t, &need)) return 1;
    if (cap < need) return 6;
    pcs_shape P; pcs_shape_of(n, nc, &P);
    fe alpha[64], v[65];
    if (!load_fes(alpha_b, n, alpha) || !load_fes(values_b, c, v)) return 1;
    fe *M[65], *E[65];
    if (!pcs_load(cols, c, &P, M, E)) { free_cols(M, (int)c); return 1; }
    uint8_t *leaves = (uint8_t *)malloc(P.W * 32), root[32];
    pcs_leaves(E, c, &P, leaves);
    uint8_t *tree = pcs_tree(leaves, &P, root);
    transcript tr; pcs_transcript(&tr, n, nc, c, t, root, alpha, v);
    memcpy(proof, "ZCP1", 4); le32(proof + 4, n); le32(proof + 8, nc); le32(proof + 12, c); le32(proof + 16, t);
    uint8_t *pp = proof + 20;
    /* u_j = sum_i eq(alpha_hi, i) M_j[i] */
    fe *eqh = (fe *)malloc(P.m * sizeof(fe));
    eq_table(alpha, P.nr, eqh);
    uint8_t *ub = pp;
    for (uint32_t j = 0; j < c; j++)
        for (size_t l = 0; l < P.w; l++) {
            fe a = f_zero();
            for (size_t i = 0; i < P.m; i++) a = f_add(a, f_mul(eqh[i], M[j][i * P.w + l]));
            f_to_bytes(a, pp); pp += 32;
        }
    tr_absorb(&tr, ub, 32 * (size_t)c * P.w);
    const fe gamma = tr_squeeze(&tr);
    /* u' = sum_{j,i} gamma^(j m + i) M_j[i] */
    fe *up = (fe *)calloc(P.w, sizeof(fe));
    fe g = f_one();
    for (uint32_t j = 0; j < c; j++)
        for (size_t i = 0; i < P.m; i++) {
            for (size_t l = 0; l < P.w; l++) up[l] = f_add(up[l], f_mul(g, M[j][i * P.w + l]));
            g = f_mul(g, gamma);
        }
    uint8_t *upb = pp;
    for (size_t l = 0; l < P.w; l++) { f_to_bytes(up[l], pp); pp += 32; }
    tr_absorb(&tr, upb, 32 * P.w);
    for (uint32_t s = 0; s < t; s++) {
        const size_t k = query_index(&tr, &P);
        for (uint32_t j = 0; j < c; j++)
            for (size_t i = 0; i < P.m; i++) { f_to_bytes(E[j][i * P.W + k], pp); pp += 32; }
        size_t off = 0, cnt = P.W, idx = k;
        for (unsigned lv = 0; lv < P.logW; lv++) {
            memcpy(pp, tree + (off + (idx ^ 1)) * 32, 32); pp += 32;
            off += cnt; cnt /= 2; idx >>= 1;
        }
    }
    *len = need;
    free(up); free(eqh); free(tree); free(leaves); free_cols(M, (int)c); free_cols(E, (int)c);
    return 0;
}

int zo_pcs_verify(uint32_t n, uint32_t nc, uint32_t c, uint32_t t, const uint8_t *root,
                  const uint8_t *alpha_b, const uint8_t *values_b, const uint8_t *proof, size_t len,
                  int *accept) {
    field_init();
    *accept = 0;
    size_t need;
    if (zo_pcs_proof_size(n, nc, c, t, &need) || len != need) return 1;
    uint8_t hdr[20]; memcpy(hdr, "ZCP1", 4);
    le32(hdr + 4, n); le32(hdr + 8, nc); le32(hdr + 12, c); le32(hdr + 16, t);
    if (memcmp(hdr, proof, 20) != 0) return 1;
    pcs_shape P; pcs_shape_of(n, nc, &P);
    fe alpha[64], v[65];
    if (!load_fes(alpha_b, n, alpha) || !load_fes(values_b, c, v)) return 1;
    fe *u = (fe *)malloc((size_t)(c + 1) * P.w * sizeof(fe));
    const uint8_t *pp = proof + 20;
    if (!load_fes(pp, (size_t)(c + 1) * P.w, u)) { free(u); return 1; }
    int ok = 1;
    /* v_j = <u_j, eq(alpha_lo, .)> */
    fe *eql = (fe *)malloc(P.w * sizeof(fe)), *eqh = (fe *)malloc(P.m * sizeof(fe));
    eq_table(alpha + P.nr, P.nc, eql);
    eq_table(alpha, P.nr, eqh);
    for (uint32_t j = 0; j < c; j++) {
        fe a = f_zero();
        for (size_t l = 0; l < P.w; l++) a = f_add(a, f_mul(u[j * P.w + l], eql[l]));
        if (!f_eq(a, v[j])) ok = 0;
    }
    transcript tr; pcs_transcript(&tr, n, nc, c, t, root, alpha, v);
    tr_absorb(&tr, pp, 32 * (size_t)c * P.w);
    const fe gamma = tr_squeeze(&tr);
    tr_absorb(&tr, pp + 32 * (size_t)c * P.w, 32 * P.w);
    pp += 32 * (size_t)(c + 1) * P.w;
    fe *gp = (fe *)malloc((size_t)c * P.m * sizeof(fe));
    powers(gamma, (size_t)c * P.m, gp);
    const fe wW = root_of_unity(P.logW), seven = f_from_u64(7);
    fe *col = (fe *)malloc((size_t)c * P.m * sizeof(fe));
    uint8_t *buf = (uint8_t *)malloc(P.m * 32), *dg = (uint8_t *)malloc(32 * (size_t)c);
    for (uint32_t s = 0; s < t && ok; s++) {
        const size_t k = query_index(&tr, &P);
        if (!load_fes(pp, (size_t)c * P.m, col)) { ok = 0; break; }
        /* hash the column up to the root */
        for (uint32_t j = 0; j < c; j++) sha256(pp + 32 * (size_t)j * P.m, P.m * 32, dg + 32 * j);
        uint8_t node[32], pair[64];
        sha256(dg, 32 * (size_t)c, node);
        pp += 32 * (size_t)c * P.m;
        size_t idx = k;
        for (unsigned lv = 0; lv < P.logW; lv++) {
            if (idx & 1) { memcpy(pair, pp, 32); memcpy(pair + 32, node, 32); }
            else { memcpy(pair, node, 32); memcpy(pair + 32, pp, 32); }
            sha256(pair, 64, node);
            pp += 32; idx >>= 1;
        }
        uint8_t msg[40], r2[32];
        for (int i = 0; i < 8; i++) msg[i] = (uint8_t)((uint64_t)P.W >> (8 * i));
        memcpy(msg + 8, node, 32);
        sha256(msg, 40, r2);
        if (memcmp(r2, root, 32) != 0) ok = 0;
        /* encodings of u_j and u' at x_k against the column's combinations */
        const fe xk = f_mul(seven, f_pow_u64(wW, k));
        for (uint32_t j = 0; j <= c; j++) {
            fe enc_u = f_zero();                            /* Horner: sum_l u[l] x_k^l */
            for (size_t l = P.w; l-- > 0;) enc_u = f_add(f_mul(enc_u, xk), u[j * P.w + l]);
            fe comb = f_zero();
            if (j < c) {
                for (size_t i = 0; i < P.m; i++) comb = f_add(comb, f_mul(eqh[i], col[j * P.m + i]));
            } else {
                for (size_t q = 0; q < (size_t)c * P.m; q++) comb = f_add(comb, f_mul(gp[q], col[q]));
            }
            if (!f_eq(enc_u, comb)) ok = 0;
        }
    }
    free(u); free(eql); free(eqh); free(gp); free(col); free(buf); free(dg);
    *accept = ok;
    return 0;
}

/* -------------------------------------------- hooks for the pin tests -- */
/* canonical little-endian bytes in and out */

int zo_fr(int op, const uint8_t *a, const uint8_t *b, uint8_t *out) {
    field_init();
    fe x, y = f_zero();
    if (!f_from_bytes(a, &x)) return 1;
    if (b && !f_from_bytes(b, &y)) return 1;
    fe z;
    switch (op) {
        case 0: z = f_add(x, y); break;
        case 1: z = f_sub(x, y); break;
        case 2: z = f_mul(x, y); break;
        case 3: if (f_is_zero(x)) return 1; z = f_inv(x); break;
        case 4: z = f_neg(x); break;
        default: return 1;
    }
    f_to_bytes(z, out);
    return 0;
}

int zo_root_of_unity(uint32_t logn, uint8_t *out) {
    field_init();
    if (logn > 32) return 1;
    f_to_bytes(root_of_unity(logn), out);
    return 0;
}

void zo_sha256(const uint8_t *m, size_t len, uint8_t *out) { sha256(m, len, out); }

int zo_root(const uint8_t *v, size_t L, uint8_t *out) { return root_of(v, L, out) ? 0 : 1; }

/* forward (inverse=0): A[i] = sum_k a[k] w^(ik); inverse=1: coefficients
 * N^{-1} sum_i a[i] w^(-ik) */
int zo_ntt(const uint8_t *in, uint32_t logn, int inverse, uint8_t *out) {
    field_init();
    size_t N = (size_t)1 << logn;
    fe *a = (fe *)malloc(N * sizeof(fe));
    for (size_t k = 0; k < N; k++) if (!f_from_bytes(in + 32 * k, &a[k])) { free(a); return 1; }
    if (inverse) intt_h(a, logn);
    else ntt_inplace(a, logn, root_of_unity(logn));
    for (size_t k = 0; k < N; k++) f_to_bytes(a[k], out + 32 * k);
    free(a);
    return 0;
}

int zo_coset_lde(const uint8_t *coef, uint32_t n, uint32_t logm, uint8_t *out) {
    field_init();
    size_t N = (size_t)1 << n, M = (size_t)1 << logm;
    fe *a = (fe *)malloc(N * sizeof(fe)), *o = (fe *)malloc(M * sizeof(fe));
    for (size_t k = 0; k < N; k++) if (!f_from_bytes(coef + 32 * k, &a[k])) { free(a); free(o); return 1; }
    coset_lde(a, n, logm, o);
    for (size_t k = 0; k < M; k++) f_to_bytes(o[k], out + 32 * k);
    free(a); free(o);
    return 0;
}

/* transcript squeeze after absorbing one message (pins the byte convention) */
int zo_transcript_demo(uint32_t form, uint32_t gate, uint32_t n, uint32_t d, uint32_t logm,
                       const uint8_t *m, size_t len, uint8_t *out) {
    field_init();
    transcript t; tr_init(&t, form, gate, n, d, logm);
    tr_absorb(&t, m, len);
    f_to_bytes(tr_squeeze(&t), out);
    return 0;
}

int zo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
