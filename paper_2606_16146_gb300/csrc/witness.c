/*
 * witness.c -- seeded synthetic ZeroCheck witnesses.
 *
 * Input generator shared by the tests, the benchmark and the oracle runs.
 * It draws uniform field elements from per-column splitmix64 streams
 * (Steele, Lea, Flood 2014; Vigna's published constants) and then sets the
 * one dependent column so that the gate vanishes at every point of the
 * domain, as the workload definition requires:
 *   Plonk   : columns qL,qR,qM,qO,qC,a,b,c ; c = -(qL a + qR b + qM a b + qC) / qO
 *   Product : columns q,w1..w_{d-1},o      ; o = q w1 ... w_{d-1}
 *   Sum     : columns g_1..g_{d+m}          ; g_{d+m} = -(g_1 ... g_d + g_{d+1} + ... + g_{d+m-1})
 *             for m >= 1; for m = 0 (f = g_1 ... g_d) every point zeroes one
 *             factor, chosen uniformly by the stream seeded with
 *             seed ^ 0xD1B54A32D192ED03.
 * Column j draws from a stream seeded with seed ^ (0x9E3779B97F4A7C15 (j+1)).
 * Each draw takes four 64-bit outputs as a little-endian 256-bit integer,
 * clears bit 255 and is kept if it is below r (rejection sampling).
 * Values are written canonical, 32 bytes little-endian per element.
 *
 * zw_generate_edge draws instead from a list of boundary values of the field
 * (0, 1, 2, r-1, r-2, r - 2^k, 2^k, 2^256 mod r and its square, (r +- 1)/2,
 * all-ones limbs below r, ...) mixed with uniform draws; no column is solved,
 * so the gate does not vanish.  The provers' bytes are defined for any
 * canonical input, and such columns push values next to the modulus and
 * zero limbs through every carry and conditional subtraction.
 *
 * Its modular arithmetic (a small Montgomery multiplier over 64-bit words)
 * exists only to construct satisfying inputs; it is not the prover's.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

typedef unsigned __int128 u128;
typedef struct { uint64_t v[4]; } el;

static const el MODULUS = {{0xffffffff00000001ULL, 0x53bda402fffe5bfeULL,
                            0x3339d80809a1d805ULL, 0x73eda753299d7d48ULL}};

static int below_mod(const el *a) {
    for (int i = 3; i >= 0; i--) {
        if (a->v[i] != MODULUS.v[i]) return a->v[i] < MODULUS.v[i];
    }
    return 0;
}

static el addm(el a, el b) {
    el s; u128 c = 0;
    for (int i = 0; i < 4; i++) { c += (u128)a.v[i] + b.v[i]; s.v[i] = (uint64_t)c; c >>= 64; }
    if (!below_mod(&s)) {
        u128 br = 0;
        for (int i = 0; i < 4; i++) {
            u128 t = (u128)s.v[i] - MODULUS.v[i] - br;
            s.v[i] = (uint64_t)t; br = (t >> 127) & 1;
        }
    }
    return s;
}

static el negm(el a) {
    if ((a.v[0] | a.v[1] | a.v[2] | a.v[3]) == 0) return a;
    el s; u128 br = 0;
    for (int i = 0; i < 4; i++) {
        u128 t = (u128)MODULUS.v[i] - a.v[i] - br;
        s.v[i] = (uint64_t)t; br = (t >> 127) & 1;
    }
    return s;
}

/* Montgomery product over 64-bit words (separated operand scanning). */
static uint64_t MINV;
static el RR;            /* 2^512 mod r */
static el ONE_M;         /* 2^256 mod r */

static el montmul(el a, el b) {
    uint64_t t[9] = {0};
    for (int i = 0; i < 4; i++) {            /* full 512-bit product */
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)a.v[i] * b.v[j] + t[i + j];
            t[i + j] = (uint64_t)c; c >>= 64;
        }
        t[i + 4] = (uint64_t)c;
    }
    for (int i = 0; i < 4; i++) {            /* word-by-word reduction */
        uint64_t m = t[i] * MINV;
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)m * MODULUS.v[j] + t[i + j];
            t[i + j] = (uint64_t)c; c >>= 64;
        }
        for (int k = i + 4; k < 9 && c; k++) { c += t[k]; t[k] = (uint64_t)c; c >>= 64; }
    }
    el s; memcpy(s.v, t + 4, 32);
    if (t[8] || !below_mod(&s)) {
        u128 br = 0;
        for (int i = 0; i < 4; i++) {
            u128 x = (u128)s.v[i] - MODULUS.v[i] - br;
            s.v[i] = (uint64_t)x; br = (x >> 127) & 1;
        }
    }
    return s;
}

static void setup(void) {
    static int done = 0;
    if (done) return;
    uint64_t x = 1;                           /* r^{-1} mod 2^64, Newton */
    for (int i = 0; i < 6; i++) x *= 2 - MODULUS.v[0] * x;
    MINV = (uint64_t)0 - x;
    el y = {{1, 0, 0, 0}};
    for (int i = 1; i <= 512; i++) { y = addm(y, y); if (i == 256) ONE_M = y; }
    RR = y;
    done = 1;
}

static el to_m(el a) { return montmul(a, RR); }
static el from_m(el a) { el one = {{1, 0, 0, 0}}; return montmul(a, one); }

static el inv_m(el a) {                       /* a^(r-2), Montgomery in/out */
    el e = MODULUS; e.v[0] -= 2;
    el acc = ONE_M;
    for (int i = 3; i >= 0; i--)
        for (int b = 63; b >= 0; b--) {
            acc = montmul(acc, acc);
            if ((e.v[i] >> b) & 1) acc = montmul(acc, a);
        }
    return acc;
}

static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static el draw(uint64_t *s, int nonzero) {
    for (;;) {
        el a;
        for (int i = 0; i < 4; i++) a.v[i] = splitmix64(s);
        a.v[3] &= 0x7fffffffffffffffULL;
        if (!below_mod(&a)) continue;
        if (nonzero && (a.v[0] | a.v[1] | a.v[2] | a.v[3]) == 0) continue;
        return a;
    }
}

static void put(uint8_t *dst, el a) {
    for (int i = 0; i < 4; i++)
        for (int k = 0; k < 8; k++) dst[8 * i + k] = (uint8_t)(a.v[i] >> (8 * k));
}

static el get(const uint8_t *src) {
    el a;
    for (int i = 0; i < 4; i++) {
        uint64_t w = 0;
        for (int k = 7; k >= 0; k--) w = (w << 8) | src[8 * i + k];
        a.v[i] = w;
    }
    return a;
}

static void fill_uniform(uint8_t *col, size_t N, uint64_t seed, int j, int nonzero) {
    uint64_t s = seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(j + 1));
    for (size_t k = 0; k < N; k++) put(col + 32 * k, draw(&s, nonzero));
}

/* gate 1 = Plonk (d must be 3), gate 2 = product (d >= 2), gate 3 | m << 8 =
 * sum of one d-fold product and m single columns.  cols[j] holds N*32 bytes.
 * tamper != 0 adds 1 to column a (Plonk), w1 (product) or the solved last
 * column (sum gate, m >= 1), or sets the zeroed factor to 1 (m = 0), at
 * index seed mod N afterwards.  Returns 0 on success. */
int zw_generate(uint32_t gate, uint32_t n, uint32_t d, uint64_t seed, int tamper, uint8_t *const *cols) {
    setup();
    size_t N = (size_t)1 << n;
    if (gate == 1) {
        if (d != 3) return 1;
        for (int j = 0; j < 7; j++) fill_uniform(cols[j], N, seed, j, j == 3);
        el *den = (el *)malloc(N * sizeof(el)), *pre = (el *)malloc(N * sizeof(el));
        if (!den || !pre) { free(den); free(pre); return 2; }
        el acc = ONE_M;                        /* batch inversion of qO */
        for (size_t k = 0; k < N; k++) {
            den[k] = to_m(get(cols[3] + 32 * k));
            pre[k] = acc; acc = montmul(acc, den[k]);
        }
        el inv = inv_m(acc);
        for (size_t k = N; k-- > 0;) {
            el t = montmul(inv, pre[k]);
            inv = montmul(inv, den[k]);
            den[k] = t;
        }
        free(pre);
        #pragma omp parallel for schedule(static)
        for (long kk = 0; kk < (long)N; kk++) {
            size_t k = (size_t)kk;
            el qL = to_m(get(cols[0] + 32 * k)), qR = to_m(get(cols[1] + 32 * k));
            el qM = to_m(get(cols[2] + 32 * k)), qC = to_m(get(cols[4] + 32 * k));
            el a = to_m(get(cols[5] + 32 * k)), b = to_m(get(cols[6] + 32 * k));
            el s = addm(addm(montmul(qL, a), montmul(qR, b)), addm(montmul(montmul(qM, a), b), qC));
            put(cols[7] + 32 * k, from_m(montmul(negm(s), den[k])));
        }
        free(den);
        if (tamper) {
            size_t k = (size_t)(seed % N);
            el one = {{1, 0, 0, 0}};
            put(cols[5] + 32 * k, addm(get(cols[5] + 32 * k), one));
        }
        return 0;
    }
    if (gate == 2) {
        if (d < 2 || d > 64) return 1;
        for (uint32_t j = 0; j < d; j++) fill_uniform(cols[j], N, seed, (int)j, 0);
        #pragma omp parallel for schedule(static)
        for (long kk = 0; kk < (long)N; kk++) {
            size_t k = (size_t)kk;
            el p = to_m(get(cols[0] + 32 * k));
            for (uint32_t j = 1; j < d; j++) p = montmul(p, to_m(get(cols[j] + 32 * k)));
            put(cols[d] + 32 * k, from_m(p));
        }
        if (tamper) {
            size_t k = (size_t)(seed % N);
            el one = {{1, 0, 0, 0}};
            put(cols[1] + 32 * k, addm(get(cols[1] + 32 * k), one));
        }
        return 0;
    }
    if ((gate & 0xff) == 3) {
        const uint32_t m = gate >> 8, c = d + m;
        if (d < 2 || d > 64 || m > 63 || c > 65) return 1;
        if (m == 0) {
            for (uint32_t j = 0; j < d; j++) fill_uniform(cols[j], N, seed, (int)j, 1);
            uint64_t s = seed ^ 0xD1B54A32D192ED03ULL;
            const el zero = {{0, 0, 0, 0}};
            for (size_t k = 0; k < N; k++) put(cols[splitmix64(&s) % d] + 32 * k, zero);
            if (tamper) {
                /* the zeroed factor of point seed mod N becomes 1 */
                size_t k0 = (size_t)(seed % N);
                uint64_t s2 = seed ^ 0xD1B54A32D192ED03ULL;
                uint32_t jz = 0;
                for (size_t k = 0; k <= k0; k++) jz = (uint32_t)(splitmix64(&s2) % d);
                const el one = {{1, 0, 0, 0}};
                put(cols[jz] + 32 * k0, one);
            }
            return 0;
        }
        for (uint32_t j = 0; j + 1 < c; j++) fill_uniform(cols[j], N, seed, (int)j, 0);
        #pragma omp parallel for schedule(static)
        for (long kk = 0; kk < (long)N; kk++) {
            size_t k = (size_t)kk;
            el p = to_m(get(cols[0] + 32 * k));
            for (uint32_t j = 1; j < d; j++) p = montmul(p, to_m(get(cols[j] + 32 * k)));
            el sum = from_m(p);
            for (uint32_t j = d; j + 1 < c; j++) sum = addm(sum, get(cols[j] + 32 * k));
            put(cols[c - 1] + 32 * k, negm(sum));
        }
        if (tamper) {
            size_t k = (size_t)(seed % N);
            el one = {{1, 0, 0, 0}};
            put(cols[c - 1] + 32 * k, addm(get(cols[c - 1] + 32 * k), one));
        }
        return 0;
    }
    return 1;
}

/* Boundary values of the field, canonical (each < r). */
static int edge_values(el *out) {
    const el one = {{1, 0, 0, 0}};
    int k = 0;
    el z = {{0, 0, 0, 0}};
    out[k++] = z;                                   /* 0 */
    out[k++] = one;                                 /* 1 */
    out[k++] = addm(one, one);                      /* 2 */
    el rm1 = negm(one);
    out[k++] = rm1;                                 /* r - 1 */
    out[k++] = addm(rm1, rm1);                      /* r - 2 */
    out[k++] = negm(addm(one, addm(one, one)));     /* r - 3 */
    const int sh[] = {31, 32, 63, 64, 127, 128, 191, 192, 224, 253, 254};
    for (unsigned t = 0; t < sizeof sh / sizeof sh[0]; t++) {
        el p2 = z;
        p2.v[sh[t] / 64] = 1ULL << (sh[t] % 64);    /* 2^k < r for k <= 254 */
        out[k++] = p2;                              /* 2^k */
        out[k++] = negm(p2);                        /* r - 2^k */
        el m1 = p2;                                 /* 2^k - 1: all-ones limbs */
        u128 br = 1;
        for (int i = 0; i < 4; i++) { u128 x = (u128)m1.v[i] - br; m1.v[i] = (uint64_t)x; br = (x >> 127) & 1; }
        out[k++] = m1;
    }
    out[k++] = ONE_M;                               /* 2^256 mod r (Montgomery one) */
    out[k++] = to_m(RR);                            /* 2^768 mod r */
    out[k++] = RR;                                  /* 2^512 mod r */
    out[k++] = negm(ONE_M);                         /* r - R */
    el half = MODULUS;                              /* (r - 1) / 2 */
    for (int i = 0; i < 4; i++) half.v[i] = (MODULUS.v[i] >> 1) | (i < 3 ? MODULUS.v[i + 1] << 63 : 0);
    out[k++] = half;
    out[k++] = addm(half, one);                     /* (r + 1) / 2 */
    el top = MODULUS;                               /* r with its low limb cleared: < r */
    top.v[0] = 0;
    out[k++] = top;
    el lowmax = {{~0ULL, ~0ULL, ~0ULL, 0}};         /* 2^192 - 1 */
    out[k++] = lowmax;
    el lim = MODULUS;                               /* limbs of r - 1 with the top limb one less */
    lim.v[0] -= 1;
    lim.v[3] -= 1;
    out[k++] = lim;
    return k;
}

/* Columns of boundary values (see the header).  only_edges != 0 draws every
 * element from the boundary list, else half of them (per element) are
 * uniform.  Column j uses the stream seed ^ (0x9E3779B97F4A7C15 (j+1)), as
 * zw_generate does.  Returns 0 on success. */
int zw_generate_edge(uint32_t gate, uint32_t n, uint32_t d, uint64_t seed, int only_edges,
                     uint8_t *const *cols) {
    setup();
    int c;
    if (gate == 1) { if (d != 3) return 1; c = 8; }
    else if (gate == 2) { if (d < 2 || d > 64) return 1; c = (int)d + 1; }
    else if ((gate & 0xff) == 3) {
        const uint32_t m = gate >> 8;
        if (d < 2 || d > 64 || m > 63 || d + m > 65) return 1;
        c = (int)(d + m);
    } else return 1;
    el edges[64];
    const int ne = edge_values(edges);
    size_t N = (size_t)1 << n;
    for (int j = 0; j < c; j++) {
        uint64_t s = seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(j + 1));
        for (size_t k = 0; k < N; k++) {
            const uint64_t pick = splitmix64(&s);
            if (!only_edges && (pick & 1)) put(cols[j] + 32 * k, draw(&s, 0));
            else put(cols[j] + 32 * k, edges[(pick >> 1) % (uint64_t)ne]);
        }
    }
    return 0;
}
