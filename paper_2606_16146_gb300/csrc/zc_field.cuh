// zc_field.cuh -- arithmetic in the BLS12-381 scalar field r on sm_103a.
//
// Elements are 8 x 32-bit little-endian limbs (32 bytes).  The device
// multiplier is a CIOS Montgomery product (Koc, Acar, Kaliski 1996) written
// as PTX carry chains (mad.lo.cc / madc.hi.cc) on the integer pipe; r's low
// limb is 1, so -r^{-1} mod 2^32 = 0xffffffff and the per-row quotient digit
// is just the negated low word.  r < 2^255 keeps every intermediate of a row
// inside nine words.
//
// "Level" bookkeeping: a Montgomery product of values x (stored as x R^i)
// and y (stored as y R^j) returns x y R^(i+j-1).  Canonical storage is level
// 0, the usual Montgomery form level 1.  The provers keep tables at whatever
// level makes the gate need no conversions and fold the R powers into
// per-proof constants.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define ZC_HD __host__ __device__ __forceinline__
#define ZC_D __device__ __forceinline__
#else
#define ZC_HD inline
#define ZC_D inline
#endif

namespace zc {

struct fr {
  uint32_t v[8];
};

// r = 0x73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001
#define ZC_P0 0x00000001u
#define ZC_P1 0xffffffffu
#define ZC_P2 0xfffe5bfeu
#define ZC_P3 0x53bda402u
#define ZC_P4 0x09a1d805u
#define ZC_P5 0x3339d808u
#define ZC_P6 0x299d7d48u
#define ZC_P7 0x73eda753u

// limb i of r (i is a compile-time constant after unrolling)
ZC_HD uint32_t p_limb(int i) {
  switch (i) {
    case 0: return ZC_P0;
    case 1: return ZC_P1;
    case 2: return ZC_P2;
    case 3: return ZC_P3;
    case 4: return ZC_P4;
    case 5: return ZC_P5;
    case 6: return ZC_P6;
    default: return ZC_P7;
  }
}

ZC_HD fr fr_zero() {
  fr z;
  for (int i = 0; i < 8; i++) z.v[i] = 0;
  return z;
}

ZC_HD bool fr_is_zero(const fr& a) {
  uint32_t x = 0;
  for (int i = 0; i < 8; i++) x |= a.v[i];
  return x == 0;
}

ZC_HD bool fr_equal(const fr& a, const fr& b) {
  uint32_t x = 0;
  for (int i = 0; i < 8; i++) x |= a.v[i] ^ b.v[i];
  return x == 0;
}

// a < r as an integer (canonical check)
ZC_HD bool fr_is_canonical(const fr& a) {
  const uint32_t P[8] = {ZC_P0, ZC_P1, ZC_P2, ZC_P3, ZC_P4, ZC_P5, ZC_P6, ZC_P7};
  for (int i = 7; i >= 0; i--) {
    if (a.v[i] != P[i]) return a.v[i] < P[i];
  }
  return false;
}

// ---------------------------------------------------------------- generic --
// Portable versions (host verifier, set-up constants).  64-bit intermediates.

ZC_HD fr fr_add_g(const fr& a, const fr& b) {
  const uint32_t P[8] = {ZC_P0, ZC_P1, ZC_P2, ZC_P3, ZC_P4, ZC_P5, ZC_P6, ZC_P7};
  fr s, t;
  uint64_t c = 0;
  for (int i = 0; i < 8; i++) {
    c += (uint64_t)a.v[i] + b.v[i];
    s.v[i] = (uint32_t)c;
    c >>= 32;
  }
  int64_t br = 0;
  for (int i = 0; i < 8; i++) {
    int64_t d = (int64_t)s.v[i] - P[i] + br;
    t.v[i] = (uint32_t)d;
    br = d >> 32;  // 0 or -1
  }
  return (c == 0 && br < 0) ? s : t;
}

ZC_HD fr fr_sub_g(const fr& a, const fr& b) {
  const uint32_t P[8] = {ZC_P0, ZC_P1, ZC_P2, ZC_P3, ZC_P4, ZC_P5, ZC_P6, ZC_P7};
  fr s;
  int64_t br = 0;
  for (int i = 0; i < 8; i++) {
    int64_t d = (int64_t)a.v[i] - b.v[i] + br;
    s.v[i] = (uint32_t)d;
    br = d >> 32;
  }
  if (br < 0) {
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) {
      c += (uint64_t)s.v[i] + P[i];
      s.v[i] = (uint32_t)c;
      c >>= 32;
    }
  }
  return s;
}

// Montgomery product a b 2^-256 mod r, inputs < r, output < r.
ZC_HD fr fr_mul_g(const fr& a, const fr& b) {
  const uint32_t P[8] = {ZC_P0, ZC_P1, ZC_P2, ZC_P3, ZC_P4, ZC_P5, ZC_P6, ZC_P7};
  uint32_t t[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 8; i++) {
    uint64_t c = 0;
    for (int j = 0; j < 8; j++) {
      c += (uint64_t)a.v[j] * b.v[i] + t[j];
      t[j] = (uint32_t)c;
      c >>= 32;
    }
    c += t[8];
    t[8] = (uint32_t)c;
    t[9] = (uint32_t)(c >> 32);
    uint32_t m = 0u - t[0];  // t0 * (-r^{-1}) mod 2^32, r0 = 1
    c = (uint64_t)m * P[0] + t[0];
    c >>= 32;
    for (int j = 1; j < 8; j++) {
      c += (uint64_t)m * P[j] + t[j];
      t[j - 1] = (uint32_t)c;
      c >>= 32;
    }
    c += t[8];
    t[7] = (uint32_t)c;
    t[8] = t[9] + (uint32_t)(c >> 32);
  }
  fr r;
  for (int i = 0; i < 8; i++) r.v[i] = t[i];
  if (t[8] != 0 || !fr_is_canonical(r)) {
    int64_t br = 0;
    for (int i = 0; i < 8; i++) {
      int64_t d = (int64_t)r.v[i] - P[i] + br;
      r.v[i] = (uint32_t)d;
      br = d >> 32;
    }
  }
  return r;
}

// ---------------------------------------------------------------- device --
#if defined(__CUDACC__)

ZC_D fr fr_add(const fr& a, const fr& b) {
  fr s, t;
  uint32_t bw;
  asm("add.cc.u32 %0, %8, %16;\n\t"
      "addc.cc.u32 %1, %9, %17;\n\t"
      "addc.cc.u32 %2, %10, %18;\n\t"
      "addc.cc.u32 %3, %11, %19;\n\t"
      "addc.cc.u32 %4, %12, %20;\n\t"
      "addc.cc.u32 %5, %13, %21;\n\t"
      "addc.cc.u32 %6, %14, %22;\n\t"
      "addc.u32 %7, %15, %23;"
      : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
        "=r"(s.v[6]), "=r"(s.v[7])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
        "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
        "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
  asm("sub.cc.u32 %0, %9, %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32 %8, 0, 0;"
      : "=r"(t.v[0]), "=r"(t.v[1]), "=r"(t.v[2]), "=r"(t.v[3]), "=r"(t.v[4]), "=r"(t.v[5]),
        "=r"(t.v[6]), "=r"(t.v[7]), "=r"(bw)
      : "r"(s.v[0]), "r"(s.v[1]), "r"(s.v[2]), "r"(s.v[3]), "r"(s.v[4]), "r"(s.v[5]),
        "r"(s.v[6]), "r"(s.v[7]), "n"(ZC_P0), "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4),
        "n"(ZC_P5), "n"(ZC_P6), "n"(ZC_P7));
  // bw == 0xffffffff: s < r, keep s
#pragma unroll
  for (int i = 0; i < 8; i++) s.v[i] = bw ? s.v[i] : t.v[i];
  return s;
}

// Lazily reduced sum and difference of canonical a, b: results in [0, 2r)
// (2r < 2^256) without the conditional correction.  Such a value may be the
// SECOND operand of fr_mul: its rows run over b's limbs with a < r, so every
// row stays below 2r + 1 and the product below 2r before its final
// subtraction, whatever b < 2^256 is.  fr_reduce1 brings it to [0, r).
ZC_D fr fr_add_lazy(const fr& a, const fr& b) {
  fr s;
  asm("add.cc.u32 %0, %8, %16;\n\t"
      "addc.cc.u32 %1, %9, %17;\n\t"
      "addc.cc.u32 %2, %10, %18;\n\t"
      "addc.cc.u32 %3, %11, %19;\n\t"
      "addc.cc.u32 %4, %12, %20;\n\t"
      "addc.cc.u32 %5, %13, %21;\n\t"
      "addc.cc.u32 %6, %14, %22;\n\t"
      "addc.u32 %7, %15, %23;"
      : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
        "=r"(s.v[6]), "=r"(s.v[7])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
        "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
        "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
  return s;
}

// a - b + r mod 2^256, in (0, 2r) for canonical a, b
ZC_D fr fr_sub_lazy(const fr& a, const fr& b) {
  fr s;
  asm("sub.cc.u32 %0, %8, %16;\n\t"
      "subc.cc.u32 %1, %9, %17;\n\t"
      "subc.cc.u32 %2, %10, %18;\n\t"
      "subc.cc.u32 %3, %11, %19;\n\t"
      "subc.cc.u32 %4, %12, %20;\n\t"
      "subc.cc.u32 %5, %13, %21;\n\t"
      "subc.cc.u32 %6, %14, %22;\n\t"
      "subc.u32 %7, %15, %23;"
      : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
        "=r"(s.v[6]), "=r"(s.v[7])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
        "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
        "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
  asm("add.cc.u32 %0, %0, %8;\n\t"
      "addc.cc.u32 %1, %1, %9;\n\t"
      "addc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\t"
      "addc.cc.u32 %4, %4, %12;\n\t"
      "addc.cc.u32 %5, %5, %13;\n\t"
      "addc.cc.u32 %6, %6, %14;\n\t"
      "addc.u32 %7, %7, %15;"
      : "+r"(s.v[0]), "+r"(s.v[1]), "+r"(s.v[2]), "+r"(s.v[3]), "+r"(s.v[4]), "+r"(s.v[5]),
        "+r"(s.v[6]), "+r"(s.v[7])
      : "n"(ZC_P0), "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4), "n"(ZC_P5), "n"(ZC_P6),
        "n"(ZC_P7));
  return s;
}

// x - r when x >= r, for x < 2r
ZC_D fr fr_reduce1(const fr& x) {
  fr t;
  uint32_t bw;
  asm("sub.cc.u32 %0, %9, %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32 %8, 0, 0;"
      : "=r"(t.v[0]), "=r"(t.v[1]), "=r"(t.v[2]), "=r"(t.v[3]), "=r"(t.v[4]), "=r"(t.v[5]),
        "=r"(t.v[6]), "=r"(t.v[7]), "=r"(bw)
      : "r"(x.v[0]), "r"(x.v[1]), "r"(x.v[2]), "r"(x.v[3]), "r"(x.v[4]), "r"(x.v[5]),
        "r"(x.v[6]), "r"(x.v[7]), "n"(ZC_P0), "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4),
        "n"(ZC_P5), "n"(ZC_P6), "n"(ZC_P7));
  fr r;
#pragma unroll
  for (int i = 0; i < 8; i++) r.v[i] = bw ? x.v[i] : t.v[i];
  return r;
}

ZC_D fr fr_sub(const fr& a, const fr& b) {
  fr s;
  uint32_t bw;
  asm("sub.cc.u32 %0, %9, %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32 %8, 0, 0;"
      : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
        "=r"(s.v[6]), "=r"(s.v[7]), "=r"(bw)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
        "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
        "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
  asm("add.cc.u32 %0, %0, %8;\n\t"
      "addc.cc.u32 %1, %1, %9;\n\t"
      "addc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\t"
      "addc.cc.u32 %4, %4, %12;\n\t"
      "addc.cc.u32 %5, %5, %13;\n\t"
      "addc.cc.u32 %6, %6, %14;\n\t"
      "addc.u32 %7, %7, %15;"
      : "+r"(s.v[0]), "+r"(s.v[1]), "+r"(s.v[2]), "+r"(s.v[3]), "+r"(s.v[4]), "+r"(s.v[5]),
        "+r"(s.v[6]), "+r"(s.v[7])
      : "r"(bw & ZC_P0), "r"(bw & ZC_P1), "r"(bw & ZC_P2), "r"(bw & ZC_P3), "r"(bw & ZC_P4),
        "r"(bw & ZC_P5), "r"(bw & ZC_P6), "r"(bw & ZC_P7));
  return s;
}

// One CIOS row: t += a * b; then t += m r with m = -t0, and shift one word.
// t holds nine words; t8 is zero on entry and becomes the new top word.
#define ZC_ROW(B)                                                                        \
  asm("mad.lo.cc.u32 %0, %9, %17, %0;\n\t"                                               \
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"                                             \
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"                                             \
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"                                             \
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"                                             \
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"                                             \
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"                                             \
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"                                             \
      "addc.u32 %8, 0, 0;\n\t"                                                           \
      "mad.hi.cc.u32 %1, %9, %17, %1;\n\t"                                               \
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"                                             \
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"                                             \
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"                                             \
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"                                             \
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"                                             \
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"                                             \
      "madc.hi.u32 %8, %16, %17, %8;"                                                    \
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), \
        "+r"(t8)                                                                         \
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),    \
        "r"(a.v[6]), "r"(a.v[7]), "r"(B));                                               \
  {                                                                                      \
    uint32_t m = 0u - t0;                                                                \
    asm("add.cc.u32 %0, %0, %9;\n\t"                                                     \
        "madc.lo.cc.u32 %1, %9, %10, %1;\n\t"                                            \
        "madc.lo.cc.u32 %2, %9, %11, %2;\n\t"                                            \
        "madc.lo.cc.u32 %3, %9, %12, %3;\n\t"                                            \
        "madc.lo.cc.u32 %4, %9, %13, %4;\n\t"                                            \
        "madc.lo.cc.u32 %5, %9, %14, %5;\n\t"                                            \
        "madc.lo.cc.u32 %6, %9, %15, %6;\n\t"                                            \
        "madc.lo.cc.u32 %7, %9, %16, %7;\n\t"                                            \
        "addc.u32 %8, %8, 0;\n\t"                                                        \
        "mad.hi.cc.u32 %2, %9, %10, %2;\n\t"                                             \
        "madc.hi.cc.u32 %3, %9, %11, %3;\n\t"                                            \
        "madc.hi.cc.u32 %4, %9, %12, %4;\n\t"                                            \
        "madc.hi.cc.u32 %5, %9, %13, %5;\n\t"                                            \
        "madc.hi.cc.u32 %6, %9, %14, %6;\n\t"                                            \
        "madc.hi.cc.u32 %7, %9, %15, %7;\n\t"                                            \
        "madc.hi.u32 %8, %9, %16, %8;"                                                   \
        : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), \
          "+r"(t8)                                                                       \
        : "r"(m), "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4), "n"(ZC_P5), "n"(ZC_P6), \
          "n"(ZC_P7));                                                                   \
  }                                                                                      \
  t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8; t8 = 0;

// In the reduction asm, %9 is m and %10..%16 are r1..r7; r0 = 1 turns its
// low product into a plain add and its high product into zero.

ZC_D fr fr_reduce_final(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, uint32_t t4,
                        uint32_t t5, uint32_t t6, uint32_t t7) {
  fr s, r;
  uint32_t bw;
  asm("sub.cc.u32 %0, %9, %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32 %8, 0, 0;"
      : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
        "=r"(s.v[6]), "=r"(s.v[7]), "=r"(bw)
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7), "n"(ZC_P0),
        "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4), "n"(ZC_P5), "n"(ZC_P6), "n"(ZC_P7));
  r.v[0] = bw ? t0 : s.v[0];
  r.v[1] = bw ? t1 : s.v[1];
  r.v[2] = bw ? t2 : s.v[2];
  r.v[3] = bw ? t3 : s.v[3];
  r.v[4] = bw ? t4 : s.v[4];
  r.v[5] = bw ? t5 : s.v[5];
  r.v[6] = bw ? t6 : s.v[6];
  r.v[7] = bw ? t7 : s.v[7];
  return r;
}

// Carry-chain variant (mad.lo.cc / madc.hi.cc), kept for comparison.
ZC_D fr fr_mul_cc(const fr& a, const fr& b) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0;
  ZC_ROW(b.v[0])
  ZC_ROW(b.v[1])
  ZC_ROW(b.v[2])
  ZC_ROW(b.v[3])
  ZC_ROW(b.v[4])
  ZC_ROW(b.v[5])
  ZC_ROW(b.v[6])
  ZC_ROW(b.v[7])
  return fr_reduce_final(t0, t1, t2, t3, t4, t5, t6, t7);
}

// CIOS with 64-bit partial products (mul.wide.u32, IMAD.WIDE on the integer
// pipe).  Each row forms the eight products q_j = a_j b_i as 64-bit values
// with no addend (an addend pair costs extra register moves on the same
// pipe), joins lo(q_j) with hi(q_{j-1}) in one add-with-carry chain and adds
// that to t in a second chain on the ALU pipe.  The reduction row does the
// same with m r_j; r_0 = 1 and r_1 = 2^32 - 1 need no multiplication
// (m (2^32 - 1) has low word -m = t_0 and high word m - [m != 0]).
#define ZC_LO(x) ((uint32_t)(x))
#define ZC_HI(x) ((uint32_t)((x) >> 32))

ZC_D void zc_row_wide(const fr& a, uint32_t bi, uint32_t& t0, uint32_t& t1, uint32_t& t2,
                      uint32_t& t3, uint32_t& t4, uint32_t& t5, uint32_t& t6, uint32_t& t7) {
  uint64_t q0, q1, q2, q3, q4, q5, q6, q7;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q0) : "r"(a.v[0]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q1) : "r"(a.v[1]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q2) : "r"(a.v[2]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q3) : "r"(a.v[3]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q4) : "r"(a.v[4]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q5) : "r"(a.v[5]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q6) : "r"(a.v[6]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q7) : "r"(a.v[7]), "r"(bi));
  uint32_t s1, s2, s3, s4, s5, s6, s7, s8;
  asm("add.cc.u32 %0, %8, %9;\n\t"
      "addc.cc.u32 %1, %10, %11;\n\t"
      "addc.cc.u32 %2, %12, %13;\n\t"
      "addc.cc.u32 %3, %14, %15;\n\t"
      "addc.cc.u32 %4, %16, %17;\n\t"
      "addc.cc.u32 %5, %18, %19;\n\t"
      "addc.cc.u32 %6, %20, %21;\n\t"
      "addc.u32 %7, %22, 0;"
      : "=r"(s1), "=r"(s2), "=r"(s3), "=r"(s4), "=r"(s5), "=r"(s6), "=r"(s7), "=r"(s8)
      : "r"(ZC_LO(q1)), "r"(ZC_HI(q0)), "r"(ZC_LO(q2)), "r"(ZC_HI(q1)), "r"(ZC_LO(q3)),
        "r"(ZC_HI(q2)), "r"(ZC_LO(q4)), "r"(ZC_HI(q3)), "r"(ZC_LO(q5)), "r"(ZC_HI(q4)),
        "r"(ZC_LO(q6)), "r"(ZC_HI(q5)), "r"(ZC_LO(q7)), "r"(ZC_HI(q6)), "r"(ZC_HI(q7)));
  uint32_t u0, u1, u2, u3, u4, u5, u6, u7, u8;
  asm("add.cc.u32 %0, %9, %17;\n\t"
      "addc.cc.u32 %1, %10, %18;\n\t"
      "addc.cc.u32 %2, %11, %19;\n\t"
      "addc.cc.u32 %3, %12, %20;\n\t"
      "addc.cc.u32 %4, %13, %21;\n\t"
      "addc.cc.u32 %5, %14, %22;\n\t"
      "addc.cc.u32 %6, %15, %23;\n\t"
      "addc.cc.u32 %7, %16, %24;\n\t"
      "addc.u32 %8, %25, 0;"
      : "=r"(u0), "=r"(u1), "=r"(u2), "=r"(u3), "=r"(u4), "=r"(u5), "=r"(u6), "=r"(u7), "=r"(u8)
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7), "r"(ZC_LO(q0)),
        "r"(s1), "r"(s2), "r"(s3), "r"(s4), "r"(s5), "r"(s6), "r"(s7), "r"(s8));
  // reduction: m = -u0 (r0 = 1), add m r, drop the zero low word
  const uint32_t m = 0u - u0, c0 = u0 != 0 ? 1u : 0u;
  const uint32_t r1lo = u0, r1hi = m - c0;  // m (2^32 - 1)
  uint64_t r2, r3, r4, r5, r6, r7;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r2) : "r"(m), "n"(ZC_P2));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r3) : "r"(m), "n"(ZC_P3));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r4) : "r"(m), "n"(ZC_P4));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r5) : "r"(m), "n"(ZC_P5));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r6) : "r"(m), "n"(ZC_P6));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r7) : "r"(m), "n"(ZC_P7));
  uint32_t v1, v2, v3, v4, v5, v6, v7, v8;
  asm("add.cc.u32 %0, %8, %9;\n\t"
      "addc.cc.u32 %1, %10, %11;\n\t"
      "addc.cc.u32 %2, %12, %13;\n\t"
      "addc.cc.u32 %3, %14, %15;\n\t"
      "addc.cc.u32 %4, %16, %17;\n\t"
      "addc.cc.u32 %5, %18, %19;\n\t"
      "addc.cc.u32 %6, %20, %21;\n\t"
      "addc.u32 %7, %22, 0;"
      : "=r"(v1), "=r"(v2), "=r"(v3), "=r"(v4), "=r"(v5), "=r"(v6), "=r"(v7), "=r"(v8)
      : "r"(r1lo), "r"(c0), "r"(ZC_LO(r2)), "r"(r1hi), "r"(ZC_LO(r3)), "r"(ZC_HI(r2)),
        "r"(ZC_LO(r4)), "r"(ZC_HI(r3)), "r"(ZC_LO(r5)), "r"(ZC_HI(r4)), "r"(ZC_LO(r6)),
        "r"(ZC_HI(r5)), "r"(ZC_LO(r7)), "r"(ZC_HI(r6)), "r"(ZC_HI(r7)));
  asm("add.cc.u32 %0, %8, %16;\n\t"
      "addc.cc.u32 %1, %9, %17;\n\t"
      "addc.cc.u32 %2, %10, %18;\n\t"
      "addc.cc.u32 %3, %11, %19;\n\t"
      "addc.cc.u32 %4, %12, %20;\n\t"
      "addc.cc.u32 %5, %13, %21;\n\t"
      "addc.cc.u32 %6, %14, %22;\n\t"
      "addc.u32 %7, %15, %23;"
      : "=r"(t0), "=r"(t1), "=r"(t2), "=r"(t3), "=r"(t4), "=r"(t5), "=r"(t6), "=r"(t7)
      : "r"(u1), "r"(u2), "r"(u3), "r"(u4), "r"(u5), "r"(u6), "r"(u7), "r"(u8), "r"(v1),
        "r"(v2), "r"(v3), "r"(v4), "r"(v5), "r"(v6), "r"(v7), "r"(v8));
}

ZC_D fr fr_mul_inl(const fr& a, const fr& b) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0;
  zc_row_wide(a, b.v[0], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[1], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[2], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[3], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[4], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[5], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[6], t0, t1, t2, t3, t4, t5, t6, t7);
  zc_row_wide(a, b.v[7], t0, t1, t2, t3, t4, t5, t6, t7);
  return fr_reduce_final(t0, t1, t2, t3, t4, t5, t6, t7);
}

// Sums of products with one reduction: (a0 b0 + ... + a_{K-1} b_{K-1}) R^-1
// mod r, for inputs below r, K = 2 or 3.  Each CIOS row adds a_p b_p[i] for
// every p into a 10-word accumulator, then one reduction step m r (m = -t0)
// and a one-word shift.  Between rows the accumulator stays below (K+1) r
// < 2^257 (nine words), before the shift below 2^289 (ten); at the end it is
// (sum a_p b_p + M r) / 2^256 < r (K r / 2^256 + 1) < 2.36 r for K = 3, so
// at most two subtractions of r give the canonical result.  Against K
// separate products and K - 1 additions this saves K - 1 reductions and the
// final corrections (~30 % fewer instructions for K = 3).

// t[0..9] += a * bi
ZC_D void zc_acc_row(const fr& a, uint32_t bi, uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t& t3,
                     uint32_t& t4, uint32_t& t5, uint32_t& t6, uint32_t& t7, uint32_t& t8, uint32_t& t9) {
  uint64_t q0, q1, q2, q3, q4, q5, q6, q7;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q0) : "r"(a.v[0]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q1) : "r"(a.v[1]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q2) : "r"(a.v[2]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q3) : "r"(a.v[3]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q4) : "r"(a.v[4]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q5) : "r"(a.v[5]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q6) : "r"(a.v[6]), "r"(bi));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(q7) : "r"(a.v[7]), "r"(bi));
  uint32_t s1, s2, s3, s4, s5, s6, s7, s8;
  asm("add.cc.u32 %0, %8, %9;\n\t"
      "addc.cc.u32 %1, %10, %11;\n\t"
      "addc.cc.u32 %2, %12, %13;\n\t"
      "addc.cc.u32 %3, %14, %15;\n\t"
      "addc.cc.u32 %4, %16, %17;\n\t"
      "addc.cc.u32 %5, %18, %19;\n\t"
      "addc.cc.u32 %6, %20, %21;\n\t"
      "addc.u32 %7, %22, 0;"
      : "=r"(s1), "=r"(s2), "=r"(s3), "=r"(s4), "=r"(s5), "=r"(s6), "=r"(s7), "=r"(s8)
      : "r"(ZC_LO(q1)), "r"(ZC_HI(q0)), "r"(ZC_LO(q2)), "r"(ZC_HI(q1)), "r"(ZC_LO(q3)),
        "r"(ZC_HI(q2)), "r"(ZC_LO(q4)), "r"(ZC_HI(q3)), "r"(ZC_LO(q5)), "r"(ZC_HI(q4)),
        "r"(ZC_LO(q6)), "r"(ZC_HI(q5)), "r"(ZC_LO(q7)), "r"(ZC_HI(q6)), "r"(ZC_HI(q7)));
  asm("add.cc.u32 %0, %0, %10;\n\t"
      "addc.cc.u32 %1, %1, %11;\n\t"
      "addc.cc.u32 %2, %2, %12;\n\t"
      "addc.cc.u32 %3, %3, %13;\n\t"
      "addc.cc.u32 %4, %4, %14;\n\t"
      "addc.cc.u32 %5, %5, %15;\n\t"
      "addc.cc.u32 %6, %6, %16;\n\t"
      "addc.cc.u32 %7, %7, %17;\n\t"
      "addc.cc.u32 %8, %8, %18;\n\t"
      "addc.u32 %9, %9, 0;"
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8), "+r"(t9)
      : "r"(ZC_LO(q0)), "r"(s1), "r"(s2), "r"(s3), "r"(s4), "r"(s5), "r"(s6), "r"(s7), "r"(s8));
}

// t <- (t + m r) / 2^32 with m = -t0 (r0 = 1, r1 = 2^32 - 1); t9 becomes 0
ZC_D void zc_reduce_row(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t& t3, uint32_t& t4, uint32_t& t5,
                        uint32_t& t6, uint32_t& t7, uint32_t& t8, uint32_t& t9) {
  const uint32_t m = 0u - t0, c0 = t0 != 0 ? 1u : 0u;
  const uint32_t r1lo = t0, r1hi = m - c0;  // m (2^32 - 1)
  uint64_t r2, r3, r4, r5, r6, r7;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r2) : "r"(m), "n"(ZC_P2));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r3) : "r"(m), "n"(ZC_P3));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r4) : "r"(m), "n"(ZC_P4));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r5) : "r"(m), "n"(ZC_P5));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r6) : "r"(m), "n"(ZC_P6));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r7) : "r"(m), "n"(ZC_P7));
  uint32_t v1, v2, v3, v4, v5, v6, v7, v8;
  asm("add.cc.u32 %0, %8, %9;\n\t"
      "addc.cc.u32 %1, %10, %11;\n\t"
      "addc.cc.u32 %2, %12, %13;\n\t"
      "addc.cc.u32 %3, %14, %15;\n\t"
      "addc.cc.u32 %4, %16, %17;\n\t"
      "addc.cc.u32 %5, %18, %19;\n\t"
      "addc.cc.u32 %6, %20, %21;\n\t"
      "addc.u32 %7, %22, 0;"
      : "=r"(v1), "=r"(v2), "=r"(v3), "=r"(v4), "=r"(v5), "=r"(v6), "=r"(v7), "=r"(v8)
      : "r"(r1lo), "r"(c0), "r"(ZC_LO(r2)), "r"(r1hi), "r"(ZC_LO(r3)), "r"(ZC_HI(r2)),
        "r"(ZC_LO(r4)), "r"(ZC_HI(r3)), "r"(ZC_LO(r5)), "r"(ZC_HI(r4)), "r"(ZC_LO(r6)),
        "r"(ZC_HI(r5)), "r"(ZC_LO(r7)), "r"(ZC_HI(r6)), "r"(ZC_HI(r7)));
  // t0 + (m r mod 2^32) = 0 with a carry exactly when t0 != 0 (c0 above);
  // the shifted sum goes to fresh registers
  uint32_t n0, n1, n2, n3, n4, n5, n6, n7, n8;
  asm("add.cc.u32 %0, %9, %18;\n\t"
      "addc.cc.u32 %1, %10, %19;\n\t"
      "addc.cc.u32 %2, %11, %20;\n\t"
      "addc.cc.u32 %3, %12, %21;\n\t"
      "addc.cc.u32 %4, %13, %22;\n\t"
      "addc.cc.u32 %5, %14, %23;\n\t"
      "addc.cc.u32 %6, %15, %24;\n\t"
      "addc.cc.u32 %7, %16, %25;\n\t"
      "addc.u32 %8, %17, 0;"
      : "=r"(n0), "=r"(n1), "=r"(n2), "=r"(n3), "=r"(n4), "=r"(n5), "=r"(n6), "=r"(n7), "=r"(n8)
      : "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7), "r"(t8), "r"(t9), "r"(v1),
        "r"(v2), "r"(v3), "r"(v4), "r"(v5), "r"(v6), "r"(v7), "r"(v8));
  t0 = n0; t1 = n1; t2 = n2; t3 = n3; t4 = n4; t5 = n5; t6 = n6; t7 = n7; t8 = n8;
  t9 = 0;
}

// t (nine words, below 3r) minus r when it is at least r
ZC_D void zc_sub_r_if(uint32_t& t0, uint32_t& t1, uint32_t& t2, uint32_t& t3, uint32_t& t4, uint32_t& t5,
                      uint32_t& t6, uint32_t& t7, uint32_t& t8) {
  uint32_t s0, s1, s2, s3, s4, s5, s6, s7, s8, bw;
  asm("sub.cc.u32 %0, %10, %19;\n\t"
      "subc.cc.u32 %1, %11, %20;\n\t"
      "subc.cc.u32 %2, %12, %21;\n\t"
      "subc.cc.u32 %3, %13, %22;\n\t"
      "subc.cc.u32 %4, %14, %23;\n\t"
      "subc.cc.u32 %5, %15, %24;\n\t"
      "subc.cc.u32 %6, %16, %25;\n\t"
      "subc.cc.u32 %7, %17, %26;\n\t"
      "subc.cc.u32 %8, %18, 0;\n\t"
      "subc.u32 %9, 0, 0;"
      : "=r"(s0), "=r"(s1), "=r"(s2), "=r"(s3), "=r"(s4), "=r"(s5), "=r"(s6), "=r"(s7), "=r"(s8), "=r"(bw)
      : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4), "r"(t5), "r"(t6), "r"(t7), "r"(t8), "n"(ZC_P0),
        "n"(ZC_P1), "n"(ZC_P2), "n"(ZC_P3), "n"(ZC_P4), "n"(ZC_P5), "n"(ZC_P6), "n"(ZC_P7));
  // bw == 0xffffffff: t < r, keep it
  t0 = bw ? t0 : s0; t1 = bw ? t1 : s1; t2 = bw ? t2 : s2; t3 = bw ? t3 : s3; t4 = bw ? t4 : s4;
  t5 = bw ? t5 : s5; t6 = bw ? t6 : s6; t7 = bw ? t7 : s7; t8 = bw ? t8 : s8;
}

template <int K>
ZC_D fr fr_mul_sum_inl(const fr (&a)[K], const fr (&b)[K]) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8 = 0, t9 = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
#pragma unroll
    for (int p = 0; p < K; p++) zc_acc_row(a[p], b[p].v[i], t0, t1, t2, t3, t4, t5, t6, t7, t8, t9);
    zc_reduce_row(t0, t1, t2, t3, t4, t5, t6, t7, t8, t9);
  }
  zc_sub_r_if(t0, t1, t2, t3, t4, t5, t6, t7, t8);
  if (K > 2) zc_sub_r_if(t0, t1, t2, t3, t4, t5, t6, t7, t8);
  fr x;
  x.v[0] = t0; x.v[1] = t1; x.v[2] = t2; x.v[3] = t3; x.v[4] = t4; x.v[5] = t5; x.v[6] = t6; x.v[7] = t7;
  return x;
}

// out-of-line copy shared by the kernels (see fr_mul_call)
static __device__ __noinline__ fr fr_mul_sum3_call(fr a0, fr b0, fr a1, fr b1, fr a2, fr b2) {
  const fr a[3] = {a0, a1, a2}, b[3] = {b0, b1, b2};
  return fr_mul_sum_inl<3>(a, b);
}
// (a0 b0 + a1 b1 + a2 b2) R^-1, canonical
ZC_D fr fr_mul_sum3(const fr& a0, const fr& b0, const fr& a1, const fr& b1, const fr& a2, const fr& b2) {
  return fr_mul_sum3_call(a0, b0, a1, b1, a2, b2);
}

// The multiplier is ~400 instructions; kernels call one out-of-line copy so
// that their code fits the instruction cache (inlined at every call site, a
// round body of ~30 products missed the cache on almost every instruction).
static __device__ __noinline__ fr fr_mul_call(fr a, fr b) { return fr_mul_inl(a, b); }
ZC_D fr fr_mul(const fr& a, const fr& b) { return fr_mul_call(a, b); }

#else
inline fr fr_add(const fr& a, const fr& b) { return fr_add_g(a, b); }
inline fr fr_sub(const fr& a, const fr& b) { return fr_sub_g(a, b); }
inline fr fr_mul(const fr& a, const fr& b) { return fr_mul_g(a, b); }
#endif

ZC_HD fr fr_from_u32(uint32_t x) {
  fr z = fr_zero();
  z.v[0] = x;
  return z;
}

}  // namespace zc
