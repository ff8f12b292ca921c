// zc_sha256.cuh -- SHA-256 (FIPS 180-4) for host and device code.
//
// Used for the Fiat-Shamir transcript (the paper's Hash(.) in Fig.
// side-by-side-zc) and the Merkle-root commitment stand-in.  The device
// compression keeps the 64-word schedule in a 16-word ring so that one
// thread hashes with registers only.
#pragma once
#include <stdint.h>
#include "zc_field.cuh"

namespace zc {

#if defined(__CUDACC__)
#define ZC_SHA_K_DECL __device__ __constant__
#else
#define ZC_SHA_K_DECL static
#endif

ZC_SHA_K_DECL const uint32_t kShaK[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};

#if !defined(__CUDACC__)
static const uint32_t* sha_k_host() { return kShaK; }
#else
static const uint32_t kShaKHost[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};
#endif

ZC_HD uint32_t sha_rotr(uint32_t x, int n) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(x, x, n);
#else
  return (x >> n) | (x << (32 - n));
#endif
}

ZC_HD uint32_t sha_bswap(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __byte_perm(x, 0, 0x0123);
#else
  return (x >> 24) | ((x >> 8) & 0xff00u) | ((x << 8) & 0xff0000u) | (x << 24);
#endif
}

// Compress one 64-byte block given as 16 big-endian message words.
ZC_HD void sha256_compress(uint32_t h[8], const uint32_t w_in[16]) {
#if defined(__CUDA_ARCH__)
  const uint32_t* K = kShaK;
#elif defined(__CUDACC__)
  const uint32_t* K = kShaKHost;
#else
  const uint32_t* K = sha_k_host();
#endif
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 16; i++) w[i] = w_in[i];
  uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#pragma unroll
  for (int t = 0; t < 64; t++) {
    uint32_t wt;
    if (t < 16) {
      wt = w[t];
    } else {
      uint32_t x15 = w[(t + 1) & 15], x2 = w[(t + 14) & 15];
      uint32_t s0 = sha_rotr(x15, 7) ^ sha_rotr(x15, 18) ^ (x15 >> 3);
      uint32_t s1 = sha_rotr(x2, 17) ^ sha_rotr(x2, 19) ^ (x2 >> 10);
      wt = w[t & 15] + s0 + w[(t + 9) & 15] + s1;
      w[t & 15] = wt;
    }
    uint32_t t1 = hh + (sha_rotr(e, 6) ^ sha_rotr(e, 11) ^ sha_rotr(e, 25)) + ((e & f) ^ (~e & g)) +
                  K[t] + wt;
    uint32_t t2 = (sha_rotr(a, 2) ^ sha_rotr(a, 13) ^ sha_rotr(a, 22)) + ((a & b) | (c & (a | b)));
    hh = g;
    g = f;
    f = e;
    e = d + t1;
    d = c;
    c = b;
    b = a;
    a = t1 + t2;
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d;
  h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

#if defined(__CUDACC__)
// Two out-of-line copies of the compression for the transcript, where one
// thread hashes a few blocks per challenge.  Both are single shared copies
// (__noinline__): an inlined unrolled body is ~25 KB per call site, fetched
// cold each round.  sha256_compress_hot is the unrolled body, fastest once
// it is in the instruction cache (rounds that follow one another inside one
// launch); sha256_compress_small is a 16-round body run four times (the
// schedule update skipped in the first pass by a uniform branch, the round
// constants read by index), for a challenge that runs once in a launch and
// finds its code cold.
static __device__ __noinline__ void sha256_compress_hot(uint32_t h[8], const uint32_t w_in[16]) {
  sha256_compress(h, w_in);
}

static __device__ __noinline__ void sha256_compress_small(uint32_t h[8], const uint32_t w_in[16]) {
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 16; i++) w[i] = w_in[i];
  uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#pragma unroll 1
  for (int j = 0; j < 64; j += 16) {
#pragma unroll
    for (int i = 0; i < 16; i++) {
      if (j > 0) {
        const uint32_t x15 = w[(i + 1) & 15], x2 = w[(i + 14) & 15];
        const uint32_t s0 = sha_rotr(x15, 7) ^ sha_rotr(x15, 18) ^ (x15 >> 3);
        const uint32_t s1 = sha_rotr(x2, 17) ^ sha_rotr(x2, 19) ^ (x2 >> 10);
        w[i] = w[i] + s0 + w[(i + 9) & 15] + s1;
      }
      const uint32_t t1 = hh + (sha_rotr(e, 6) ^ sha_rotr(e, 11) ^ sha_rotr(e, 25)) + ((e & f) ^ (~e & g)) +
                          kShaK[j + i] + w[i];
      const uint32_t t2 = (sha_rotr(a, 2) ^ sha_rotr(a, 13) ^ sha_rotr(a, 22)) + ((a & b) | (c & (a | b)));
      hh = g;
      g = f;
      f = e;
      e = d + t1;
      d = c;
      c = b;
      b = a;
      a = t1 + t2;
    }
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d;
  h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}
#endif

ZC_HD void sha256_init(uint32_t h[8]) {
  h[0] = 0x6a09e667; h[1] = 0xbb67ae85; h[2] = 0x3c6ef372; h[3] = 0xa54ff53a;
  h[4] = 0x510e527f; h[5] = 0x9b05688c; h[6] = 0x1f83d9ab; h[7] = 0x5be0cd19;
}

// Incremental hasher over bytes (used for short transcript messages).
struct Sha256 {
  uint32_t h[8];
  uint32_t blk[16];
  uint32_t nbytes;   // bytes in the current block
  uint64_t total;

  ZC_HD void init() {
    sha256_init(h);
    nbytes = 0;
    total = 0;
    for (int i = 0; i < 16; i++) blk[i] = 0;
  }
  ZC_HD void put_byte(uint8_t x) {
    uint32_t wi = nbytes >> 2, sh = 24 - 8 * (nbytes & 3);
    blk[wi] |= (uint32_t)x << sh;
    nbytes++;
    total++;
    if (nbytes == 64) {
      sha256_compress(h, blk);
      for (int i = 0; i < 16; i++) blk[i] = 0;
      nbytes = 0;
    }
  }
  ZC_HD void update(const uint8_t* m, uint64_t len) {
    for (uint64_t i = 0; i < len; i++) put_byte(m[i]);
  }
  // 32-bit little-endian words, e.g. a field element's limbs
  ZC_HD void update_words_le(const uint32_t* wds, int count) {
    for (int i = 0; i < count; i++) {
      uint32_t x = wds[i];
      put_byte((uint8_t)x);
      put_byte((uint8_t)(x >> 8));
      put_byte((uint8_t)(x >> 16));
      put_byte((uint8_t)(x >> 24));
    }
  }
  ZC_HD void final(uint8_t out[32]) {
    uint64_t bits = total * 8;
    put_byte(0x80);
    while (nbytes != 56) put_byte(0);
    for (int i = 7; i >= 0; i--) put_byte((uint8_t)(bits >> (8 * i)));
    for (int i = 0; i < 8; i++) {
      out[4 * i] = (uint8_t)(h[i] >> 24);
      out[4 * i + 1] = (uint8_t)(h[i] >> 16);
      out[4 * i + 2] = (uint8_t)(h[i] >> 8);
      out[4 * i + 3] = (uint8_t)h[i];
    }
  }
};

ZC_HD void sha256_bytes(const uint8_t* m, uint64_t len, uint8_t out[32]) {
  Sha256 s;
  s.init();
  s.update(m, len);
  s.final(out);
}

}  // namespace zc
