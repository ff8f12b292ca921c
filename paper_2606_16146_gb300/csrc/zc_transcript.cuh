// zc_transcript.cuh -- Fiat-Shamir transcript on the device, word-based.
//
// The paper derives every challenge by hashing (Fig. side-by-side-zc:
// "r <- Hash([g])", "alpha_i <- Hash(G_i)").  State S is a SHA-256 digest;
// absorb(m): S = SHA-256(S | m); squeeze: S = SHA-256(S | 0x43) and the
// challenge is int_le(S) mod r.  All absorbed messages here are whole 32-bit
// words (digests and canonical field elements), so blocks are assembled as
// words: a field element's little-endian bytes are its limbs byte-swapped.
#pragma once
#include "zc_internal.cuh"

namespace zc {

#if defined(__CUDACC__)

// One compression for transcript hashing: COLD picks the compact copy, for a
// hash that runs once in a launch (see zc_sha256.cuh).
template <bool COLD>
__device__ __forceinline__ void tr_compress(uint32_t h[8], const uint32_t w[16]) {
  if (COLD) sha256_compress_small(h, w);
  else sha256_compress_hot(h, w);
}

// SHA-256 of a word message in pieces: tr_blocks compresses the complete
// 16-word blocks [b0, b1); tr_last compresses what remains after the last
// complete block, with the padding and the bit length.
template <bool COLD>
__device__ inline void tr_blocks(uint32_t h[8], const uint32_t* w, uint32_t b0, uint32_t b1) {
  uint32_t blk[16];
  for (uint32_t b = b0; b < b1; b++) {
#pragma unroll
    for (int i = 0; i < 16; i++) blk[i] = w[16 * b + i];
    tr_compress<COLD>(h, blk);
  }
}

template <bool COLD>
__device__ inline void tr_last(uint32_t h[8], const uint32_t* w, uint32_t nwords) {
  uint32_t blk[16];
  const uint32_t full = nwords / 16, rem = nwords - 16 * full;
#pragma unroll
  for (int i = 0; i < 16; i++) blk[i] = 0;
  for (uint32_t i = 0; i < rem; i++) blk[i] = w[16 * full + i];
  blk[rem] = 0x80000000u;
  const uint64_t bits = (uint64_t)nwords * 32;
  if (rem + 1 > 14) {
    tr_compress<COLD>(h, blk);
#pragma unroll
    for (int i = 0; i < 16; i++) blk[i] = 0;
  }
  blk[14] = (uint32_t)(bits >> 32);
  blk[15] = (uint32_t)bits;
  tr_compress<COLD>(h, blk);
}

// SHA-256 over nwords big-endian message words (any count), digest in out.
template <bool COLD = false>
__device__ inline void sha256_words(const uint32_t* w, uint32_t nwords, uint32_t out[8]) {
  sha256_init(out);
  tr_blocks<COLD>(out, w, 0, nwords / 16);
  tr_last<COLD>(out, w, nwords);
}

// S <- SHA-256(S | m) for a 32-byte message given as bytes
__device__ inline void tr_absorb32(uint32_t S[8], const uint8_t* m) {
  uint32_t w[16];
  for (int i = 0; i < 8; i++) w[i] = S[i];
  for (int i = 0; i < 8; i++)
    w[8 + i] = ((uint32_t)m[4 * i] << 24) | ((uint32_t)m[4 * i + 1] << 16) |
               ((uint32_t)m[4 * i + 2] << 8) | m[4 * i + 3];
  sha256_words(w, 16, S);
}

// int_le(digest) mod r as a canonical element (2^256 < 3r: at most two subtractions)
__device__ inline fr digest_mod_r(const uint32_t h[8]) {
  fr x;
  for (int i = 0; i < 8; i++) x.v[i] = sha_bswap(h[i]);
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

// S <- SHA-256(S | 0x43); returns the canonical challenge
template <bool COLD = false>
__device__ inline fr tr_squeeze(uint32_t S[8]) {
  uint32_t w[16];
  for (int i = 0; i < 8; i++) w[i] = S[i];
  w[8] = 0x43800000u;  // the byte 0x43, then the padding bit
  for (int i = 9; i < 15; i++) w[i] = 0;
  w[15] = 33 * 8;
  uint32_t h[8];
  sha256_init(h);
  tr_compress<COLD>(h, w);
  for (int i = 0; i < 8; i++) S[i] = h[i];
  return digest_mod_r(h);
}

#endif

}  // namespace zc
