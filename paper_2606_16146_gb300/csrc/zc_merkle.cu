// zc_merkle.cu -- commitment stand-in root(v) on the device.
//
// The paper commits to [g] and [q] before the Fiat-Shamir challenge (Fig.
// side-by-side-zc, "Commit"); the commitment scheme itself is outside its
// comparison (Sec. 3.4).  Here root(v) is a binary SHA-256 Merkle tree:
// leaf t = SHA-256 of the canonical bytes of v[64 t .. min(64 t + 63, L-1)]
// (the last leaf is shorter when 64 does not divide L), node =
// SHA-256(left | right), and at a level with an odd count the last node
// moves up unchanged; root = SHA-256(le64(len) | top).  One thread hashes
// one 2 KB leaf; a CTA reduces its 128 leaves to one node in shared memory;
// a second kernel reduces the CTA nodes of each column.  The CTAs' leaf
// ranges start at multiples of 128, so their subtrees are the global tree's
// first seven levels (a ragged last CTA's node arrives at level 7 unchanged,
// as the odd last node of every level above it).
#include "zc_internal.cuh"
#include "zc_transcript.cuh"

namespace zc {

constexpr int kLeafElems = 64;
constexpr int kLeafCta = 128;

struct RootLeafArgs {
  const fr* col[kMaxCols];
  uint64_t L;
  uint32_t per;        // elements per leaf (the last leaf may have fewer)
  uint64_t nleaves;
  uint32_t ctas;       // CTAs per column
  uint32_t* nodes;     // [c][ctas][8] digest words
};

struct RootTopArgs {
  uint32_t* nodes;     // [c][ctas][8]
  uint32_t* tmp;       // same size
  uint32_t ctas;
  uint64_t L;
  uint8_t* roots;      // [c][32]
};

// SHA-256 of len bytes at p (len a multiple of 32, p 16-byte aligned).
__device__ void sha256_device_mem(const uint8_t* p, uint32_t len, uint32_t h[8]) {
  sha256_init(h);
  const uint4* q = reinterpret_cast<const uint4*>(p);
  uint32_t nfull = len / 64;
  uint32_t w[16];
  for (uint32_t b = 0; b < nfull; b++) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      uint4 x = __ldg(q + 4 * b + i);
      w[4 * i] = sha_bswap(x.x);
      w[4 * i + 1] = sha_bswap(x.y);
      w[4 * i + 2] = sha_bswap(x.z);
      w[4 * i + 3] = sha_bswap(x.w);
    }
    sha256_compress(h, w);
  }
  uint32_t rem = len - nfull * 64;  // 0 or 32
#pragma unroll
  for (int i = 0; i < 16; i++) w[i] = 0;
  if (rem) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
      uint4 x = __ldg(q + 4 * nfull + i);
      w[4 * i] = sha_bswap(x.x);
      w[4 * i + 1] = sha_bswap(x.y);
      w[4 * i + 2] = sha_bswap(x.z);
      w[4 * i + 3] = sha_bswap(x.w);
    }
    w[8] = 0x80000000u;
  } else {
    w[0] = 0x80000000u;
  }
  uint64_t bits = (uint64_t)len * 8;
  w[14] = (uint32_t)(bits >> 32);
  w[15] = (uint32_t)bits;
  sha256_compress(h, w);
}

// node = SHA-256(left | right) for two digests given as words
__device__ __forceinline__ void sha256_node(const uint32_t* l, const uint32_t* r, uint32_t out[8]) {
  uint32_t w[16];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    w[i] = l[i];
    w[8 + i] = r[i];
  }
  sha256_init(out);
  sha256_compress(out, w);
#pragma unroll
  for (int i = 0; i < 16; i++) w[i] = 0;
  w[0] = 0x80000000u;
  w[15] = 512;
  sha256_compress(out, w);
}

__global__ void __launch_bounds__(kLeafCta) k_root_leaves(RootLeafArgs A) {
  __shared__ uint32_t dig[kLeafCta][9];
  const int c = blockIdx.y;
  const uint64_t leaf = (uint64_t)blockIdx.x * kLeafCta + threadIdx.x;
  uint64_t cnt64 = A.nleaves - (uint64_t)blockIdx.x * kLeafCta;
  const uint32_t cnt = cnt64 < kLeafCta ? (uint32_t)cnt64 : kLeafCta;
  uint32_t h[8];
  if (threadIdx.x < cnt) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(A.col[c] + leaf * A.per);
    const uint64_t left = A.L - leaf * A.per;
    const uint32_t elems = left < A.per ? (uint32_t)left : A.per;
    sha256_device_mem(p, elems * 32, h);
#pragma unroll
    for (int i = 0; i < 8; i++) dig[threadIdx.x][i] = h[i];
  }
  for (uint32_t w = cnt; w > 1; w = (w + 1) / 2) {
    __syncthreads();
    const bool pair = threadIdx.x < w / 2, carry = (w & 1) && threadIdx.x == w / 2;
    if (pair) sha256_node(dig[2 * threadIdx.x], dig[2 * threadIdx.x + 1], h);
    if (carry) {
#pragma unroll
      for (int i = 0; i < 8; i++) h[i] = dig[w - 1][i];
    }
    __syncthreads();
    if (pair || carry) {
#pragma unroll
      for (int i = 0; i < 8; i++) dig[threadIdx.x][i] = h[i];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t* out = A.nodes + ((size_t)c * A.ctas + blockIdx.x) * 8;
#pragma unroll
    for (int i = 0; i < 8; i++) out[i] = dig[0][i];
  }
}

__global__ void __launch_bounds__(256) k_root_top(RootTopArgs A) {
  const int c = blockIdx.x;
  uint32_t* a = A.nodes + (size_t)c * A.ctas * 8;
  uint32_t* b = A.tmp + (size_t)c * A.ctas * 8;
  for (uint32_t w = A.ctas; w > 1; w = (w + 1) / 2) {
    for (uint32_t t = threadIdx.x; t < w / 2; t += blockDim.x) {
      uint32_t h[8];
      sha256_node(a + 16 * t, a + 16 * t + 8, h);
#pragma unroll
      for (int i = 0; i < 8; i++) b[8 * t + i] = h[i];
    }
    if ((w & 1) && threadIdx.x == 0)  // the odd last node moves up unchanged
      for (int i = 0; i < 8; i++) b[8 * (w / 2) + i] = a[8 * (w - 1) + i];
    __syncthreads();
    uint32_t* x = a;
    a = b;
    b = x;
  }
  if (threadIdx.x == 0) {
    // root = SHA-256(le64(L) | top): 40 bytes, one block
    uint32_t w[16];
    uint64_t L = A.L;
    uint8_t lb[8];
    for (int i = 0; i < 8; i++) lb[i] = (uint8_t)(L >> (8 * i));
    w[0] = ((uint32_t)lb[0] << 24) | ((uint32_t)lb[1] << 16) | ((uint32_t)lb[2] << 8) | lb[3];
    w[1] = ((uint32_t)lb[4] << 24) | ((uint32_t)lb[5] << 16) | ((uint32_t)lb[6] << 8) | lb[7];
    for (int i = 0; i < 8; i++) w[2 + i] = a[i];
    w[10] = 0x80000000u;
    for (int i = 11; i < 15; i++) w[i] = 0;
    w[15] = 40 * 8;
    uint32_t h[8];
    sha256_init(h);
    sha256_compress(h, w);
    uint8_t* out = A.roots + 32 * c;
    for (int i = 0; i < 8; i++) {
      out[4 * i] = (uint8_t)(h[i] >> 24);
      out[4 * i + 1] = (uint8_t)(h[i] >> 16);
      out[4 * i + 2] = (uint8_t)(h[i] >> 8);
      out[4 * i + 3] = (uint8_t)h[i];
    }
  }
}

zc_status launch_roots(zc_ctx* ctx, const fr* const* dcols, int c, uint64_t L, uint8_t* droots,
                       cudaStream_t st) {
  if (L == 0 || c < 1 || c > kMaxCols) {
    ctx->err = "root: empty vector or too many columns";
    return ZC_ERR_ARG;
  }
  RootLeafArgs la{};
  for (int j = 0; j < c; j++) la.col[j] = dcols[j];
  la.L = L;
  la.per = L < (uint64_t)kLeafElems ? (uint32_t)L : (uint32_t)kLeafElems;
  la.nleaves = (L + la.per - 1) / la.per;
  la.ctas = (uint32_t)((la.nleaves + kLeafCta - 1) / kLeafCta);
  size_t words = (size_t)c * la.ctas * 8;
  uint32_t* nodes = ctx->arena.take<uint32_t>(words);
  uint32_t* tmp = ctx->arena.take<uint32_t>(words);
  if (!nodes || !tmp) {
    ctx->err = "root: scratch arena too small";
    return ZC_ERR_OOM;
  }
  la.nodes = nodes;
  dim3 grid(la.ctas, c);
  k_root_leaves<<<grid, kLeafCta, 0, st>>>(la);
  ctx->launches++;
  RootTopArgs ta{};
  ta.nodes = nodes;
  ta.tmp = tmp;
  ta.ctas = la.ctas;
  ta.L = L;
  ta.roots = droots;
  k_root_top<<<c, 256, 0, st>>>(ta);
  ctx->launches++;
  ZC_CUDA_TRY(ctx, cudaGetLastError());
  return ZC_OK;
}

size_t root_scratch_bytes(int c, uint64_t L) {
  uint64_t per = L < (uint64_t)kLeafElems ? L : (uint64_t)kLeafElems;
  uint64_t nl = (L + per - 1) / per;
  uint64_t ctas = (nl + kLeafCta - 1) / kLeafCta;
  return 2 * ((size_t)c * ctas * 32 + 256);
}

// ---- hash-based commitment (zc_pcs.cu): digest of codeword position k of
// column j = SHA-256 of its m canonical entries enc[j][k m .. k m + m);
// leaf k = SHA-256 of the c digests of position k; tree levels above.

struct PcsDigestArgs {
  const fr* enc[kMaxCols];
  uint32_t c;
  uint64_t m, W;
  uint32_t* dig;      // [k][j][8] words
};

__global__ void __launch_bounds__(128) k_pcs_digests(PcsDigestArgs A) {
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.W * A.c) return;
  const uint64_t k = e / A.c;
  const uint32_t j = (uint32_t)(e - k * A.c);
  uint32_t h[8];
  sha256_device_mem(reinterpret_cast<const uint8_t*>(A.enc[j] + k * A.m), (uint32_t)(A.m * 32), h);
#pragma unroll
  for (int i = 0; i < 8; i++) A.dig[8 * e + i] = h[i];
}

struct PcsLevelArgs {
  const uint32_t* in;  // nodes of the level below (8 words each), or the digests
  uint32_t* out;
  uint64_t count;      // nodes written
  uint32_t words;      // words hashed per node (16 for a pair, 8 c for a leaf)
};

__global__ void k_pcs_level(PcsLevelArgs A) {
  const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= A.count) return;
  uint32_t h[8];
  sha256_words(A.in + (uint64_t)A.words * u, A.words, h);
#pragma unroll
  for (int i = 0; i < 8; i++) A.out[8 * u + i] = h[i];
}

zc_status pcs_hash_tree(zc_ctx* ctx, const fr* const* enc, int c, uint64_t m, uint64_t W, uint32_t* dig,
                        uint32_t* tree, cudaStream_t st) {
  PcsDigestArgs da{};
  for (int j = 0; j < c; j++) da.enc[j] = enc[j];
  da.c = (uint32_t)c;
  da.m = m;
  da.W = W;
  da.dig = dig;
  const uint64_t nd = W * (uint64_t)c;
  k_pcs_digests<<<(unsigned)((nd + 127) / 128), 128, 0, st>>>(da);
  ctx->launches++;
  PcsLevelArgs la{};
  la.in = dig;
  la.out = tree;
  la.count = W;
  la.words = 8u * (uint32_t)c;
  k_pcs_level<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(la);
  ctx->launches++;
  uint64_t off = 0;
  for (uint64_t cnt = W; cnt > 1; cnt /= 2) {
    la.in = tree + 8 * off;
    la.out = tree + 8 * (off + cnt);
    la.count = cnt / 2;
    la.words = 16;
    k_pcs_level<<<(unsigned)((cnt / 2 + 127) / 128), 128, 0, st>>>(la);
    ctx->launches++;
    off += cnt;
  }
  return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

}  // namespace zc
