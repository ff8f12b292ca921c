// zc_pcs.cu -- hash-based polynomial commitment around the ZeroCheck.
//
// Stages (1) and (3) of the prover workflow (Sec. 3.1): commit to the
// witness columns before the ZeroCheck, then open them at the point its
// SumCheck ends in, with the lightweight hash-based commitment the paper
// points to (Ligero).  The c columns (MLE tables of N = 2^n values, x_1 the
// most significant index bit) are m x w matrices (w = 2^nc, m = 2^nr,
// nr = n - nc, row i = entries i w .. i w + w - 1).
//   Commit: every row is Reed-Solomon encoded at rate 1/4, the values of
//   the row polynomial at x_k = 7 w_W^k, W = 4w (pcs_encode: slices of
//   w-point transforms); column digest D_kj = SHA-256 of the m entries of
//   position k of column j, leaf k = SHA-256(D_k0 | ... | D_k,c-1), binary
//   Merkle tree, root = SHA-256(le64(W) | top) (pcs_hash_tree).
//   Open at alpha with values v_j: u_j = sum_i eq(alpha_hi, i) M_j[i]
//   (v_j = <u_j, eq(alpha_lo, .)>), gamma from the transcript, u' = sum
//   gamma^(j m + i) M_j[i], t queried positions with their columns and
//   sibling paths.  The combinations and the column gather run on the
//   device; the transcript, the query indices and the paths on the host.
//   Verify (host): inner products, paths, and each queried column's
//   combinations against the encodings of u_j and u' at x_k.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "zc_internal.cuh"
#include "zc_transcript.cuh"

namespace zc {

struct PcsCombineArgs {
  const fr* col[kMaxCols];
  const fr* coef;     // level 1: [i] (per column) or [j m + i] (summed over columns)
  fr* part;           // [chunk][out][l] partial sums
  uint32_t c;
  uint64_t m, w;
  uint32_t sum_all;   // 1: one output summing every column
  uint32_t rows;      // rows per chunk (blockIdx.z)
};

// Partial sums over one chunk of rows: per column j (blockIdx.y) sum_i
// coef[i] M_j[i][l], or over the chunk of the c m stacked rows sum coef[q]
// M[q][l]; canonical columns times level-1 coefficients: canonical out.
// Consecutive threads take consecutive l: every row read is coalesced.
__global__ void __launch_bounds__(256) k_pcs_combine(PcsCombineArgs A) {
  const uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= A.w) return;
  const uint64_t q0 = (uint64_t)blockIdx.z * A.rows;
  fr acc = fr_zero();
  if (A.sum_all) {
    const uint64_t q1 = min(q0 + A.rows, (uint64_t)A.c * A.m);
    for (uint64_t q = q0; q < q1; q++) {
      const uint64_t j = q / A.m, i = q - j * A.m;
      acc = fr_add(acc, fr_mul(ld_fr(A.coef + q), ld_fr(A.col[j] + i * A.w + l)));
    }
  } else {
    const uint32_t j = blockIdx.y;
    const uint64_t q1 = min(q0 + A.rows, A.m);
    for (uint64_t i = q0; i < q1; i++) acc = fr_add(acc, fr_mul(ld_fr(A.coef + i), ld_fr(A.col[j] + i * A.w + l)));
  }
  const uint64_t outs = A.sum_all ? 1 : A.c;
  st_fr(A.part + ((uint64_t)blockIdx.z * outs + blockIdx.y) * A.w + l, acc);
}

// out[e] = sum over the chunks of part[chunk][e], e < count
__global__ void k_pcs_sum_chunks(const fr* part, uint64_t count, uint32_t chunks, fr* out) {
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  fr acc = fr_zero();
  for (uint32_t z = 0; z < chunks; z++) acc = fr_add(acc, ld_fr(part + (uint64_t)z * count + e));
  st_fr(out + e, acc);
}

struct PcsGatherArgs {
  const fr* enc[kMaxCols];
  const uint32_t* k;  // t queried positions
  fr* out;            // [s][j][i]
  uint32_t c, t;
  uint64_t m;
};

__global__ void k_pcs_gather(PcsGatherArgs A) {
  const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t per = (uint64_t)A.c * A.m;
  if (e >= per * A.t) return;
  const uint64_t s = e / per, r = e - s * per, j = r / A.m, i = r - j * A.m;
  st_fr(A.out + e, ld_fr(A.enc[j] + (uint64_t)A.k[s] * A.m + i));
}

// ---------------------------------------------------------------- host --

struct PcsShape {
  uint32_t n = 0, nc = 0, nr = 0, c = 0, t = 0, logW = 0;
  uint64_t m = 0, w = 0, W = 0;
};

static bool pcs_shape(const zc_pcs_params* p, PcsShape* S) {
  if (!p || p->n < 1 || p->n > 24 || p->c < 1 || p->c > (uint32_t)kMaxCols || p->t < 1 || p->t > (1u << 20))
    return false;
  S->n = p->n;
  S->nc = p->nc ? p->nc : (p->n < 12 ? p->n : 12);
  if (S->nc < 1 || S->nc > 12 || S->nc > p->n) return false;
  S->nr = p->n - S->nc;
  S->c = p->c;
  S->t = p->t;
  S->m = 1ull << S->nr;
  S->w = 1ull << S->nc;
  S->W = 4 * S->w;
  S->logW = S->nc + 2;
  return true;
}

static size_t pcs_proof_bytes(const PcsShape& S) {
  return 20 + 32 * ((size_t)S.c * S.w + S.w + (size_t)S.t * S.c * S.m + (size_t)S.t * S.logW);
}

static void put_le32(uint8_t* b, uint32_t v) {
  for (int i = 0; i < 4; i++) b[i] = (uint8_t)(v >> (8 * i));
}

static void digest_bytes(const uint32_t h[8], uint8_t out[32]) {
  for (int i = 0; i < 8; i++) {
    out[4 * i] = (uint8_t)(h[i] >> 24);
    out[4 * i + 1] = (uint8_t)(h[i] >> 16);
    out[4 * i + 2] = (uint8_t)(h[i] >> 8);
    out[4 * i + 3] = (uint8_t)h[i];
  }
}

static void root_of_top(uint64_t W, const uint8_t top[32], uint8_t root[32]) {
  uint8_t msg[40];
  for (int i = 0; i < 8; i++) msg[i] = (uint8_t)(W >> (8 * i));
  std::memcpy(msg + 8, top, 32);
  sha256_bytes(msg, 40, root);
}

// the opening's transcript: SHA-256("zerocheck-gb300/pcs-v1" | u32 n | u32 nc
// | u32 c | u32 t | root | enc(alpha_i) | enc(v_j)); absorb / squeeze as the
// ZeroCheck's transcript
struct PcsTranscript {
  uint8_t s[32];
  void init(const PcsShape& S, const uint8_t root[32], const uint8_t (*alpha)[32],
            const uint8_t (*values)[32]) {
    Sha256 h;
    h.init();
    const char* tag = "zerocheck-gb300/pcs-v1";
    h.update(reinterpret_cast<const uint8_t*>(tag), std::strlen(tag));
    const uint32_t v[4] = {S.n, S.nc, S.c, S.t};
    for (int q = 0; q < 4; q++) {
      uint8_t b[4];
      put_le32(b, v[q]);
      h.update(b, 4);
    }
    h.update(root, 32);
    for (uint32_t i = 0; i < S.n; i++) h.update(alpha[i], 32);
    for (uint32_t j = 0; j < S.c; j++) h.update(values[j], 32);
    h.final(s);
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
  // query position: the low 64 bits of the canonical challenge, mod W
  uint64_t query(uint64_t W) {
    const fr q = squeeze();
    return ((uint64_t)q.v[0] | ((uint64_t)q.v[1] << 32)) & (W - 1);
  }
};

// eq(x, b) over variables x[0..k) for every b < 2^k (b_1 the MSB), canonical
static std::vector<fr> eq_table(const fr* x, uint32_t k, const DevConst& C) {
  std::vector<fr> e(1, h_from_u64(1));
  const fr one = h_from_u64(1);
  for (uint32_t l = 0; l < k; l++) {
    std::vector<fr> e2(e.size() * 2);
    const fr a = x[l], b = fr_sub_g(one, x[l]);
    for (size_t q = 0; q < e.size(); q++) {
      e2[2 * q] = h_canon_mul(e[q], b, C);
      e2[2 * q + 1] = h_canon_mul(e[q], a, C);
    }
    e.swap(e2);
  }
  return e;
}

static bool load_canon(const uint8_t (*in)[32], size_t count, std::vector<fr>& out) {
  out.resize(count);
  for (size_t i = 0; i < count; i++)
    if (!h_from_bytes(in[i], &out[i])) return false;
  return true;
}

}  // namespace zc

struct zc_pcs {
  zc_ctx* ctx = nullptr;
  zc::PcsShape S;
  const zc::fr* col[zc::kMaxCols] = {};  // device columns (the caller's, or the copies in mem)
  zc::fr* enc[zc::kMaxCols] = {};        // encoded columns [k m + i]
  void* mem = nullptr;
  std::vector<uint8_t> tree;             // 2W - 1 digests, leaves first (host copy)
  uint8_t root[32];
};

using namespace zc;

#define PCS_TRY(ctx, call)                                         \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      (ctx)->err = std::string("pcs: ") + cudaGetErrorString(e_); \
      return ZC_ERR_CUDA;                                          \
    }                                                              \
  } while (0)

extern "C" {

zc_status zc_pcs_proof_size(const zc_pcs_params* params, size_t* bytes) {
  PcsShape S;
  if (!bytes || !pcs_shape(params, &S)) return ZC_ERR_ARG;
  *bytes = pcs_proof_bytes(S);
  return ZC_OK;
}

void zc_pcs_destroy(zc_pcs* pcs) {
  if (!pcs) return;
  if (pcs->mem) cudaFree(pcs->mem);
  delete pcs;
}

zc_status zc_pcs_commit(zc_ctx* ctx, const zc_pcs_params* params, const void* const* cols, int cols_on_device,
                        void* cuda_stream, zc_pcs** out, uint8_t root[32]) {
  if (!ctx || !cols || !out || !root) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  PcsShape S;
  if (!pcs_shape(params, &S)) {
    ctx->err = "pcs: bad parameters (1 <= n <= 24, 1 <= nc <= min(n, 12), 1 <= c <= 65, t >= 1)";
    return ZC_ERR_ARG;
  }
  for (uint32_t j = 0; j < S.c; j++)
    if (!cols[j]) return ZC_ERR_ARG;
  PCS_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const uint64_t N = S.m * S.w;
  zc_pcs* P = new zc_pcs();
  P->ctx = ctx;
  P->S = S;
  // device memory: host-column copies, encodings, coset table, digests, tree
  const size_t bcol = align_up(N * sizeof(fr), 256), benc = align_up(4 * N * sizeof(fr), 256);
  const size_t btab = align_up(S.W * sizeof(fr), 256), bdig = align_up(S.W * S.c * 32, 256);
  const size_t btree = align_up(2 * S.W * 32, 256);
  const size_t bytes = (cols_on_device ? 0 : bcol * S.c) + benc * S.c + btab + bdig + btree;
  if (cudaMalloc(&P->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    ctx->err = "pcs: cudaMalloc of the encoded columns failed";
    return ZC_ERR_OOM;
  }
  char* q = static_cast<char*>(P->mem);
  for (uint32_t j = 0; j < S.c; j++) {
    if (cols_on_device) {
      P->col[j] = static_cast<const fr*>(cols[j]);
    } else {
      fr* d = reinterpret_cast<fr*>(q);
      q += bcol;
      if (cudaMemcpyAsync(d, cols[j], N * sizeof(fr), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        zc_pcs_destroy(P);
        return ZC_ERR_CUDA;
      }
      P->col[j] = d;
    }
  }
  for (uint32_t j = 0; j < S.c; j++) {
    P->enc[j] = reinterpret_cast<fr*>(q);
    q += benc;
  }
  fr* tab = reinterpret_cast<fr*>(q);
  q += btab;
  uint32_t* dig = reinterpret_cast<uint32_t*>(q);
  q += bdig;
  uint32_t* tree = reinterpret_cast<uint32_t*>(q);
  ctx->launches = 0;
  zc_status s = pcs_encode(ctx, P->col, (int)S.c, S.nr, S.nc, P->enc, tab, st);
  if (s == ZC_OK) s = pcs_hash_tree(ctx, P->enc, (int)S.c, S.m, S.W, dig, tree, st);
  if (s != ZC_OK) {
    zc_pcs_destroy(P);
    return s;
  }
  const uint64_t nodes = 2 * S.W - 1;
  std::vector<uint32_t> words(8 * nodes);
  if (cudaMemcpyAsync(words.data(), tree, words.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    zc_pcs_destroy(P);
    ctx->err = "pcs: commit kernels failed";
    return ZC_ERR_CUDA;
  }
  P->tree.resize(32 * nodes);
  for (uint64_t u = 0; u < nodes; u++) digest_bytes(&words[8 * u], &P->tree[32 * u]);
  root_of_top(S.W, &P->tree[32 * (nodes - 1)], P->root);
  std::memcpy(root, P->root, 32);
  *out = P;
  return ZC_OK;
}

zc_status zc_pcs_open(zc_pcs* P, const uint8_t (*alpha)[32], const uint8_t (*values)[32], void* cuda_stream,
                      uint8_t* proof, size_t cap, size_t* len) {
  if (!P || !alpha || !values || !proof || !len) return ZC_ERR_ARG;
  zc_ctx* ctx = P->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  const PcsShape& S = P->S;
  const size_t need = pcs_proof_bytes(S);
  *len = need;
  if (cap < need) return ZC_ERR_BUFFER_TOO_SMALL;
  const DevConst& C = ctx->hconst;
  std::vector<fr> a, v;
  if (!load_canon(alpha, S.n, a) || !load_canon(values, S.c, v)) {
    ctx->err = "pcs: alpha or a value not canonical";
    return ZC_ERR_ARG;
  }
  PCS_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // device buffers of the opening
  const size_t ncoef = std::max<uint64_t>(S.m, (uint64_t)S.c * S.m);
  const size_t bcoef = align_up(ncoef * sizeof(fr), 256), bu = align_up((S.c + 1) * S.w * sizeof(fr), 256);
  const size_t bq = align_up(S.t * 4, 256), bg = align_up((size_t)S.t * S.c * S.m * sizeof(fr), 256);
  // partial sums: chunks of kRows rows, enough CTAs to fill the GPU
  constexpr uint32_t kRows = 32;
  const uint32_t ch_u = (uint32_t)((S.m + kRows - 1) / kRows);
  const uint32_t ch_g = (uint32_t)(((uint64_t)S.c * S.m + kRows - 1) / kRows);
  const size_t bp = align_up(std::max<uint64_t>((uint64_t)ch_u * S.c, ch_g) * S.w * sizeof(fr), 256);
  void* mem = nullptr;
  if (cudaMalloc(&mem, bcoef + bu + bq + bg + bp) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "pcs: cudaMalloc of the opening buffers failed";
    return ZC_ERR_OOM;
  }
  struct Free {
    void* p;
    ~Free() { cudaFree(p); }
  } guard{mem};
  char* q = static_cast<char*>(mem);
  fr* dcoef = reinterpret_cast<fr*>(q);
  fr* du = reinterpret_cast<fr*>(q + bcoef);
  uint32_t* dk = reinterpret_cast<uint32_t*>(q + bcoef + bu);
  fr* dg = reinterpret_cast<fr*>(q + bcoef + bu + bq);
  fr* dpart = reinterpret_cast<fr*>(q + bcoef + bu + bq + bg);

  PcsTranscript tr;
  tr.init(S, P->root, alpha, values);
  uint8_t* pp = proof;
  std::memcpy(pp, "ZCP1", 4);
  put_le32(pp + 4, S.n);
  put_le32(pp + 8, S.nc);
  put_le32(pp + 12, S.c);
  put_le32(pp + 16, S.t);
  pp += 20;
  // u_j = sum_i eq(alpha_hi, i) M_j[i]
  std::vector<fr> co = eq_table(a.data(), S.nr, C);
  for (auto& x : co) x = h_canon_mul(x, C.one, C);  // level 1
  PcsCombineArgs ca{};
  for (uint32_t j = 0; j < S.c; j++) ca.col[j] = P->col[j];
  ca.c = S.c;
  ca.m = S.m;
  ca.w = S.w;
  ca.coef = dcoef;
  ca.part = dpart;
  ca.sum_all = 0;
  ca.rows = kRows;
  PCS_TRY(ctx, cudaMemcpyAsync(dcoef, co.data(), S.m * sizeof(fr), cudaMemcpyHostToDevice, st));
  k_pcs_combine<<<dim3((unsigned)((S.w + 255) / 256), S.c, ch_u), 256, 0, st>>>(ca);
  k_pcs_sum_chunks<<<(unsigned)((S.c * S.w + 255) / 256), 256, 0, st>>>(dpart, S.c * S.w, ch_u, du);
  PCS_TRY(ctx, cudaMemcpyAsync(pp, du, (size_t)S.c * S.w * sizeof(fr), cudaMemcpyDeviceToHost, st));
  PCS_TRY(ctx, cudaStreamSynchronize(st));
  tr.absorb(pp, (size_t)S.c * S.w * 32);
  pp += (size_t)S.c * S.w * 32;
  // u' = sum_{j,i} gamma^(j m + i) M_j[i]
  const fr gamma = tr.squeeze();
  co.resize((size_t)S.c * S.m);
  fr g = C.one, gm = h_canon_mul(gamma, C.one, C);  // level 1
  for (size_t e = 0; e < co.size(); e++) {
    co[e] = g;
    g = fr_mul_g(g, gm);
  }
  ca.sum_all = 1;
  PCS_TRY(ctx, cudaMemcpyAsync(dcoef, co.data(), co.size() * sizeof(fr), cudaMemcpyHostToDevice, st));
  k_pcs_combine<<<dim3((unsigned)((S.w + 255) / 256), 1, ch_g), 256, 0, st>>>(ca);
  k_pcs_sum_chunks<<<(unsigned)((S.w + 255) / 256), 256, 0, st>>>(dpart, S.w, ch_g, du);
  PCS_TRY(ctx, cudaMemcpyAsync(pp, du, S.w * sizeof(fr), cudaMemcpyDeviceToHost, st));
  PCS_TRY(ctx, cudaStreamSynchronize(st));
  tr.absorb(pp, S.w * 32);
  pp += S.w * 32;
  // queries: the columns from the device, the paths from the host tree
  std::vector<uint32_t> ks(S.t);
  for (uint32_t s2 = 0; s2 < S.t; s2++) ks[s2] = (uint32_t)tr.query(S.W);
  PCS_TRY(ctx, cudaMemcpyAsync(dk, ks.data(), S.t * 4, cudaMemcpyHostToDevice, st));
  PcsGatherArgs ga{};
  for (uint32_t j = 0; j < S.c; j++) ga.enc[j] = P->enc[j];
  ga.k = dk;
  ga.out = dg;
  ga.c = S.c;
  ga.t = S.t;
  ga.m = S.m;
  const uint64_t tot = (uint64_t)S.t * S.c * S.m;
  k_pcs_gather<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ga);
  std::vector<uint8_t> cols((size_t)tot * 32);
  PCS_TRY(ctx, cudaMemcpyAsync(cols.data(), dg, cols.size(), cudaMemcpyDeviceToHost, st));
  PCS_TRY(ctx, cudaStreamSynchronize(st));
  const size_t per = (size_t)S.c * S.m * 32;
  for (uint32_t s2 = 0; s2 < S.t; s2++) {
    std::memcpy(pp, &cols[s2 * per], per);
    pp += per;
    uint64_t off = 0, cnt = S.W, idx = ks[s2];
    for (uint32_t lv = 0; lv < S.logW; lv++) {
      std::memcpy(pp, &P->tree[32 * (off + (idx ^ 1))], 32);
      pp += 32;
      off += cnt;
      cnt /= 2;
      idx >>= 1;
    }
  }
  return ZC_OK;
}

zc_status zc_pcs_verify(const zc_pcs_params* params, const uint8_t root[32], const uint8_t (*alpha)[32],
                        const uint8_t (*values)[32], const uint8_t* proof, size_t len, int* accept) {
  if (!accept) return ZC_ERR_ARG;
  *accept = 0;
  PcsShape S;
  if (!pcs_shape(params, &S) || !root || !alpha || !values || !proof) return ZC_ERR_ARG;
  if (len != pcs_proof_bytes(S)) return ZC_ERR_ARG;
  uint8_t hdr[20];
  std::memcpy(hdr, "ZCP1", 4);
  put_le32(hdr + 4, S.n);
  put_le32(hdr + 8, S.nc);
  put_le32(hdr + 12, S.c);
  put_le32(hdr + 16, S.t);
  if (std::memcmp(hdr, proof, 20) != 0) return ZC_ERR_ARG;
  const DevConst& C = host_constants();
  std::vector<fr> a, v, u;
  if (!load_canon(alpha, S.n, a) || !load_canon(values, S.c, v)) return ZC_ERR_ARG;
  const uint8_t* pp = proof + 20;
  if (!load_canon(reinterpret_cast<const uint8_t(*)[32]>(pp), (size_t)(S.c + 1) * S.w, u)) return ZC_ERR_ARG;
  bool ok = true;
  // v_j = <u_j, eq(alpha_lo, .)>
  const std::vector<fr> eql = eq_table(a.data() + S.nr, S.nc, C), eqh = eq_table(a.data(), S.nr, C);
  for (uint32_t j = 0; j < S.c; j++) {
    fr acc = fr_zero();
    for (uint64_t l = 0; l < S.w; l++) acc = fr_add_g(acc, h_canon_mul(u[j * S.w + l], eql[l], C));
    if (!fr_equal(acc, v[j])) ok = false;
  }
  PcsTranscript tr;
  tr.init(S, root, alpha, values);
  tr.absorb(pp, (size_t)S.c * S.w * 32);
  const fr gamma = tr.squeeze();
  tr.absorb(pp + (size_t)S.c * S.w * 32, S.w * 32);
  pp += (size_t)(S.c + 1) * S.w * 32;
  std::vector<fr> gp((size_t)S.c * S.m);
  fr g = h_from_u64(1);
  for (auto& x : gp) {
    x = g;
    g = h_canon_mul(g, gamma, C);
  }
  const fr wW = h_root_of_unity(S.logW, C), seven = h_from_u64(7);
  // The query positions come from the transcript alone; each query is then
  // checked on its own (its path, and the encodings of u_j and u' at x_k
  // against the column's combinations), the queries spread over host threads.
  std::vector<uint64_t> ks(S.t);
  for (uint32_t s2 = 0; s2 < S.t; s2++) ks[s2] = tr.query(S.W);
  const size_t qbytes = (size_t)S.c * S.m * 32 + (size_t)S.logW * 32;
  std::atomic<int> bad_fmt{0}, bad{ok ? 0 : 1};
  std::atomic<uint32_t> next{0};
  auto worker = [&]() {
    std::vector<fr> col;
    std::vector<uint8_t> dg(32 * (size_t)S.c);
    for (uint32_t s2; (s2 = next.fetch_add(1)) < S.t;) {
      if (bad.load() || bad_fmt.load()) return;
      const uint64_t k = ks[s2];
      const uint8_t* q = pp + s2 * qbytes;
      if (!load_canon(reinterpret_cast<const uint8_t(*)[32]>(q), (size_t)S.c * S.m, col)) {
        bad_fmt = 1;
        return;
      }
      // the column up to the root
      for (uint32_t j = 0; j < S.c; j++) sha256_bytes(q + 32 * (size_t)j * S.m, S.m * 32, &dg[32 * j]);
      uint8_t node[32], pair[64];
      sha256_bytes(dg.data(), dg.size(), node);
      q += (size_t)S.c * S.m * 32;
      uint64_t idx = k;
      for (uint32_t lv = 0; lv < S.logW; lv++) {
        if (idx & 1) {
          std::memcpy(pair, q, 32);
          std::memcpy(pair + 32, node, 32);
        } else {
          std::memcpy(pair, node, 32);
          std::memcpy(pair + 32, q, 32);
        }
        sha256_bytes(pair, 64, node);
        q += 32;
        idx >>= 1;
      }
      uint8_t r2[32];
      root_of_top(S.W, node, r2);
      if (std::memcmp(r2, root, 32) != 0) bad = 1;
      const fr xk = h_canon_mul(seven, h_pow(wW, k, C), C);
      for (uint32_t j = 0; j <= S.c; j++) {
        fr enc_u = fr_zero();
        for (uint64_t l = S.w; l-- > 0;) enc_u = fr_add_g(h_canon_mul(enc_u, xk, C), u[j * S.w + l]);
        fr comb = fr_zero();
        if (j < S.c)
          for (uint64_t i = 0; i < S.m; i++) comb = fr_add_g(comb, h_canon_mul(eqh[i], col[j * S.m + i], C));
        else
          for (size_t e = 0; e < gp.size(); e++) comb = fr_add_g(comb, h_canon_mul(gp[e], col[e], C));
        if (!fr_equal(enc_u, comb)) bad = 1;
      }
    }
  };
  const unsigned nthr = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), S.t));
  std::vector<std::thread> pool;
  for (unsigned w = 1; w < nthr; w++) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (bad_fmt) return ZC_ERR_ARG;
  ok = bad.load() == 0;
  *accept = ok ? 1 : 0;
  return ZC_OK;
}

}  // extern "C"
