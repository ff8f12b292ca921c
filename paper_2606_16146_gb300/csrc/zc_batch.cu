// zc_batch.cu -- many ZeroCheck instances of mixed size, degree and form in
// one submission, optionally captured as a single CUDA graph.
//
// The paper evaluates one proof at a time; batching is a deployment mode of
// the same arithmetic.  A batch runs on lanes: child contexts that share the
// parent's constants and per-size NTT tables and own a scratch arena and a
// stream.  Instances go longest-first to the least-loaded lane (by a cost
// estimate in modular multiplications); each lane proves its instances in
// order, lanes run concurrently, so small instances that cannot fill the GPU
// on their own overlap.  All allocation happens in the prepare step, so the
// submission itself only enqueues kernels and can be captured into a graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "zc_internal.cuh"

namespace zc {

constexpr int kDefaultLanes = 16;
constexpr int kMaxLanes = 64;

static double instance_cost(const zc_params& p, zc_form f) {
  const double N = std::ldexp(1.0, (int)p.n);
  const int c = gate_ncols(p.gate, p.d);
  if (f != ZC_FORM_NTT) {
    const double g = p.gate == ZC_GATE_PLONK ? 5.0 : (double)p.d - 1;
    return N * ((p.d + 1) * (g + 1) + 1 + c);
  }
  NttDomain D;
  if (!ntt_domain(p.n, p.d, p.log_blowup, &D)) return 0.0;
  const double M = (double)D.M, s = M / N;
  return c * N / 2 * p.n + c * s * (N + N / 2 * p.n) + M * (p.n + D.k) / 2 + M * p.d;
}

zc_status make_lanes(zc_ctx* ctx, int K) {
  while ((int)ctx->lanes.size() < K) {
    zc_ctx* L = new zc_ctx();
    L->device = ctx->device;
    L->max_n = ctx->max_n;
    L->max_d = ctx->max_d;
    L->budget = 0;
    L->sm_count = ctx->sm_count;
    L->hconst = ctx->hconst;
    L->dconst = ctx->dconst;
    L->dtabs = ctx->dtabs;
    L->htabs = ctx->htabs;
    L->owns_const = false;
    L->table_owner = ctx;
    L->skip_point = ctx->skip_point;
    if (cudaMallocHost(&L->pinned, 1 << 16) != cudaSuccess) {
      cudaGetLastError();
      delete L;
      return ZC_ERR_OOM;
    }
    L->pinned_cap = 1 << 16;
    for (int i = 0; i < 8; i++) cudaEventCreate(&L->ev[i]);
    cudaStream_t s;
    cudaEvent_t e;
    // lane 0 runs at the device's greatest stream priority: in a batch it
    // gets the longest instance (longest-first assignment), in serving the
    // large requests (zc_serve_opts.priority_bytes)
    int lo = 0, hi = 0;
    if (ctx->lanes.empty() && cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess)
      cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi);
    else
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    ctx->lanes.push_back(L);
    ctx->lane_streams.push_back(s);
    ctx->lane_join.push_back(e);
  }
  if (!ctx->fork_ev) cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

// Instance -> lane, longest first onto the least-loaded lane.
static std::vector<int> assign_lanes(uint32_t count, const zc_form* forms, const zc_params* params,
                                     int K) {
  std::vector<uint32_t> order(count);
  std::iota(order.begin(), order.end(), 0u);
  std::vector<double> cost(count);
  for (uint32_t i = 0; i < count; i++) cost[i] = instance_cost(params[i], forms[i]);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
  std::vector<double> load(K, 0.0);
  std::vector<int> lane(count, 0);
  for (uint32_t i : order) {
    int best = 0;
    for (int k = 1; k < K; k++)
      if (load[k] < load[best]) best = k;
    lane[i] = best;
    load[best] += cost[i];
  }
  return lane;
}

static int lanes_for(const zc_ctx* ctx, uint32_t count) {
  const int32_t t = ctx->tuned(ZC_FORM_SUMCHECK, 0, ZC_TUNE_BATCH_LANES);
  const int want = t > 0 ? std::min<int>(t, kMaxLanes) : kDefaultLanes;
  return (int)std::min<uint32_t>(count, (uint32_t)want);
}

zc_status batch_prepare(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                        const bool* q_direct, cudaStream_t st) {
  for (uint32_t i = 0; i < count; i++) {
    zc_status s = check_params(ctx, &params[i], forms[i]);
    if (s != ZC_OK) return s;
  }
  const int K = lanes_for(ctx, count);
  zc_status s = make_lanes(ctx, K);
  if (s != ZC_OK) return s;
  for (int k = 0; k < K; k++) std::memcpy(ctx->lanes[k]->tune, ctx->tune, sizeof(ctx->tune));
  const std::vector<int> lane = assign_lanes(count, forms, params, K);
  std::vector<size_t> need(K, 0);
  for (uint32_t i = 0; i < count; i++) {
    const size_t b = forms[i] != ZC_FORM_NTT
                         ? sumcheck_scratch_bytes(ctx, &params[i])
                         : ntt_scratch_bytes(&params[i], ctx->sm_count, q_direct ? q_direct[i] : false);
    need[lane[i]] = std::max(need[lane[i]], b);
    if (forms[i] == ZC_FORM_NTT) {
      s = ntt_prepare(ctx, &params[i], st);
      if (s != ZC_OK) return s;
    }
  }
  for (int k = 0; k < K; k++) {
    s = ensure_arena(ctx->lanes[k], need[k]);
    if (s != ZC_OK) {
      ctx->err = ctx->lanes[k]->err;
      return s;
    }
  }
  return cudaDeviceSynchronize() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

// Enqueue every instance (columns, proofs and q on the device); forks from
// st to the lanes and joins back.  Capture-safe once prepared.
zc_status batch_enqueue(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                        const void* const* const* cols, cudaStream_t st, uint8_t* const* proofs,
                        void* const* q_outs) {
  const int K = lanes_for(ctx, count);
  if ((int)ctx->lanes.size() < K) {
    ctx->err = "batch not prepared";
    return ZC_ERR_ARG;
  }
  const std::vector<int> lane = assign_lanes(count, forms, params, K);
  ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->fork_ev, st));
  for (int k = 0; k < K; k++) ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->lane_streams[k], ctx->fork_ev, 0));
  uint32_t launches = 0;
  struct Freeze {
    zc_ctx* c;
    ~Freeze() { c->ntt_cache_frozen = false; }
  } freeze{ctx};
  ctx->ntt_cache_frozen = true;
  for (int k = 0; k < K; k++) {
    zc_ctx* L = ctx->lanes[k];
    for (uint32_t i = 0; i < count; i++) {
      if (lane[i] != k) continue;
      zc_status s;
      if (forms[i] != ZC_FORM_NTT)
        s = sumcheck_prove(L, &params[i], cols[i], 1, nullptr, ctx->lane_streams[k], proofs[i], true,
                           forms[i] == ZC_FORM_SUMCHECK_EQ);
      else
        s = ntt_prove(L, &params[i], cols[i], 1, nullptr, ctx->lane_streams[k], proofs[i], true,
                      q_outs ? q_outs[i] : nullptr, 1);
      launches += L->launches;
      if (s != ZC_OK) {
        ctx->err = L->err;
        return s;
      }
    }
    ZC_CUDA_TRY(ctx, cudaEventRecord(ctx->lane_join[k], ctx->lane_streams[k]));
    ZC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->lane_join[k], 0));
  }
  ctx->launches = launches;
  ctx->nev = 0;
  return ZC_OK;
}

void destroy_lanes(zc_ctx* ctx) {
  for (size_t k = 0; k < ctx->lanes.size(); k++) {
    zc_ctx* L = ctx->lanes[k];
    if (L->arena.base && !L->arena_borrowed) cudaFree(L->arena.base);
    if (L->pinned) cudaFreeHost(L->pinned);
    for (int i = 0; i < 8; i++)
      if (L->ev[i]) cudaEventDestroy(L->ev[i]);
    delete L;
    cudaStreamDestroy(ctx->lane_streams[k]);
    cudaEventDestroy(ctx->lane_join[k]);
  }
  ctx->lanes.clear();
  ctx->lane_streams.clear();
  ctx->lane_join.clear();
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  ctx->fork_ev = nullptr;
}

}  // namespace zc

struct zc_batch {
  zc_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  uint32_t count = 0;
  uint32_t launches = 0;
};

using namespace zc;

static zc_status check_batch_args(zc_ctx* ctx, uint32_t count, const zc_form* forms,
                                  const zc_params* params, const void* const* const* cols,
                                  uint8_t* const* proofs) {
  if (!ctx || !forms || !params || !cols || !proofs || count == 0) return ZC_ERR_ARG;
  for (uint32_t i = 0; i < count; i++) {
    if (forms[i] != ZC_FORM_SUMCHECK && forms[i] != ZC_FORM_NTT && forms[i] != ZC_FORM_SUMCHECK_EQ)
      return ZC_ERR_ARG;
    const int c = gate_ncols(params[i].gate, params[i].d);
    if (c < 0 || !cols[i] || !proofs[i]) return ZC_ERR_ARG;
    for (int j = 0; j < c; j++)
      if (!cols[i][j]) return ZC_ERR_ARG;
  }
  return ZC_OK;
}

extern "C" {

zc_status zc_prove_batch(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                         const void* const* const* cols, void* cuda_stream, uint8_t* const* proofs,
                         void* const* q_outs) {
  zc_status s = check_batch_args(ctx, count, forms, params, cols, proofs);
  if (s != ZC_OK) return s;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<char> qd(count, 0);
  for (uint32_t i = 0; i < count; i++) qd[i] = (q_outs && q_outs[i]) ? 1 : 0;
  s = batch_prepare(ctx, count, forms, params, reinterpret_cast<const bool*>(qd.data()), st);
  if (s != ZC_OK) return s;
  return batch_enqueue(ctx, count, forms, params, cols, st, proofs, q_outs);
}

zc_status zc_batch_create(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                          const void* const* const* cols, uint8_t* const* proofs, void* const* q_outs,
                          zc_batch** out) {
  if (!out) return ZC_ERR_ARG;
  *out = nullptr;
  zc_status s = check_batch_args(ctx, count, forms, params, cols, proofs);
  if (s != ZC_OK) return s;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  zc_batch* b = new zc_batch();
  b->ctx = ctx;
  b->count = count;
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return ZC_ERR_CUDA;
  }
  std::vector<char> qd(count, 0);
  for (uint32_t i = 0; i < count; i++) qd[i] = (q_outs && q_outs[i]) ? 1 : 0;
  s = batch_prepare(ctx, count, forms, params, reinterpret_cast<const bool*>(qd.data()), b->capture);
  if (s == ZC_OK) {
    if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      s = ZC_ERR_CUDA;
    } else {
      s = batch_enqueue(ctx, count, forms, params, cols, b->capture, proofs, q_outs);
      b->launches = ctx->launches;
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
      if (s == ZC_OK && e != cudaSuccess) s = ZC_ERR_CUDA;
      b->graph = g;
      if (s == ZC_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) s = ZC_ERR_CUDA;
    }
  }
  if (s != ZC_OK) {
    cudaGetLastError();
    if (ctx->err.empty()) ctx->err = "batch graph capture failed";
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaStreamDestroy(b->capture);
    delete b;
    return s;
  }
  *out = b;
  return ZC_OK;
}

zc_status zc_batch_launch(zc_batch* b, void* cuda_stream) {
  if (!b || !b->exec) return ZC_ERR_ARG;
  if (cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) {
    cudaGetLastError();
    return ZC_ERR_CUDA;
  }
  b->ctx->launches = b->launches;
  return ZC_OK;
}

uint32_t zc_batch_kernels(const zc_batch* b) { return b ? b->launches : 0; }

void zc_batch_destroy(zc_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->capture);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaStreamDestroy(b->capture);
  delete b;
}

}  // extern "C"
