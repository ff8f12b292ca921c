// zc_serve.cu -- the request loop: admission by free slot and device-pool
// space, continuous batching over streams, completion by event polling.
//
// The paper proves one ZeroCheck instance at a time; serving runs many of
// them as they arrive.  The host thread is the scheduler: requests become
// visible at their arrival time, wait in arrival order, and are admitted
// when a slot (child context + stream) is free and a first-fit block of the
// device pool holds their scratch (the per-proof tables, folded columns,
// quotient and transcript state).  Completion is observed with an event
// query; the block and the slot then go to the next waiting request, so new
// proofs start while earlier ones are still on the GPU.  Nothing is
// allocated while the loop runs: the pool is allocated once and kept, the
// NTT tables of every size in the request list are built beforehand.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <thread>

#include "zc_internal.cuh"

namespace zc {

constexpr size_t kPoolAlign = 2u << 20;
constexpr uint32_t kMaxSlots = 64;

// First-fit allocator over one device region (host bookkeeping only).
class PoolAlloc {
 public:
  explicit PoolAlloc(size_t cap) {
    if (cap) free_[0] = cap;
  }
  size_t take(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > bytes) free_[off + bytes] = sz - bytes;
      return off;
    }
    return SIZE_MAX;
  }
  void give(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;  // offset -> length
};

void destroy_serve_pool(zc_ctx* ctx) {
  if (ctx->serve_pool) cudaFree(ctx->serve_pool);
  ctx->serve_pool = nullptr;
  ctx->serve_pool_cap = 0;
}

static zc_status proof_scratch(zc_ctx* ctx, const zc_params* p, zc_form form, bool q_dev, size_t* out) {
  zc_status s = check_params(ctx, p, form);
  if (s != ZC_OK) return s;
  *out = form != ZC_FORM_NTT ? sumcheck_scratch_bytes(ctx, p) : ntt_scratch_bytes(p, ctx->sm_count, q_dev);
  return ZC_OK;
}

static void release_lane_arenas(zc_ctx* ctx) {
  for (zc_ctx* L : ctx->lanes) {
    if (L->arena_borrowed) {
      L->arena.base = nullptr;
      L->arena.cap = 0;
      L->arena.used = 0;
      L->arena_borrowed = false;
    }
  }
}

}  // namespace zc

using namespace zc;

extern "C" {

zc_status zc_scratch_bytes(zc_ctx* ctx, const zc_params* params, zc_form form, int q_on_device,
                           size_t* bytes) {
  if (!ctx || !params || !bytes) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  return proof_scratch(ctx, params, form, q_on_device != 0, bytes);
}

zc_status zc_serve(zc_ctx* ctx, const zc_request* reqs, uint32_t count, const zc_serve_opts* o,
                   zc_result* res) {
  using clock = std::chrono::steady_clock;
  if (!ctx || !o || (count && (!reqs || !res))) return ZC_ERR_ARG;
  if (o->slots < 1 || o->slots > kMaxSlots || o->hbm_budget_bytes < kPoolAlign) return ZC_ERR_ARG;
  if (!(o->timeout_s >= 0)) return ZC_ERR_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  ZC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));

  // validate and size every request before anything runs
  std::vector<size_t> fp(count);
  for (uint32_t i = 0; i < count; i++) {
    const zc_request& r = reqs[i];
    std::memset(&res[i], 0, sizeof(zc_result));
    res[i].admit_s = res[i].done_s = -1.0;
    if (!(r.arrival_s >= 0) || !std::isfinite(r.arrival_s) || !r.cols || !r.proof) return ZC_ERR_ARG;
    size_t b = 0;
    zc_status s = proof_scratch(ctx, &r.params, r.form, r.q_out != nullptr, &b);
    if (s != ZC_OK) return s;
    const int c = gate_ncols(r.params.gate, r.params.d);
    for (int j = 0; j < c; j++)
      if (!r.cols[j]) return ZC_ERR_ARG;
    fp[i] = align_up(b, kPoolAlign);
  }

  const size_t budget = align_up(o->hbm_budget_bytes, kPoolAlign);
  if (ctx->serve_pool_cap != budget) {
    ZC_CUDA_TRY(ctx, cudaDeviceSynchronize());
    destroy_serve_pool(ctx);
    if (cudaMalloc(&ctx->serve_pool, budget) != cudaSuccess) {
      cudaGetLastError();
      ctx->serve_pool = nullptr;
      ctx->err = "cudaMalloc of the serving pool failed";
      return ZC_ERR_OOM;
    }
    ctx->serve_pool_cap = budget;
  }
  const int K = (int)o->slots;
  zc_status s = make_lanes(ctx, K);
  if (s != ZC_OK) return s;
  for (int k = 0; k < K; k++) {
    zc_ctx* L = ctx->lanes[k];
    std::memcpy(L->tune, ctx->tune, sizeof(ctx->tune));
    if (L->arena.base && !L->arena_borrowed) cudaFree(L->arena.base);
    L->arena.base = nullptr;
    L->arena.cap = 0;
    L->arena_borrowed = true;
  }
  cudaStream_t prep = ctx->lane_streams[0];
  for (uint32_t i = 0; i < count; i++) {
    if (reqs[i].form != ZC_FORM_NTT || fp[i] > budget) continue;
    s = ntt_prepare(ctx, &reqs[i].params, prep);
    if (s != ZC_OK) {
      release_lane_arenas(ctx);
      return s;
    }
  }
  std::vector<cudaEvent_t> done(K, nullptr);
  for (int k = 0; k < K; k++) cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    for (auto e : done) cudaEventDestroy(e);
    release_lane_arenas(ctx);
    ctx->err = "device error before the serving loop";
    return ZC_ERR_CUDA;
  }

  std::vector<uint32_t> order(count);
  for (uint32_t i = 0; i < count; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return reqs[a].arrival_s < reqs[b].arrival_s; });

  PoolAlloc pool(budget);
  char* base = static_cast<char*>(ctx->serve_pool);
  std::vector<int64_t> slot_req(K, -1);
  std::vector<size_t> slot_off(K, 0);
  std::deque<uint32_t> waiting;
  size_t next = 0;
  uint32_t completed = 0, launches = 0;
  zc_status first_err = ZC_OK;
  struct Freeze {
    zc_ctx* c;
    ~Freeze() { c->ntt_cache_frozen = false; }
  } freeze{ctx};
  ctx->ntt_cache_frozen = true;

  const auto t0 = clock::now();
  auto now_s = [&]() { return std::chrono::duration<double>(clock::now() - t0).count(); };
  bool timed_out = false;
  while (completed < count) {
    const double now = now_s();
    if (o->timeout_s > 0 && now > o->timeout_s) {
      timed_out = true;
      break;
    }
    bool progress = false;
    while (next < count && reqs[order[next]].arrival_s <= now) {
      const uint32_t i = order[next++];
      if (fp[i] > budget) {  // can never fit: fails alone
        res[i].status = ZC_ERR_OOM;
        res[i].scratch_bytes = fp[i];
        res[i].admit_s = res[i].done_s = now;
        completed++;
        if (first_err == ZC_OK) first_err = ZC_ERR_OOM;
        continue;
      }
      waiting.push_back(i);
      progress = true;
    }
    // completions
    for (int k = 0; k < K; k++) {
      if (slot_req[k] < 0) continue;
      const cudaError_t q = cudaEventQuery(done[k]);
      if (q == cudaErrorNotReady) continue;
      const uint32_t i = (uint32_t)slot_req[k];
      res[i].done_s = now_s();
      if (q != cudaSuccess) {
        res[i].status = ZC_ERR_CUDA;
        if (first_err == ZC_OK) {
          first_err = ZC_ERR_CUDA;
          ctx->err = std::string("serving: ") + cudaGetErrorString(q);
        }
      }
      pool.give(slot_off[k], fp[i]);
      slot_req[k] = -1;
      completed++;
      progress = true;
    }
    // admissions: with priority_bytes set, a request whose scratch is at
    // least that large runs on slot 0 (the greatest stream priority), one
    // such request at a time in arrival order, and the others use slots
    // 1..K-1, so small proofs fill the GPU around a large one instead of
    // waiting behind it or slowing it down
    const bool prio = o->priority_bytes > 0 && K > 1;
    for (auto it = waiting.begin(); it != waiting.end();) {
      const uint32_t i = *it;
      const bool big = prio && fp[i] >= o->priority_bytes;
      int k = prio && !big ? 1 : 0;
      if (big) k = slot_req[0] >= 0 ? K : 0;
      else
        while (k < K && slot_req[k] >= 0) k++;
      if (k == K) {
        if (o->in_order || !prio) break;
        ++it;
        continue;
      }
      const size_t off = pool.take(fp[i]);
      if (off == SIZE_MAX) {
        res[i].waited_for_memory = 1;
        if (o->in_order) break;
        ++it;
        continue;
      }
      const zc_request& r = reqs[i];
      zc_ctx* L = ctx->lanes[k];
      L->arena.base = base + off;
      L->arena.cap = fp[i];
      L->arena.used = 0;
      res[i].admit_s = now_s();
      res[i].scratch_bytes = fp[i];
      res[i].slot = (uint32_t)k;
      zc_status ps;
      if (r.form != ZC_FORM_NTT)
        ps = sumcheck_prove(L, &r.params, r.cols, 1, nullptr, ctx->lane_streams[k], r.proof, true,
                            r.form == ZC_FORM_SUMCHECK_EQ);
      else
        ps = ntt_prove(L, &r.params, r.cols, 1, nullptr, ctx->lane_streams[k], r.proof, true, r.q_out, 1);
      launches += L->launches;
      if (ps == ZC_OK && cudaEventRecord(done[k], ctx->lane_streams[k]) != cudaSuccess) ps = ZC_ERR_CUDA;
      if (ps != ZC_OK) {
        // nothing of it is in flight unless a launch was queued: wait for the lane, then free
        cudaStreamSynchronize(ctx->lane_streams[k]);
        cudaGetLastError();
        res[i].status = ps;
        res[i].done_s = now_s();
        if (first_err == ZC_OK) {
          first_err = ps;
          ctx->err = "serving: " + L->err;
        }
        pool.give(off, fp[i]);
        completed++;
      } else {
        slot_req[k] = i;
        slot_off[k] = off;
      }
      it = waiting.erase(it);
      progress = true;
    }
    if (!progress) {
      bool busy = false;
      for (int k = 0; k < K; k++) busy |= slot_req[k] >= 0;
      if (!busy && waiting.empty() && next < count) {
        // idle until the next arrival (at most 1 ms at a time)
        const double wait = std::min(reqs[order[next]].arrival_s - now_s(), 1e-3);
        if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
      } else {
        std::this_thread::yield();
      }
    }
  }
  if (timed_out) {
    for (int k = 0; k < K; k++)
      if (slot_req[k] >= 0) cudaStreamSynchronize(ctx->lane_streams[k]);
    for (uint32_t i = 0; i < count; i++)
      if (res[i].done_s < 0) res[i].status = ZC_ERR_TIMEOUT;
    if (first_err == ZC_OK) {
      first_err = ZC_ERR_TIMEOUT;
      ctx->err = "serving loop timed out";
    }
  }
  for (auto e : done) cudaEventDestroy(e);
  release_lane_arenas(ctx);
  ctx->launches = launches;
  ctx->nev = 0;
  return first_err;
}

}  // extern "C"
