// pq_serve.cu -- continuous-batching serving loop and the autotuner.
//
// Requests (plans over resident tables) queue in submission order.  A server
// thread owns `serve_slots` streams; whenever a stream is free it admits the
// queued requests that fit the arena (up to kMaxBatch), runs them as one batch
// (pq_run_batch's persistent kernels) and goes back to admitting, so requests
// that arrive while earlier batches are on the GPU start as soon as a slot and
// memory are free and overlap with them on the device.  D-sets are cached
// across requests (hash tables kept resident).  Completion is signalled by a
// host callback enqueued after each batch, so no thread polls the GPU.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "pq_plan_host.h"

using namespace pqk;

namespace pqh {

namespace {
constexpr int kMaxBatch = 512;
using Clock = std::chrono::steady_clock;
}  // namespace

struct Request {
  uint64_t ticket;
  pq_plan plan;
  size_t bytes;
  Clock::time_point t0;
};

struct Finished {
  pq_result res;
  double latency_us;
};

struct ServeSlot {
  cudaStream_t s = nullptr;
  pq_result* results = nullptr;  // pinned, kMaxBatch entries
  std::vector<Request> reqs;
  // busy: the slot holds a batch; it is set, together with reqs, under the
  // server's lock BEFORE the batch is enqueued, and the completion callback
  // only ever sets `completed`, so a batch that finishes before the server
  // thread re-takes the lock is still delivered.
  bool busy = false;
  bool completed = false;
  struct Server* srv = nullptr;
};

struct Server {
  pq_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv;       // wakes the server thread
  std::condition_variable cv_done;  // wakes pq_poll callers
  std::deque<Request> pending;
  std::unordered_map<uint64_t, Finished> done;
  std::vector<ServeSlot> slots;
  std::thread th;
  bool stop = false;
  Clock::time_point stop_by;        // deadline for the batches in flight at stop
  bool abandoned = false;           // a batch was still in flight at the deadline
  bool budget_wait = false;         // admission waits for a batch to complete
  uint64_t next_ticket = 1;

  void loop();
  void finish(const std::vector<Request>& reqs, pq_status st);
};

static void CUDART_CB on_batch_done(void* arg) {
  ServeSlot* sl = (ServeSlot*)arg;
  {
    std::lock_guard<std::mutex> g(sl->srv->mu);
    sl->completed = true;
  }
  sl->srv->cv.notify_all();
}

// Requests that will not run: their tickets complete with status `st`.
// Called with `mu` held.
void Server::finish(const std::vector<Request>& reqs, pq_status st) {
  for (auto& r : reqs) {
    Finished f;
    memset(&f.res, 0, sizeof f.res);
    f.res.status = st;
    f.latency_us = 0;
    done[r.ticket] = f;
  }
  cv_done.notify_all();
}

void Server::loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    // Deliver finished batches.
    for (auto& sl : slots) {
      if (!sl.busy || !sl.completed) continue;
      const auto now = Clock::now();
      for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Finished f;
        f.res = sl.results[i];
        f.latency_us = std::chrono::duration<double, std::micro>(now - sl.reqs[i].t0).count();
        done[sl.reqs[i].ticket] = f;
      }
      sl.reqs.clear();
      sl.busy = sl.completed = false;
      budget_wait = false;
      cv_done.notify_all();
    }
    if (stop) {
      // Requests not yet admitted never run; batches in flight get until
      // the deadline.
      if (!pending.empty()) {
        finish(std::vector<Request>(pending.begin(), pending.end()), PQ_ERR_TIMEOUT);
        pending.clear();
      }
      bool any = false;
      for (auto& sl : slots) any = any || sl.busy;
      if (!any) return;
      if (Clock::now() >= stop_by) {
        abandoned = true;
        return;
      }
      cv.wait_until(lk, stop_by);
      continue;
    }
    ServeSlot* free_slot = nullptr;
    for (auto& sl : slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot || pending.empty() || budget_wait) {
      cv.wait(lk, [&] {
        if (stop) return true;
        bool any_free = false;
        for (auto& sl : slots) {
          if (sl.busy && sl.completed) return true;
          any_free = any_free || !sl.busy;
        }
        return any_free && !pending.empty() && !budget_wait;
      });
      continue;
    }
    // The arena's free space is read without the server's lock: the arena
    // may wait for the GPU, and the completion callbacks need this lock.
    lk.unlock();
    const size_t budget = ctx->arena.largest_free();
    lk.lock();
    if (stop || pending.empty()) continue;
    ServeSlot& sl = *free_slot;
    size_t used = batch_layout(kMaxBatch).end;
    std::vector<Request> take;
    // An aggregate-first request forms a batch of its own.
    auto agg = [](const Request& q) { return (q.plan.flags & PQ_PLAN_AGG_FIRST) != 0; };
    while (!pending.empty() && (int)take.size() < kMaxBatch &&
           (take.empty() || (used + pending.front().bytes <= budget && !agg(pending.front())))) {
      used += pending.front().bytes;
      take.push_back(pending.front());
      pending.pop_front();
      if (agg(take.back())) break;
    }
    std::vector<pq_plan> plans;
    for (auto& r : take) plans.push_back(r.plan);
    sl.reqs = std::move(take);
    sl.busy = true;
    sl.completed = false;
    lk.unlock();
    pq_status st = run_batch_internal(ctx, plans.data(), (int)plans.size(), sl.results, sl.s,
                                      false);
    bool callback = false;
    if (st == PQ_OK) {
      callback = cudaLaunchHostFunc(sl.s, on_batch_done, &sl) == cudaSuccess;
      if (!callback) st = PQ_ERR_CUDA;
    }
    lk.lock();
    if (callback) continue;  // the callback completes the slot
    // No callback will come: the slot is free again at once (its stream
    // keeps any work already queued in order before the next batch).
    std::vector<Request> reqs = std::move(sl.reqs);
    sl.reqs.clear();
    sl.busy = sl.completed = false;
    bool others_busy = false;
    for (auto& o : slots) others_busy = others_busy || o.busy;
    if (st == PQ_ERR_BUDGET && others_busy) {
      // Not enough memory while other batches hold it: requeue and admit
      // again once one of them completes.
      for (auto it = reqs.rbegin(); it != reqs.rend(); ++it) pending.push_front(*it);
      budget_wait = true;
      continue;
    }
    finish(reqs, st);
  }
}

// Stop the serving loop.  Batches in flight get kStopWaitMs to complete;
// if one does not, the server (its streams, pinned buffers and thread state,
// which a late completion callback would still touch) is left allocated and
// PQ_ERR_TIMEOUT returned, instead of waiting without end.
constexpr int kStopWaitMs = 30000;

pq_status server_stop(pq_ctx* ctx) {
  Server* srv = ctx->server;
  if (!srv) return PQ_OK;
  const auto deadline = Clock::now() + std::chrono::milliseconds(kStopWaitMs);
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    srv->stop_by = deadline;
  }
  srv->cv.notify_all();
  if (srv->th.joinable()) srv->th.join();
  ctx->server = nullptr;
  bool idle = !srv->abandoned;
  for (auto& sl : srv->slots) {
    while (idle && sl.s && cudaStreamQuery(sl.s) == cudaErrorNotReady) {
      if (Clock::now() >= deadline) idle = false;
      else std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  cudaGetLastError();
  if (!idle)
    return fail(ctx, PQ_ERR_TIMEOUT, "serving loop: a batch did not complete within %d ms",
                kStopWaitMs);
  for (auto& sl : srv->slots) {
    if (sl.s) cudaStreamDestroy(sl.s);
    if (sl.results) cudaFreeHost(sl.results);
  }
  delete srv;
  return PQ_OK;
}

static pq_status server_start(pq_ctx* ctx) {
  if (ctx->server) return PQ_OK;
  std::unique_ptr<Server> srv(new Server());
  srv->ctx = ctx;
  srv->slots.resize(std::max(1, ctx->opt.serve_slots));
  for (auto& sl : srv->slots) {
    sl.srv = srv.get();
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void**)&sl.results, sizeof(pq_result) * kMaxBatch, 0) != cudaSuccess) {
      for (auto& o : srv->slots) {
        if (o.s) cudaStreamDestroy(o.s);
        if (o.results) cudaFreeHost(o.results);
      }
      return fail(ctx, PQ_ERR_CUDA, "serving loop: stream or pinned buffer");
    }
  }
  Server* raw = srv.release();
  ctx->server = raw;
  raw->th = std::thread([raw] {
    cudaSetDevice(raw->ctx->device);
    raw->loop();
  });
  return PQ_OK;
}

}  // namespace pqh

using namespace pqh;

extern "C" {

pq_status pq_submit(pq_ctx* ctx, const pq_plan* plan, uint64_t* ticket) {
  if (!ctx || !plan || !ticket) return PQ_ERR_INVALID_ARG;
  ResolvedPlan r;
  const bool agg = plan->flags & PQ_PLAN_AGG_FIRST;
  pq_status st = resolve_plan(ctx, *plan, r, agg);
  if (st != PQ_OK) return st;
  const bool streamed = !r.resident[0] || !r.resident[1] || !r.resident[2];
  // An aggregate-first plan is checked here (resident tables, dense keys) and
  // later runs in a batch of its own.
  size_t agg_bytes = 0;
  if (agg && (st = aggfirst_bytes(ctx, *plan, &agg_bytes)) != PQ_OK) return st;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    st = server_start(ctx);
  }
  if (st != PQ_OK) return st;
  Server* srv = ctx->server;
  Request q;
  q.plan = *plan;
  if (!agg) q.plan.flags |= PQ_PLAN_CACHE_DSET;
  // A batch of streamed plans also holds the chunk ring: a share of it per
  // request (a batch that still does not fit is retried when others finish).
  q.bytes = agg ? agg_bytes
                : plan_bytes(r) + 256 +
                      (streamed ? (size_t)std::max(2, ctx->opt.ring_slots) *
                                      (size_t)(2 * ctx->opt.chunk_bytes) / 8
                                : 0);
  q.t0 = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if ((int)srv->pending.size() >= ctx->opt.serve_queue)
      return fail(ctx, PQ_ERR_BUSY, "serving queue holds %d requests", ctx->opt.serve_queue);
    q.ticket = srv->next_ticket++;
    srv->pending.push_back(q);
  }
  srv->cv.notify_all();
  *ticket = q.ticket;
  return PQ_OK;
}

pq_status pq_poll(pq_ctx* ctx, uint64_t ticket, pq_result* result, int timeout_ms) {
  if (!ctx || !result) return PQ_ERR_INVALID_ARG;
  Server* srv = ctx->server;
  if (!srv) return fail(ctx, PQ_ERR_INVALID_ARG, "no request was submitted");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto ready = [&] { return srv->done.count(ticket) > 0; };
  if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
  else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return PQ_ERR_TIMEOUT;
  Finished f = srv->done[ticket];
  srv->done.erase(ticket);
  lk.unlock();
  *result = f.res;
  ctx->last_latency_us = f.latency_us;
  return (pq_status)(f.res.status == PQ_OK ? PQ_OK : f.res.status);
}

double pq_last_latency_us(pq_ctx* ctx) { return ctx ? ctx->last_latency_us : 0.0; }

pq_status pq_autotune(pq_ctx* ctx, const pq_plan* sample, pq_tuning* out) {
  if (!ctx || !sample || !out) return PQ_ERR_INVALID_ARG;
  if (sample->flags & PQ_PLAN_AGG_FIRST)
    return fail(ctx, PQ_ERR_INVALID_ARG, "autotune: the join-first plan only");
  ResolvedPlan r;
  pq_status st = resolve_plan(ctx, *sample, r, true);
  if (st != PQ_OK) return st;
  cudaStream_t s;
  PQ_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  pq_result* res = nullptr;
  cudaEvent_t a, b;
  if (cudaHostAlloc((void**)&res, sizeof(pq_result), 0) != cudaSuccess ||
      cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    cudaStreamDestroy(s);
    return fail(ctx, PQ_ERR_CUDA, "autotune setup");
  }
  const int saved_bps = ctx->tune_bps;
  memset(out, 0, sizeof *out);
  out->best_ms = 1e30f;
  // Median time of plan p under blocks-per-SM `bps` (first run untimed).
  auto measure = [&](const pq_plan& p, int bps, float* ms_out) -> pq_status {
    ctx->tune_bps = bps;
    float t[5];
    int ok = 0;
    for (int rep = 0; rep < 6; ++rep) {
      cudaEventRecord(a, s);
      pq_status e = run_batch_internal(ctx, &p, 1, res, s, false);
      cudaEventRecord(b, s);
      if (e != PQ_OK) return e;
      if (cudaEventSynchronize(b) != cudaSuccess) return PQ_ERR_CUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) t[ok++] = ms;  // the first run warms caches and code
    }
    std::sort(t, t + ok);
    *ms_out = t[ok / 2];
    return PQ_OK;
  };
  pq_plan p = *sample;
  p.flags = (p.flags | PQ_PLAN_NO_GRAPH) & ~PQ_PLAN_PARTITIONED;
  p.log2P = 0;
  p.load_factor = sample->load_factor > 0 ? sample->load_factor : ctx->opt.load_factor;
  int best_bps = std::max(1, saved_bps), best_lp = 0;
  float best_lf = p.load_factor, best = 1e30f;
  auto consider = [&](float ms, int bps, float lf, int lp) {
    out->tried++;
    if (ms < best) best = ms, best_bps = bps, best_lf = lf, best_lp = lp;
  };
  // Coordinate descent: resident blocks per SM of the persistent kernels,
  // then the hash-table load factor, then the partition fan-out (2^0 = not
  // partitioned), each swept with the best settings found so far.
  const int bps_set[] = {1, 2, 3, 4, 6, 8};
  const float lf_set[] = {0.25f, 0.4f, 0.5f, 0.7f};
  const int lp_set[] = {4, 6, 8, 10};
  for (int bps : bps_set) {
    float ms;
    if ((st = measure(p, bps, &ms)) != PQ_OK) break;
    consider(ms, bps, p.load_factor, 0);
  }
  for (float lf : lf_set) {
    if (st != PQ_OK) break;
    pq_plan q = p;
    q.load_factor = lf;
    float ms;
    if ((st = measure(q, best_bps, &ms)) != PQ_OK) break;
    consider(ms, best_bps, lf, 0);
  }
  for (int lp : lp_set) {
    if (st != PQ_OK) break;
    pq_plan q = p;
    q.load_factor = best_lf;
    q.flags |= PQ_PLAN_PARTITIONED;
    q.log2P = lp;
    float ms;
    if ((st = measure(q, best_bps, &ms)) != PQ_OK) break;
    consider(ms, best_bps, best_lf, lp);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeHost(res);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st != PQ_OK) {
    ctx->tune_bps = saved_bps;
    return st;
  }
  out->block_threads = 256;  // fixed: the plan kernels are written for 8 warps
  out->blocks_per_sm = best_bps;
  out->load_factor = best_lf;
  out->partitioned = best_lp > 0 ? 1 : 0;
  out->log2P = best_lp > 0 ? best_lp : ctx->opt.log2P;
  out->best_ms = best;
  ctx->tune_bps = best_bps;
  ctx->opt.blocks_per_sm = best_bps;
  ctx->opt.load_factor = best_lf;
  if (best_lp > 0) ctx->opt.log2P = best_lp;
  return PQ_OK;
}

}  // extern "C"
