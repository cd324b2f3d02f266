// pq_core.cu -- context, arena allocator, status word, tables, profiling.
#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "pq_internal.h"

using namespace pqh;
using pqk::i64;

namespace pqh {

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- Arena ----
void Arena::init(char* base, size_t bytes) {
  std::lock_guard<std::mutex> g(mu_);
  base_ = base;
  cap_ = bytes;
  free_.clear();
  live_.clear();
  if (bytes) free_[0] = bytes;
  in_use_ = high_ = 0;
}

void Arena::shutdown() {
  std::lock_guard<std::mutex> g(mu_);
  for (auto& p : pending_) cudaEventSynchronize(p.ev), events_.push_back(p.ev);
  pending_.clear();
  for (auto e : events_) cudaEventDestroy(e);
  events_.clear();
}

void Arena::insert_free(size_t off, size_t size) {
  auto next = free_.lower_bound(off);
  if (next != free_.end() && off + size == next->first) {
    size += next->second;
    next = free_.erase(next);
  }
  if (next != free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      prev->second += size;
      return;
    }
  }
  free_[off] = size;
}

void Arena::reclaim(bool wait_one) {
  while (!pending_.empty()) {
    Pending& p = pending_.front();
    if (wait_one) {
      cudaEventSynchronize(p.ev);
      wait_one = false;
    } else if (cudaEventQuery(p.ev) != cudaSuccess) {
      break;
    }
    insert_free(p.off, p.size);
    in_use_ -= p.size;
    events_.push_back(p.ev);
    pending_.pop_front();
  }
}

void* Arena::alloc(size_t bytes, size_t align) {
  std::lock_guard<std::mutex> g(mu_);
  bytes = round_up(bytes ? bytes : 1, 256);
  align = std::max<size_t>(align, 256);
  reclaim(false);
  while (true) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      const size_t off = it->first, size = it->second;
      const size_t a = round_up((size_t)(base_ + off), align) - (size_t)base_;
      if (a + bytes <= off + size) {
        free_.erase(it);
        if (a > off) free_[off] = a - off;
        if (a + bytes < off + size) free_[a + bytes] = off + size - (a + bytes);
        live_[a] = bytes;
        in_use_ += bytes;
        high_ = std::max(high_, in_use_);
        return base_ + a;
      }
    }
    if (pending_.empty()) return nullptr;
    reclaim(true);
  }
}

size_t Arena::largest_free() {
  std::lock_guard<std::mutex> g(mu_);
  reclaim(false);
  size_t best = 0;
  for (auto& kv : free_) best = std::max(best, kv.second);
  return best;
}

void Arena::release_now(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu_);
  size_t off = (char*)p - base_;
  auto it = live_.find(off);
  if (it == live_.end()) return;
  size_t size = it->second;
  live_.erase(it);
  insert_free(off, size);
  in_use_ -= size;
}

void Arena::release(void* p, cudaStream_t s) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu_);
  size_t off = (char*)p - base_;
  auto it = live_.find(off);
  if (it == live_.end()) return;
  size_t size = it->second;
  live_.erase(it);
  cudaEvent_t ev;
  if (!events_.empty()) {
    ev = events_.back();
    events_.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamSynchronize(s);
    insert_free(off, size);
    in_use_ -= size;
    return;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone || cudaEventRecord(ev, s) != cudaSuccess) {
    // Never free inside a capture: keep the block until the context is reset.
    events_.push_back(ev);
    live_[off] = size;
    return;
  }
  pending_.push_back({off, size, ev});
}

// ----------------------------------------------------------- PinnedRing ----
bool PinnedRing::init(size_t slot_bytes, int slots) {
  slot_ = slot_bytes;
  n_ = slots;
  if (cudaHostAlloc((void**)&host_, slot_ * n_, cudaHostAllocDefault) != cudaSuccess) return false;
  ev_.resize(n_);
  for (int i = 0; i < n_; ++i)
    if (cudaEventCreateWithFlags(&ev_[i], cudaEventDisableTiming) != cudaSuccess) return false;
  for (int i = 0; i < n_; ++i) cudaEventRecord(ev_[i], 0);
  return true;
}

void PinnedRing::shutdown() {
  for (auto e : ev_) cudaEventSynchronize(e), cudaEventDestroy(e);
  ev_.clear();
  if (host_) cudaFreeHost(host_);
  host_ = nullptr;
}

cudaError_t PinnedRing::upload(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  std::lock_guard<std::mutex> g(mu_);
  char* at = (char*)src;
  while (bytes) {
    size_t b = std::min(bytes, slot_);
    int k = next_;
    next_ = (next_ + 1) % n_;
    cudaError_t e = cudaEventSynchronize(ev_[k]);
    if (e != cudaSuccess) return e;
    memcpy(host_ + k * slot_, at, b);
    e = cudaMemcpyAsync(dst, host_ + k * slot_, b, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev_[k], s);
    if (e != cudaSuccess) return e;
    dst = (char*)dst + b;
    at += b;
    bytes -= b;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------- helpers ----
pq_status fail(pq_ctx* ctx, pq_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = std::string(pq_status_string(st)) + ": " + buf;
  }
  return st;
}

SmallPinned::SmallPinned(pq_ctx* c) : ctx(c) {
  {
    std::lock_guard<std::mutex> g(ctx->small_mu);
    if (!ctx->small_free.empty()) {
      p = ctx->small_free.back();
      ctx->small_free.pop_back();
      return;
    }
  }
  own = cudaHostAlloc((void**)&p, kSmallBytes, 0) == cudaSuccess;
  if (!own) p = nullptr, cudaGetLastError();
}

SmallPinned::~SmallPinned() {
  if (!p) return;
  if (own) {
    cudaFreeHost(p);
    return;
  }
  std::lock_guard<std::mutex> g(ctx->small_mu);
  ctx->small_free.push_back(p);
}

pq_status cuda_fail(pq_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, PQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t dtype_size(int type) {
  switch (type) {
    case PQ_INT8: return 1;
    case PQ_INT32: return 4;
    case PQ_INT64: return 8;
  }
  return 0;
}

bool valid_dtype(int type) { return type == PQ_INT8 || type == PQ_INT32 || type == PQ_INT64; }

pqk::Pred make_pred(int op, int64_t c, bool* ok) {
  pqk::Pred p{INT64_MIN, INT64_MAX, 0, 0};
  *ok = true;
  switch (op) {
    case PQ_LT:
      if (c == INT64_MIN) p.lo = 1, p.hi = 0;  // empty
      else p.hi = c - 1;
      break;
    case PQ_LE: p.hi = c; break;
    case PQ_GT:
      if (c == INT64_MAX) p.lo = 1, p.hi = 0;
      else p.lo = c + 1;
      break;
    case PQ_GE: p.lo = c; break;
    case PQ_EQ: p.lo = p.hi = c; break;
    case PQ_NE: p.lo = p.hi = c, p.neg = 1; break;
    case PQ_ALL: break;
    default: *ok = false;
  }
  return p;
}

int grid_persistent(pq_ctx* ctx, int threads) {
  int per_sm = ctx->tune_bps * 256 / std::max(threads, 32);
  return ctx->num_sms * std::max(per_sm, 1);
}

void prof_begin(pq_ctx* ctx, const char* name, cudaStream_t s, cudaEvent_t* stop_out) {
  *stop_out = nullptr;
  if (!ctx->opt.profile) return;
  std::lock_guard<std::mutex> g(ctx->mu);
  Profile& p = ctx->prof[name];
  if (p.used == p.pairs.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    p.pairs.push_back({a, b});
  }
  auto& pr = p.pairs[p.used++];
  cudaEventRecord(pr.first, s);
  *stop_out = pr.second;
}

void prof_end(cudaEvent_t stop, cudaStream_t s) {
  if (stop) cudaEventRecord(stop, s);
}

void prof_collect(pq_ctx* ctx) {
  for (auto& kv : ctx->prof) {
    Profile& p = kv.second;
    for (size_t i = 0; i < p.used; ++i) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p.pairs[i].first, p.pairs[i].second) == cudaSuccess) {
        p.total_ms += ms;
        p.launches++;
      }
    }
    p.used = 0;
  }
}

}  // namespace pqh

// -------------------------------------------------------- device status ----
__global__ void k_take_status(pqk::DevStatus* st, pqk::DevStatus* out) {
  int code = atomicExch(&st->code, 0);
  out->code = code;
  out->detail = (long long)atomicExch((unsigned long long*)&st->detail, 0ULL);
}

// ------------------------------------------------------------------ C ABI ----
extern "C" {

const char* pq_status_string(int s) {
  switch (s) {
    case PQ_OK: return "PQ_OK";
    case PQ_ERR_INVALID_ARG: return "PQ_ERR_INVALID_ARG";
    case PQ_ERR_BUDGET: return "PQ_ERR_BUDGET";
    case PQ_ERR_CAPACITY: return "PQ_ERR_CAPACITY";
    case PQ_ERR_CUDA: return "PQ_ERR_CUDA";
    case PQ_ERR_IO: return "PQ_ERR_IO";
    case PQ_ERR_TIMEOUT: return "PQ_ERR_TIMEOUT";
    case PQ_ERR_OVERFLOW: return "PQ_ERR_OVERFLOW";
    case PQ_ERR_BUSY: return "PQ_ERR_BUSY";
    case PQ_ERR_RESERVED_KEY: return "PQ_ERR_RESERVED_KEY";
  }
  return "PQ_ERR_UNKNOWN";
}

pq_status pq_default_options(pq_options* o) {
  if (!o) return PQ_ERR_INVALID_ARG;
  memset(o, 0, sizeof *o);
  o->block_threads = 256;
  o->blocks_per_sm = 4;
  o->load_factor = 0.5f;
  o->log2P = 6;
  o->chunk_bytes = 128ll << 20;
  o->ingest_threads = 4;
  o->copy_streams = 2;
  o->ring_slots = 4;
  o->serve_slots = 4;
  o->spin_limit = 1ll << 22;
  o->serve_queue = 4096;
  o->profile = 0;
  o->hit_buffer = 16;
  return PQ_OK;
}

pq_status pq_create(const pq_options* opt, void* arena, size_t arena_bytes, pq_ctx** out) {
  if (!out) return PQ_ERR_INVALID_ARG;
  *out = nullptr;
  if (!arena || arena_bytes < (1u << 20)) return PQ_ERR_INVALID_ARG;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, arena) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return PQ_ERR_INVALID_ARG;
  }
  auto* ctx = new pq_ctx();
  pq_default_options(&ctx->opt);
  if (opt) {
    pq_options d = ctx->opt;
    pq_options o = *opt;
#define PQ_OPT(f) \
  if (o.f > 0) d.f = o.f;
    PQ_OPT(block_threads) PQ_OPT(blocks_per_sm) PQ_OPT(load_factor) PQ_OPT(log2P)
    PQ_OPT(chunk_bytes) PQ_OPT(ingest_threads) PQ_OPT(copy_streams) PQ_OPT(ring_slots)
    PQ_OPT(serve_slots) PQ_OPT(spin_limit) PQ_OPT(serve_queue)
#undef PQ_OPT
    d.profile = o.profile;
    if (o.hit_buffer > 0 || o.hit_buffer == -1) d.hit_buffer = o.hit_buffer;
    ctx->opt = d;
  }
  pq_options& o = ctx->opt;
  if (o.block_threads % 32 || o.block_threads > 1024 || o.load_factor < 0.05f ||
      o.load_factor > 0.9f || o.log2P > PQ_MAX_LOG2P || o.chunk_bytes < (1 << 20)) {
    delete ctx;
    return PQ_ERR_INVALID_ARG;
  }
  o.chunk_bytes = o.chunk_bytes / 4096 * 4096;
  ctx->tune_threads = o.block_threads;
  ctx->tune_bps = o.blocks_per_sm;
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
          cudaSuccess) {
    delete ctx;
    return PQ_ERR_CUDA;
  }
  ctx->arena.init((char*)arena, arena_bytes);
  ctx->d_status = (pqk::DevStatus*)ctx->arena.alloc(2 * sizeof(pqk::DevStatus));
  bool ok = ctx->d_status &&
            cudaHostAlloc((void**)&ctx->h_status, sizeof(pqk::DevStatus), 0) == cudaSuccess &&
            cudaHostAlloc((void**)&ctx->h_small, kSmallBytes * kSmallBufs, 0) == cudaSuccess &&
            cudaMemset(ctx->d_status, 0, 2 * sizeof(pqk::DevStatus)) == cudaSuccess &&
            ctx->ring.init(64 << 10, 32) && pqh::plan_kernels_init(ctx) == PQ_OK;
  for (int i = 0; ok && i < kSmallBufs; ++i)
    ctx->small_free.push_back(ctx->h_small + i * (kSmallBytes / 8));
  ok = ok && cudaStreamCreateWithFlags(&ctx->util_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; ok && i < o.copy_streams; ++i) {
    cudaStream_t s;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ctx->copy_streams.push_back(s);
  }
  if (!ok) {
    pq_destroy(ctx);
    return PQ_ERR_CUDA;
  }
  *out = ctx;
  return PQ_OK;
}

pq_status pq_destroy(pq_ctx* ctx) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  // A served batch that never completes leaves the context allocated: its
  // memory may still be in use on the device.
  if (server_stop(ctx) != PQ_OK) return PQ_ERR_TIMEOUT;
  cudaDeviceSynchronize();
  plan_cache_destroy(ctx);
  for (auto s : ctx->copy_streams) cudaStreamDestroy(s);
  if (ctx->util_stream) cudaStreamDestroy(ctx->util_stream);
  for (auto& kv : ctx->prof)
    for (auto& pr : kv.second.pairs) cudaEventDestroy(pr.first), cudaEventDestroy(pr.second);
  ctx->ring.shutdown();
  ctx->arena.shutdown();
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_small) cudaFreeHost(ctx->h_small);
  delete ctx;
  return PQ_OK;
}

pq_status pq_sync(pq_ctx* ctx, void* stream) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  cudaStream_t s = S(stream);
  k_take_status<<<1, 1, 0, s>>>(ctx->d_status, ctx->d_status + 1);
  PQ_LAUNCHED(ctx);
  PQ_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status + 1, sizeof(pqk::DevStatus),
                               cudaMemcpyDeviceToHost, s));
  PQ_CUDA(ctx, cudaStreamSynchronize(s));
  if (ctx->opt.profile) {
    std::lock_guard<std::mutex> g(ctx->mu);
    prof_collect(ctx);
  }
  int code = ctx->h_status->code;
  if (code != 0)
    return fail(ctx, (pq_status)code, "device reported %s (detail %lld)", pq_status_string(code),
                (long long)ctx->h_status->detail);
  return PQ_OK;
}

const char* pq_last_error(pq_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

pq_status pq_get_stats(pq_ctx* ctx, pq_stats* s) {
  if (!ctx || !s) return PQ_ERR_INVALID_ARG;
  memset(s, 0, sizeof *s);
  s->kernel_launches = ctx->launches.load();
  s->h2d_bytes = ctx->h2d.load();
  s->d2h_bytes = ctx->d2h.load();
  s->arena_bytes = (int64_t)ctx->arena.capacity();
  s->arena_in_use = (int64_t)ctx->arena.in_use();
  s->arena_high_water = (int64_t)ctx->arena.high_water();
  s->chunks_ingested = ctx->chunks.load();
  s->plans_run = ctx->plans.load();
  s->graph_replays = ctx->replays.load();
  s->out_of_core_passes = ctx->passes.load();
  return PQ_OK;
}

pq_status pq_profile_read(pq_ctx* ctx, const char* name, double* total_ms, int64_t* launches) {
  if (!ctx || !name) return PQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  prof_collect(ctx);
  auto it = ctx->prof.find(name);
  if (it == ctx->prof.end()) return fail(ctx, PQ_ERR_INVALID_ARG, "no profile entry '%s'", name);
  if (total_ms) *total_ms = it->second.total_ms;
  if (launches) *launches = it->second.launches;
  return PQ_OK;
}

pq_status pq_profile_enable(pq_ctx* ctx, int32_t on) {
  if (!ctx || (on != 0 && on != 1)) return PQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->opt.profile = on;
  return PQ_OK;
}

pq_status pq_profile_reset(pq_ctx* ctx) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(ctx->mu);
  for (auto& kv : ctx->prof) kv.second.total_ms = 0, kv.second.launches = 0, kv.second.used = 0;
  return PQ_OK;
}

// ---------------------------------------------------------------- tables ----
static pq_status copy_host_to_device(pq_ctx* ctx, void* dst, const pqh::Column& c, int64_t off,
                                     size_t bytes, cudaStream_t s);
static pq_status unpack_to_device(pq_ctx* ctx, void* dst, const pqh::Column& c, int64_t nrows,
                                  cudaStream_t s);

pq_status pq_load_columns(pq_ctx* ctx, const pq_source* srcs, int ncols, int64_t nrows, int mode,
                          pq_table** out, void* stream) {
  if (!ctx || !out || !srcs || ncols <= 0 || ncols > 64 || nrows < 0 ||
      (mode != PQ_RESIDENT && mode != PQ_STREAMING && mode != PQ_MAPPED))
    return fail(ctx, PQ_ERR_INVALID_ARG, "pq_load_columns: bad arguments");
  *out = nullptr;
  cudaStream_t s = S(stream);
  std::unique_ptr<pq_table> t(new pq_table());
  t->id = ctx->next_table_id.fetch_add(1);
  t->nrows = nrows;
  t->mode = mode;
  for (int i = 0; i < ncols; ++i) {
    const pq_source& src = srcs[i];
    pqh::Column c;
    c.type = src.type;
    c.src = src;
    if (!valid_dtype(src.type)) return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: bad type", i);
    switch (src.kind) {
      case PQ_SRC_DEVICE:
        if (!src.ptr && nrows) return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: null", i);
        c.dev = src.ptr;
        break;
      case PQ_SRC_HOST: {
        if (!src.ptr && nrows) return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: null", i);
        cudaPointerAttributes at{};
        c.pinned = cudaPointerGetAttributes(&at, src.ptr) == cudaSuccess &&
                   at.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (mode == PQ_MAPPED) {  // read in place by the kernels
          if (nrows && (!c.pinned || !at.devicePointer))
            return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: mapped tables need page-locked host memory", i);
          c.dev = nrows ? at.devicePointer : src.ptr;
        }
        break;
      }
      case PQ_SRC_PACKED: {
        if (!src.ptr) return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: null", i);
        if (mode == PQ_MAPPED)
          return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: packed columns cannot be mapped", i);
        cudaPointerAttributes at{};
        c.pinned = cudaPointerGetAttributes(&at, src.ptr) == cudaSuccess &&
                   at.type == cudaMemoryTypeHost;
        cudaGetLastError();
        if (!c.pinned)
          return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: packed columns need page-locked memory", i);
        if (!pqh::packed_info(src.ptr, src.type, nrows, &c.pk))
          return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: not a packed column of %lld rows of this type",
                      i, (long long)nrows);
        c.packed = true;
        break;
      }
      case PQ_SRC_FILE:
        if (mode == PQ_MAPPED)
          return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: files cannot be mapped", i);
        if (!src.path) return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: no path", i);
        c.path = src.path;
        c.src.path = c.path.c_str();
        break;
      default:
        return fail(ctx, PQ_ERR_INVALID_ARG, "column %d: bad source kind", i);
    }
    t->cols.push_back(c);
  }
  if (mode == PQ_RESIDENT) {
    for (auto& c : t->cols) {
      if (c.dev) continue;
      size_t bytes = dtype_size(c.type) * (size_t)nrows;
      c.owned = ctx->arena.alloc(bytes + 16);
      if (!c.owned) {
        for (auto& d : t->cols) ctx->arena.release_now(d.owned);
        return fail(ctx, PQ_ERR_BUDGET, "resident table needs %zu more bytes", bytes);
      }
      c.dev = c.owned;
      pq_status st = c.packed ? unpack_to_device(ctx, c.owned, c, nrows, s)
                              : copy_host_to_device(ctx, c.owned, c, 0, bytes, s);
      if (st != PQ_OK) {
        for (auto& d : t->cols) ctx->arena.release(d.owned, s);
        return st;
      }
    }
  }
  *out = t.release();
  return PQ_OK;
}

int64_t pq_table_rows(const pq_table* t) { return t ? t->nrows : -1; }

const void* pq_table_column(const pq_table* t, int col) {
  if (!t || col < 0 || col >= (int)t->cols.size()) return nullptr;
  return t->cols[col].dev;
}

pq_status pq_table_free(pq_ctx* ctx, pq_table* t, void* stream) {
  if (!ctx || !t) return PQ_ERR_INVALID_ARG;
  cudaStream_t s = S(stream);
  forget_table(ctx, t->id, s);
  for (auto& c : t->cols) {
    ctx->arena.release(c.owned, s);
    ctx->arena.release(c.pres.block, s);
  }
  delete t;
  return PQ_OK;
}

pq_status pq_ht_free(pq_ctx* ctx, pq_ht* ht, void* stream) {
  if (!ctx || !ht) return PQ_ERR_INVALID_ARG;
  ctx->arena.release(ht->block, S(stream));
  delete ht;
  return PQ_OK;
}

}  // extern "C"

// A packed column decoded into `dst` (nrows values): the packed bytes are
// copied into a scratch block of the arena and decoded there.
static pq_status unpack_to_device(pq_ctx* ctx, void* dst, const pqh::Column& c, int64_t nrows,
                                  cudaStream_t s) {
  const char* base = (const char*)c.src.ptr;
  const size_t tab = (const char*)c.pk.blocks - base;
  const size_t pay = (const char*)c.pk.words - base;
  const size_t bytes = pay + 4 * (size_t)(c.pk.total_words + 4);
  char* tmp = (char*)ctx->arena.alloc(bytes);
  if (!tmp) return fail(ctx, PQ_ERR_BUDGET, "decoding a packed column needs %zu bytes", bytes);
  cudaError_t e = cudaMemcpyAsync(tmp, base, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = pqh::unpack_launch((const pqh::PackBlock*)(tmp + tab), (const uint32_t*)(tmp + pay), 0, 0,
                           nrows, c.type, dst, ctx->num_sms, s);
  ctx->arena.release(tmp, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "packed column decode");
  ctx->h2d += (int64_t)bytes;
  ctx->launches++;
  return PQ_OK;
}

// Host -> device copy of `bytes` bytes of column `c` starting at byte `off`:
// pinned memory goes straight to the copy engine; pageable memory and files go
// through two pinned staging buffers so that no pageable copy reaches a stream.
static pq_status copy_host_to_device(pq_ctx* ctx, void* dst, const pqh::Column& c, int64_t off,
                                     size_t bytes, cudaStream_t s) {
  if (bytes == 0) return PQ_OK;
  if (c.src.kind == PQ_SRC_HOST && c.pinned) {
    PQ_CUDA(ctx, cudaMemcpyAsync(dst, (const char*)c.src.ptr + off, bytes,
                                 cudaMemcpyHostToDevice, s));
    ctx->h2d += (int64_t)bytes;
    return PQ_OK;
  }
  const size_t stage = 16u << 20;
  char* buf[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  pq_status st = PQ_OK;
  int fd = -1;
  if (c.src.kind == PQ_SRC_FILE) {
    fd = open(c.path.c_str(), O_RDONLY);
    if (fd < 0) return fail(ctx, PQ_ERR_IO, "open %s failed", c.path.c_str());
  }
  for (int i = 0; i < 2; ++i) {
    if (cudaHostAlloc((void**)&buf[i], stage, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
      st = fail(ctx, PQ_ERR_CUDA, "pinned staging allocation failed");
    }
  }
  size_t done = 0;
  for (int k = 0; st == PQ_OK && done < bytes; ++k) {
    int i = k & 1;
    size_t b = std::min(stage, bytes - done);
    if (k >= 2) cudaEventSynchronize(ev[i]);
    if (fd >= 0) {
      size_t got = 0;
      while (got < b) {
        ssize_t r = pread(fd, buf[i] + got, b - got, (off_t)(c.src.offset + off + done + got));
        if (r <= 0) break;
        got += (size_t)r;
      }
      if (got != b) {
        st = fail(ctx, PQ_ERR_IO, "short read from %s", c.path.c_str());
        break;
      }
    } else {
      memcpy(buf[i], (const char*)c.src.ptr + off + done, b);
    }
    if (cudaMemcpyAsync((char*)dst + done, buf[i], b, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(ev[i], s) != cudaSuccess) {
      st = fail(ctx, PQ_ERR_CUDA, "staged copy failed");
      break;
    }
    ctx->h2d += (int64_t)b;
    done += b;
  }
  for (int i = 0; i < 2; ++i) {
    if (ev[i]) cudaEventSynchronize(ev[i]), cudaEventDestroy(ev[i]);
    if (buf[i]) cudaFreeHost(buf[i]);
  }
  if (fd >= 0) close(fd);
  return st;
}
