// pq_plan.cu -- resident plan driver: batches, D-set cache, CUDA-graph cache.
#include <algorithm>
#include <cstring>

#define PQ_DEFINE_PLAN_KERNELS
#include "pq_plan_host.h"

using namespace pqk;

namespace pqh {

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

bool is_pinned(const void* p) {
  cudaPointerAttributes at{};
  bool pinned = cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost;
  cudaGetLastError();
  return pinned;
}

static bool range(const pq_table* t, int64_t row0, int64_t rows, i64* r0, i64* n) {
  if (!t || row0 < 0 || row0 > t->nrows) return false;
  if (rows < 0) rows = t->nrows - row0;
  if (row0 + rows > t->nrows) return false;
  *r0 = row0;
  *n = rows;
  return true;
}

static bool check_types(const pq_table* t, std::initializer_list<int> types) {
  if ((int)t->cols.size() < (int)types.size()) return false;
  int i = 0;
  for (int ty : types)
    if (t->cols[i++].type != ty) return false;
  return true;
}

// Range of an int32 / int64 key column (order-preserving ukey): out[0] holds
// ~min, out[1] the max, both zero-initialised and grown with atomicMax.
// out[2] counts the descents (rows whose key is greater than the next row's;
// counting stops soon after kMaxDescents) and out[3 + j] holds the row after
// descent j for the first kMaxDescents of them, in no particular order.
__global__ void k_key_range(const void* col, int is64, i64 n, u64* out) {
  u64 nmin = 0, umax = 0;
  auto at = [&](i64 i) {
    return is64 ? __ldg(reinterpret_cast<const i64*>(col) + i)
                : (i64)__ldg(reinterpret_cast<const int*>(col) + i);
  };
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    const i64 k = at(i);
    nmin = max(nmin, ~ukey(k));
    umax = max(umax, ukey(k));
    if (i + 1 < n && k > at(i + 1) && *(volatile u64*)(out + 2) <= (u64)kMaxDescents) {
      const u64 j = atomicAdd(reinterpret_cast<unsigned long long*>(out + 2), 1ULL);
      if (j < (u64)kMaxDescents) out[3 + j] = (u64)(i + 1);
    }
  }
  range_commit(nmin, umax, out, out + 1);
}

// The key range of column c of a resident table, measured once and kept with
// the column.  The measurement (one kernel and a read-back) runs on the
// context's utility stream, ordered after the work queued so far on `s` (the
// legacy default stream when `s` is null), and the host waits for it with no
// lock held.  Two threads may measure the same column at once: both find the
// same range and the first to publish it wins.
bool ensure_range(pq_ctx* ctx, const pq_table* t, int c, cudaStream_t s) {
  const Column& col = t->cols[c];
  if (col.range.known()) return true;
  if (!col.dev || t->nrows <= 0) return false;
  cudaStream_t u = ctx->util_stream;
  SmallPinned h(ctx);
  u64* d = (u64*)ctx->arena.alloc(256);
  cudaEvent_t after = nullptr;
  bool ok = h.p && d &&
            cudaEventCreateWithFlags(&after, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(after, s ? s : cudaStreamLegacy) == cudaSuccess &&
            cudaStreamWaitEvent(u, after, 0) == cudaSuccess &&
            cudaMemsetAsync(d, 0, 24, u) == cudaSuccess;
  constexpr size_t rb = 8 * (3 + kMaxDescents);
  static_assert(rb <= kSmallBytes, "read-back buffer");
  if (ok) {
    const int grid = (int)std::min<i64>((t->nrows + 255) / 256, (i64)ctx->num_sms * 8);
    k_key_range<<<grid, 256, 0, u>>>(col.dev, col.type == PQ_INT64 ? 1 : 0, t->nrows, d);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(h.p, d, rb, cudaMemcpyDeviceToHost, u) == cudaSuccess &&
         cudaStreamSynchronize(u) == cudaSuccess;
    ctx->launches++;
  }
  if (after) cudaEventDestroy(after);
  if (d) ctx->arena.release(d, u);
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> g(ctx->range_mu);
  if (col.range.known()) return true;
  KeyRange& kr = col.range;
  kr.umin = ~(u64)h.p[0];
  kr.umax = (u64)h.p[1];
  const int64_t nd = h.p[2];
  kr.ndesc = nd > kMaxDescents ? -1 : (int)nd;
  for (int j = 0; j < kr.ndesc; ++j) kr.desc[j] = h.p[3 + j];
  std::sort(kr.desc, kr.desc + std::max(kr.ndesc, 0));
  kr.ready.store(true, std::memory_order_release);
  return true;
}

// Rows per key-range bucket (kHistBuckets buckets of 2^shift keys from umin).
__global__ void k_key_hist(const i64* key, i64 n, u64 umin, int shift, u32* out) {
  __shared__ u32 h[kHistBuckets];
  for (int i = threadIdx.x; i < kHistBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x)
    atomicAdd(&h[(ukey(__ldg(key + i)) - umin) >> shift], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kHistBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(out + i, h[i]);
}

// The key histogram of int64 key column c (its range known), measured once
// like the range (utility stream, no lock held across the wait).
static bool ensure_key_hist(pq_ctx* ctx, const pq_table* t, int c, cudaStream_t s) {
  const Column& col = t->cols[c];
  if (col.hist.known()) return true;
  if (!col.range.known() || !col.dev || t->nrows <= 0 || col.type != PQ_INT64) return false;
  const u64 span = col.range.umax - col.range.umin;  // keys - 1
  const int shift = part_shift(span + 1, 10);
  static_assert(kHistBuckets == 1 << 10, "buckets");
  cudaStream_t u = ctx->util_stream;
  std::vector<u32> host(kHistBuckets);
  u32* d = (u32*)ctx->arena.alloc(kHistBuckets * 4);
  cudaEvent_t after = nullptr;
  bool ok = d && cudaEventCreateWithFlags(&after, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(after, s ? s : cudaStreamLegacy) == cudaSuccess &&
            cudaStreamWaitEvent(u, after, 0) == cudaSuccess &&
            cudaMemsetAsync(d, 0, kHistBuckets * 4, u) == cudaSuccess;
  if (ok) {
    const int grid = (int)std::min<i64>((t->nrows + 255) / 256, (i64)ctx->num_sms * 8);
    k_key_hist<<<grid, 256, 0, u>>>((const i64*)col.dev, t->nrows, col.range.umin, shift, d);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(host.data(), d, kHistBuckets * 4, cudaMemcpyDeviceToHost, u) ==
             cudaSuccess &&
         cudaStreamSynchronize(u) == cudaSuccess;
    ctx->launches++;
  }
  if (after) cudaEventDestroy(after);
  if (d) ctx->arena.release(d, u);
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> g(ctx->range_mu);
  if (col.hist.known()) return true;
  col.hist.shift = shift;
  col.hist.counts = host;
  col.hist.ready.store(true, std::memory_order_release);
  return true;
}

// Static key bitmaps (see PlanDev): a side whose table is resident and whose
// key range fits in 32 bits per slot of its table (sized for the table's
// rows) gets a bitmap over that whole range, known before the plan runs.
// While the stream is being captured nothing new is measured.
static void plan_static(pq_ctx* ctx, const pq_plan& p, ResolvedPlan& r, cudaStream_t s,
                        bool capturing) {
  PlanDev& d = r.dev;
  d.d_e = r.e_d;
  d.m_e = r.e_m;
  auto fits = [&](const pq_table* t, int e, u64* su, u64* sb) -> bool {
    const KeyRange& c = t->cols[0].range;
    if (!c.known() && (capturing || !ensure_range(ctx, t, 0, s))) return false;
    const u64 span = c.umax - c.umin;  // bits - 1
    if (c.umax < c.umin || span >= (32ULL << e) || span >= kMaxBmBits) return false;
    *su = c.umin;
    *sb = span + 1;
    return true;
  };
  d.d_static = r.resident[0] && fits(p.D, r.e_d, &d.d_su, &d.d_sb) ? 1 : 0;
  d.m_static = r.resident[1] && fits(p.M, r.e_m, &d.m_su, &d.m_sb) ? 1 : 0;
  if (d.d_static) {
    // A bitmap D-set uses only the key bitmap of its block: the smallest
    // table whose 32 bits per slot cover the key range, not a hash table
    // sized for the rows.
    int e = 6;
    while ((32ULL << e) < d.d_sb) ++e;
    r.e_d = d.d_e = e;
  }
  // Bound of one row's revenue |price * (100 - disc)|: the price column's
  // measured range times the largest |100 - disc| of an int8 (228).
  d.rev_max = 0;
  if (r.resident[2] && p.F->nrows > 0) {
    const KeyRange& pr = p.F->cols[1].range;
    if (pr.known() || (!capturing && ensure_range(ctx, p.F, 1, s))) {
      const i64 lo = (i64)(pr.umin ^ (1ULL << 63)), hi = (i64)(pr.umax ^ (1ULL << 63));
      const unsigned __int128 amax =
          std::max(lo < 0 ? (unsigned __int128)(-(__int128)lo) : (unsigned __int128)lo,
                   hi < 0 ? (unsigned __int128)(-(__int128)hi) : (unsigned __int128)hi);
      const unsigned __int128 rev = amax * 228;
      if (rev < ((unsigned __int128)1 << 63)) d.rev_max = (u64)rev;
    }
  }
}

pq_status resolve_plan(pq_ctx* ctx, const pq_plan& p, ResolvedPlan& r, bool need_resident) {
  r = ResolvedPlan();
  if (!p.D || !p.M || !p.F) return fail(ctx, PQ_ERR_INVALID_ARG, "plan: missing table");
  if (!check_types(p.D, {PQ_INT32, PQ_INT8}) || !check_types(p.M, {PQ_INT64, PQ_INT32, PQ_INT32}) ||
      !check_types(p.F, {PQ_INT64, PQ_INT64, PQ_INT8, PQ_INT32}))
    return fail(ctx, PQ_ERR_INVALID_ARG, "plan: column types do not match D/M/F");
  if (!range(p.D, p.d_row0, p.d_rows, &r.d_row0, &r.n_d) ||
      !range(p.M, p.m_row0, p.m_rows, &r.m_row0, &r.n_m) ||
      !range(p.F, p.f_row0, p.f_rows, &r.f_row0, &r.n_f))
    return fail(ctx, PQ_ERR_INVALID_ARG, "plan: row range outside a table");
  if (p.k < 1 || p.k > PQ_MAX_K) return fail(ctx, PQ_ERR_INVALID_ARG, "plan: k out of range");
  float lf = p.load_factor > 0 ? p.load_factor : ctx->opt.load_factor;
  if (lf < 0.05f || lf > 0.9f) return fail(ctx, PQ_ERR_INVALID_ARG, "plan: load factor");
  bool ok1, ok2, ok3;
  PlanDev& d = r.dev;
  d.pd = make_pred(p.d_op, p.d_c, &ok1);
  d.pm = make_pred(p.m_op, p.m_c, &ok2);
  d.pf = make_pred(p.f_op, p.f_c, &ok3);
  if (!ok1 || !ok2 || !ok3) return fail(ctx, PQ_ERR_INVALID_ARG, "plan: bad predicate");
  d.k = p.k;
  d.lf1024 = (int)(lf * 1024 + 0.5f);
  d.n_d = r.n_d;
  d.n_m = r.n_m;
  d.n_f = r.n_f;
  if (r.n_f >= (1LL << 32))
    return fail(ctx, PQ_ERR_INVALID_ARG, "plan: %lld F rows (at most 2^32 - 1 per plan)",
                (long long)r.n_f);
  d.d_tile = scan_tile(r.n_d, 512, kTD, resident_warps(ctx, 0));
  d.m_tile = scan_tile(r.n_m, 128, kTM, resident_warps(ctx, 3));
  d.f_tile = scan_tile(r.n_f, 128, kTF, resident_warps(ctx, 8));
  r.e_d = cap_log2(r.n_d, d.lf1024);
  r.e_m = cap_log2(r.n_m, d.lf1024);
  r.parts = topk_parts(r.e_m);
  const pq_table* T[3] = {p.D, p.M, p.F};
  for (int t = 0; t < 3; ++t) {
    r.resident[t] = true;
    for (auto& c : T[t]->cols) r.resident[t] = r.resident[t] && c.dev != nullptr;
    if (need_resident && !r.resident[t])
      return fail(ctx, PQ_ERR_INVALID_ARG, "plan: table %d is not resident", t);
  }
  auto col = [](const pq_table* t, int c, i64 row0) -> const char* {
    const char* base = (const char*)t->cols[c].dev;
    return base ? base + row0 * dtype_size(t->cols[c].type) : nullptr;
  };
  d.d_key = (const int*)col(p.D, 0, r.d_row0);
  d.d_seg = (const signed char*)col(p.D, 1, r.d_row0);
  d.m_key = (const i64*)col(p.M, 0, r.m_row0);
  d.m_dref = (const int*)col(p.M, 1, r.m_row0);
  d.m_date = (const int*)col(p.M, 2, r.m_row0);
  d.f_mkey = (const i64*)col(p.F, 0, r.f_row0);
  d.f_price = (const i64*)col(p.F, 1, r.f_row0);
  d.f_disc = (const signed char*)col(p.F, 2, r.f_row0);
  d.f_date = (const int*)col(p.F, 3, r.f_row0);
  const void* ptrs[9] = {d.d_key, d.d_seg, d.m_key, d.m_dref, d.m_date,
                         d.f_mkey, d.f_price, d.f_disc, d.f_date};
  d.vec = 1;
  for (auto q : ptrs) d.vec &= (((uintptr_t)q) & 15) == 0;
  d.m_pair = p.M->mode == PQ_MAPPED ? 1 : 0;
  d.f_pair = p.F->mode == PQ_MAPPED ? 1 : 0;
  d.part_log2 = 0;
  if (p.flags & PQ_PLAN_PARTITIONED) {
    if (p.flags & PQ_PLAN_AGG_FIRST)
      return fail(ctx, PQ_ERR_INVALID_ARG,
                  "plan: PQ_PLAN_PARTITIONED applies to the join-first plan only");
    const int lp = p.log2P > 0 ? p.log2P : ctx->opt.log2P;
    if (lp < 1 || lp > kMaxPartLog2)
      return fail(ctx, PQ_ERR_INVALID_ARG, "plan: partitioned fan-out 2^%d (1 .. 2^%d)", lp,
                  kMaxPartLog2);
    d.part_log2 = lp;
  }
  return PQ_OK;
}

// M side of a plan: a static bitmap means a dense dictionary of at most
// n_m members over the table's key range, else a hash table of 2^e_m slots.
static size_t mside_bytes(const ResolvedPlan& r) {
  const i64 c = r.m_cap >= 0 ? r.m_cap : r.n_m;
  return r.dev.m_static ? al256(dense_layout(c, r.dev.m_sb).total) : mtable_bytes(r.e_m);
}

size_t plan_bytes(const ResolvedPlan& r) {
  size_t b = 0;
  if (r.builds && !r.dev.d_static) b += al(r.n_d * 8);             // D list
  if (r.builds && r.dset_from == -1) b += dset_block_bytes(r.e_d);  // own D-set
  if (!r.dev.m_static) b += al(r.n_m * 8);                          // M list
  b += mside_bytes(r);                   // M dictionary or table
  b += al(r.parts * 4);                                        // top-k list lengths
  b += al(topk_cand_cap(r.e_m, r.dev.k) * 8) * 2;              // top-k tile lists
  b += al(r.n_f * 4);                                           // F hit list
  if (r.dev.part_log2)                                          // partitioned hits
    b += al(((1 << r.dev.part_log2) + 1) * 8) + al(r.n_f * 8) + al(r.n_f * 4) + al(r.n_f * 8);
  return b;
}

void plan_assign(ResolvedPlan& r, char* base) {
  PlanDev& d = r.dev;
  char* p = base;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += al(bytes);
    return q;
  };
  d.build_dset = r.builds ? 1 : 0;
  d.dlist = r.builds && !d.d_static ? (i64*)take(r.n_d * 8) : nullptr;
  if (r.builds && r.dset_from == -1) dset_block_assign(take(dset_block_bytes(r.e_d)), r.e_d, d);
  d.mlist = d.m_static ? nullptr : (i64*)take(r.n_m * 8);
  d.ht_tag = (unsigned short*)take(mside_bytes(r));
  d.tk_c = (int*)take(r.parts * 4);
  d.cand_k = (i64*)take(topk_cand_cap(r.e_m, d.k) * 8);
  d.cand_s = (i64*)take(topk_cand_cap(r.e_m, d.k) * 8);
  d.hlist = (u32*)take(r.n_f * 4);
  d.part = nullptr, d.pval0 = nullptr, d.pslot = nullptr, d.pval = nullptr;
  if (d.part_log2) {
    d.part = (u64*)take(((1 << d.part_log2) + 1) * 8);
    d.pval0 = (i64*)take(r.n_f * 8);
    d.pslot = (u32*)take(r.n_f * 4);
    d.pval = (i64*)take(r.n_f * 8);
  }
}

BatchLayout batch_layout(int nq) {
  BatchLayout L;
  size_t o = 0;
  L.desc = o;
  o += sizeof(PlanDev) * nq;
  o = (o + 15) / 16 * 16;
  L.tD = o;
  o += 8 * (nq + 1);
  L.tM = o;
  o += 8 * (nq + 1);
  L.tF = o;
  o += 8 * (nq + 1);
  L.dyn = al(o);
  o = L.dyn + 11 * 8 * (nq + 1);
  L.work = al(o);
  o = L.work + 256;
  L.ctr = o;
  o += sizeof(QCtr) * nq;
  L.out = al(o);
  o = L.out + sizeof(pq_result) * nq;
  L.end = al(o);
  return L;
}

Batch make_batch(pq_ctx* ctx, char* ws, int nq, const BatchLayout& L) {
  Batch b{};
  b.q = (PlanDev*)(ws + L.desc);
  b.nq = nq;
  b.tD = (const i64*)(ws + L.tD);
  b.tM = (const i64*)(ws + L.tM);
  b.tF = (const i64*)(ws + L.tF);
  b.dyn = (i64*)(ws + L.dyn);
  b.work = (u32*)(ws + L.work);
  b.st = ctx->d_status;
  b.spin_limit = ctx->opt.spin_limit;
  b.ov.table = 0;
  return b;
}

static const char* kPhaseName[] = {"plan_dscan", "plan_dfill",  "plan_dbuild", "plan_mscan",
                                   "plan_mfill", "plan_mbuild", "plan_mrank",  "plan_mdup",
                                   "plan_fscan", "plan_fpart",  "plan_fscatter", "plan_fagg",
                                   "plan_fprobe", "plan_topk"};
static_assert(sizeof(kPhaseName) / sizeof(kPhaseName[0]) == kPhaseTopk + 1, "phase names");

pq_status plan_kernels_init(pq_ctx* ctx) {
  const void* fn[25] = {(const void*)k_plan_dscan<true>, (const void*)k_plan_fill,
                        (const void*)k_plan_dbuild,      (const void*)k_plan_mscan<true, true>,
                        (const void*)k_plan_fill,        (const void*)k_plan_mbuild,
                        (const void*)k_plan_fscan<false, false>, (const void*)k_plan_topk,
                        (const void*)k_plan_fscan<true, false>,  (const void*)k_plan_mscan<false, true>,
                        (const void*)k_plan_topk,        (const void*)k_plan_mrank,
                        (const void*)k_plan_mdup,        (const void*)k_plan_fprobe,
                        (const void*)k_plan_mscan<true, false>,
                        (const void*)k_plan_mscan<false, false>,
                        (const void*)k_plan_mscan_bm<true, false>,
                        (const void*)k_plan_mscan_bm<false, false>,
                        (const void*)k_plan_fpart,
                        (const void*)k_plan_fscatter,
                        (const void*)k_plan_fagg,
                        (const void*)k_plan_fscan<false, true>,
                        (const void*)k_plan_fscan<true, true>,
                        (const void*)k_plan_mscan_bm<true, true>,
                        (const void*)k_plan_mscan_bm<false, true>};
  for (int i = 0; i < 25; ++i) {
    int n = 0;
    const int threads = i == 7 || i == 10 ? kTKW * 32 : 256;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn[i], threads, 0) != cudaSuccess)
      return PQ_ERR_CUDA;
    ctx->plan_occ[i] = std::max(n, 1);
  }
  return PQ_OK;
}

// Persistent grid of a plan kernel: the tuned blocks per SM, capped by what
// fits on an SM at once (a block that only starts after others exit finds
// no work left) and by the phase's largest possible tile count.
static thread_local i64 t_tiles_max = -1;
static thread_local bool t_list_m = true;  // some plan of the batch keeps an M key list
static thread_local bool t_bm_dm = false;  // every plan: static M bitmap, D-set bitmap
static thread_local bool t_buf = false;    // some plan buffers its F hits
static thread_local bool t_win = false;    // some plan is an out-of-core pass (M key window)
static int plan_grid(pq_ctx* ctx, int occ_index, int tiles_per_block = 8) {
  const i64 g = (i64)ctx->num_sms * std::max(1, std::min(ctx->tune_bps, ctx->plan_occ[occ_index]));
  if (t_tiles_max < 0) return (int)g;
  return (int)std::max<i64>(1, std::min(g, (t_tiles_max + tiles_per_block - 1) / tiles_per_block));
}

// Launch a plan kernel with programmatic stream serialization, so that its
// launch overlaps the end of the previous kernel on the stream (the kernel
// itself waits for that kernel's completion in chain_begin).  Not while the
// stream is being captured: in a replayed graph the early blocks of the next
// kernel were measured to slow the chain down.
static thread_local bool t_chain = true;
template <typename... P, typename... A>
static cudaError_t launch_chained(void (*k)(P...), int grid, int block, cudaStream_t s,
                                  A... args) {
  if (!t_chain) {
    k<<<grid, block, 0, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

void set_kernel_variants(bool buffered_hits, bool key_window) {
  t_buf = buffered_hits;
  t_win = key_window;
}

pq_status launch_phase(pq_ctx* ctx, int phase, const Batch& b, bool vec, cudaStream_t s,
                       i64 tiles_max, bool list_m, bool bm_dm) {
  t_list_m = list_m;
  t_bm_dm = bm_dm && !list_m;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  t_chain = cap == cudaStreamCaptureStatusNone;
  t_tiles_max = tiles_max;
  cudaEvent_t stop;
  prof_begin(ctx, kPhaseName[phase], s, &stop);
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case kPhaseD:
      e = vec ? launch_chained(k_plan_dscan<true>, plan_grid(ctx, 0), 256, s, b)
              : launch_chained(k_plan_dscan<false>, plan_grid(ctx, 0), 256, s, b);
      break;
    case kPhaseDfill: e = launch_chained(k_plan_fill, plan_grid(ctx, 1, 1), 256, s, b, 0); break;
    case kPhaseDbuild: e = launch_chained(k_plan_dbuild, plan_grid(ctx, 2), 256, s, b); break;
    case kPhaseM:
      if (t_bm_dm && t_win)
        e = vec ? launch_chained(k_plan_mscan_bm<true, true>, plan_grid(ctx, 23), 256, s, b)
                : launch_chained(k_plan_mscan_bm<false, true>, plan_grid(ctx, 24), 256, s, b);
      else if (t_bm_dm)
        e = vec ? launch_chained(k_plan_mscan_bm<true, false>, plan_grid(ctx, 16), 256, s, b)
                : launch_chained(k_plan_mscan_bm<false, false>, plan_grid(ctx, 17), 256, s, b);
      else if (t_list_m)
        e = vec ? launch_chained(k_plan_mscan<true, true>, plan_grid(ctx, 3), 256, s, b)
                : launch_chained(k_plan_mscan<false, true>, plan_grid(ctx, 9), 256, s, b);
      else
        e = vec ? launch_chained(k_plan_mscan<true, false>, plan_grid(ctx, 14), 256, s, b)
                : launch_chained(k_plan_mscan<false, false>, plan_grid(ctx, 15), 256, s, b);
      break;
    case kPhaseMfill: e = launch_chained(k_plan_fill, plan_grid(ctx, 4, 1), 256, s, b, 1); break;
    case kPhaseMbuild: e = launch_chained(k_plan_mbuild, plan_grid(ctx, 5), 256, s, b); break;
    case kPhaseMrank: e = launch_chained(k_plan_mrank, plan_grid(ctx, 11), 256, s, b); break;
    case kPhaseMdup: e = launch_chained(k_plan_mdup, plan_grid(ctx, 12), 256, s, b); break;
    case kPhaseFscan:
      if (t_buf)
        e = vec ? launch_chained(k_plan_fscan<true, true>, plan_grid(ctx, 22), 256, s, b)
                : launch_chained(k_plan_fscan<false, true>, plan_grid(ctx, 21), 256, s, b);
      else
        e = vec ? launch_chained(k_plan_fscan<true, false>, plan_grid(ctx, 8), 256, s, b)
                : launch_chained(k_plan_fscan<false, false>, plan_grid(ctx, 6), 256, s, b);
      break;
    case kPhaseFpart: e = launch_chained(k_plan_fpart, plan_grid(ctx, 18, 1), 256, s, b); break;
    case kPhaseFscatter:
      e = launch_chained(k_plan_fscatter, plan_grid(ctx, 19, 1), 256, s, b);
      break;
    case kPhaseFagg: e = launch_chained(k_plan_fagg, plan_grid(ctx, 20, 1), 256, s, b); break;
    case kPhaseF: e = launch_chained(k_plan_fprobe, plan_grid(ctx, 13), 256, s, b); break;
    case kPhaseTopk: e = launch_chained(k_plan_topk, plan_grid(ctx, 7, 1), kTKW * 32, s, b); break;
  }
  prof_end(stop, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "plan kernel launch");
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}

// ------------------------------------------------------------ graph cache ----
struct GraphEntry {
  std::string key;
  uint64_t tids[3];
  void* ws = nullptr;
  pq_result* out = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  uint64_t last_use = 0;
  int64_t kernels = 0;  // kernel nodes of the graph
};

struct PlanCache {
  std::vector<GraphEntry> entries;
  uint64_t tick = 0;
};

void plan_cache_destroy(pq_ctx* ctx) {
  if (ctx->plan_cache) {
    for (auto& e : ctx->plan_cache->entries) {
      if (e.exec) cudaGraphExecDestroy(e.exec);
      if (e.done) cudaEventDestroy(e.done);
      ctx->arena.release_now(e.ws);
    }
    delete ctx->plan_cache;
    ctx->plan_cache = nullptr;
  }
  for (auto& d : ctx->dsets) {
    if (d.ready) cudaEventDestroy(d.ready);
    for (auto ev : d.users) cudaEventDestroy(ev);
    ctx->arena.release_now(d.block);
  }
  ctx->dsets.clear();
}

static std::string plan_key(pq_ctx* ctx, const pq_plan& p) {
  pq_plan q = p;
  uint64_t ids[3] = {p.D->id, p.M->id, p.F->id};
  q.D = q.M = q.F = nullptr;
  std::string k((const char*)&q, sizeof q);
  k.append((const char*)ids, sizeof ids);
  k.append((const char*)&ctx->tune_bps, sizeof ctx->tune_bps);
  return k;
}

// Release a cached graph's workspace once `s` has passed its last replay;
// the executable graph itself is freed by CUDA when it is no longer running.
static void graph_release(pq_ctx* ctx, GraphEntry& e, cudaStream_t s) {
  if (e.done) cudaStreamWaitEvent(s, e.done, 0), cudaEventDestroy(e.done);
  if (e.exec) cudaGraphExecDestroy(e.exec);
  ctx->arena.release(e.ws, s);
}

// Release a cached D-set's block once `s` has passed its build and every
// batch that read it (their completion events).  No host wait.
static void dset_release(pq_ctx* ctx, DsetEntry& e, cudaStream_t s) {
  for (auto ev : e.users) cudaStreamWaitEvent(s, ev, 0), cudaEventDestroy(ev);
  e.users.clear();
  if (e.ready) cudaStreamWaitEvent(s, e.ready, 0), cudaEventDestroy(e.ready);
  e.ready = nullptr;
  ctx->arena.release(e.block, s);
}

// Drop cached graphs and D-sets that reference table `id` (called on free),
// their memory released in the order of stream `s`.  Takes ctx->mu itself.
void forget_table(pq_ctx* ctx, uint64_t id, cudaStream_t s) {
  std::vector<GraphEntry> graphs;
  std::list<DsetEntry> sets;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->plan_cache) {
      auto& v = ctx->plan_cache->entries;
      for (auto it = v.begin(); it != v.end();) {
        if (it->tids[0] == id || it->tids[1] == id || it->tids[2] == id) {
          graphs.push_back(*it);
          it = v.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (auto it = ctx->dsets.begin(); it != ctx->dsets.end();) {
      auto nx = std::next(it);
      if (it->table_id == id) {
        if (it->pins > 0) it->dead = true;  // released by its last user
        else sets.splice(sets.end(), ctx->dsets, it);
      }
      it = nx;
    }
  }
  for (auto& e : graphs) graph_release(ctx, e, s);
  for (auto& e : sets) dset_release(ctx, e, s);
}

// ------------------------------------------------------------------ batch ----
pq_status read_back(pq_ctx* ctx, pq_result* results, const pq_result* dev, int n,
                    cudaStream_t s) {
  const size_t bytes = sizeof(pq_result) * n;
  ctx->d2h += (int64_t)bytes;
  if (is_pinned(results)) {
    PQ_CUDA(ctx, cudaMemcpyAsync(results, dev, bytes, cudaMemcpyDeviceToHost, s));
    return PQ_OK;
  }
  pq_result* tmp = nullptr;
  PQ_CUDA(ctx, cudaHostAlloc((void**)&tmp, bytes, 0));
  cudaError_t e = cudaMemcpyAsync(tmp, dev, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) memcpy(results, tmp, bytes);
  cudaFreeHost(tmp);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "result read-back");
  return PQ_OK;
}

static bool same_dset(const ResolvedPlan& a, const pq_plan& pa, const ResolvedPlan& b,
                      const pq_plan& pb) {
  return pa.D->id == pb.D->id && a.d_row0 == b.d_row0 && a.n_d == b.n_d &&
         a.dev.pd.lo == b.dev.pd.lo && a.dev.pd.hi == b.dev.pd.hi &&
         a.dev.pd.neg == b.dev.pd.neg && a.dev.lf1024 == b.dev.lf1024;
}

size_t batch_workspace_bytes(pq_ctx* ctx, const pq_plan* plans, int n) {
  size_t total = batch_layout(n).end;
  for (int i = 0; i < n; ++i) {
    ResolvedPlan r;
    if (resolve_plan(ctx, plans[i], r, true) != PQ_OK) return 0;
    total += plan_bytes(r);
  }
  return total;
}

pq_status run_batch_internal(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                             cudaStream_t s, bool allow_graph, const MWindow* win) {
  if (n <= 0 || !plans || !results) return fail(ctx, PQ_ERR_INVALID_ARG, "batch: bad arguments");
  for (int i = 0; i < n; ++i)
    if (plans[i].flags & PQ_PLAN_AGG_FIRST) {  // aggregate-first plans run one by one
      for (int j = 0; j < n; ++j) {
        pq_status st = plans[j].flags & PQ_PLAN_AGG_FIRST
                           ? run_plan_aggfirst(ctx, plans[j], &results[j], s)
                           : run_batch_internal(ctx, &plans[j], 1, &results[j], s, false);
        if (st != PQ_OK) return st;
      }
      return PQ_OK;
    }
  std::vector<ResolvedPlan> R(n);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  for (int i = 0; i < n; ++i) {
    pq_status st = resolve_plan(ctx, plans[i], R[i], false);
    if (st != PQ_OK) return st;
    if (!R[i].resident[0] || !R[i].resident[1] || !R[i].resident[2])
      return run_batch_streaming(ctx, plans, n, results, s);  // some table is streamed
    plan_static(ctx, plans[i], R[i], s, cap != cudaStreamCaptureStatusNone);
  }
  set_kernel_variants(false, win != nullptr);
  if (win) {  // one pass of an out-of-core plan: its M key window
    if (n != 1 || !R[0].dev.m_static) return fail(ctx, PQ_ERR_INVALID_ARG, "plan pass");
    R[0].dev.m_su = win->lo;
    R[0].dev.m_sb = win->bits;
    R[0].m_cap = win->cap;
    allow_graph = false;
  }
  // Graph replay for a repeated single plan.
  const bool graphable = allow_graph && n == 1 && s != nullptr && !ctx->opt.profile &&
                         cap == cudaStreamCaptureStatusNone &&
                         !(plans[0].flags & (PQ_PLAN_NO_GRAPH | PQ_PLAN_CACHE_DSET));
  std::string gkey;
  if (graphable) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->plan_cache) ctx->plan_cache = new PlanCache();
    gkey = plan_key(ctx, plans[0]);
    for (auto& e : ctx->plan_cache->entries) {
      if (e.key != gkey) continue;
      e.last_use = ++ctx->plan_cache->tick;
      PQ_CUDA(ctx, cudaStreamWaitEvent(s, e.done, 0));
      PQ_CUDA(ctx, cudaGraphLaunch(e.exec, s));
      PQ_CUDA(ctx, cudaEventRecord(e.done, s));
      ctx->replays++;
      ctx->plans++;
      ctx->launches += e.kernels;
      return read_back(ctx, results, e.out, 1, s);
    }
  }

  // D-set sharing inside the batch and across batches (cache).  Cached
  // entries found here are pinned until this batch has recorded its
  // completion on them; new entries are built into blocks of their own and
  // join the cache only once their build is queued.  No host wait happens
  // under ctx->mu.
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  std::vector<cudaEvent_t> waits;
  std::vector<DsetEntry*> pinned;   // cached entries this batch reads
  std::list<DsetEntry> fresh;       // entries this batch builds
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    for (int i = 0; i < n; ++i) {
      ResolvedPlan& r = R[i];
      for (int j = 0; j < i; ++j)
        if (R[j].builds && same_dset(R[j], plans[j], r, plans[i])) {
          r.builds = false;
          r.dset_from = j;
          break;
        }
      if (!r.builds || !(plans[i].flags & PQ_PLAN_CACHE_DSET) || capturing) continue;
      for (auto& e : ctx->dsets) {
        if (!e.dead && e.table_id == plans[i].D->id && e.row0 == r.d_row0 && e.rows == r.n_d &&
            e.pred.lo == r.dev.pd.lo && e.pred.hi == r.dev.pd.hi && e.pred.neg == r.dev.pd.neg &&
            e.lf1024 == r.dev.lf1024) {
          r.builds = false;
          r.dset_from = -2;
          r.cache = &e;
          e.last_use = ++ctx->dset_tick;
          // Completed readers need no ordering any more.
          for (auto it = e.users.begin(); it != e.users.end();) {
            if (cudaEventQuery(*it) == cudaSuccess) cudaEventDestroy(*it), it = e.users.erase(it);
            else ++it;
          }
          cudaGetLastError();
          if (e.pins++ == 0 || std::find(pinned.begin(), pinned.end(), &e) == pinned.end())
            pinned.push_back(&e);
          else
            e.pins--;  // already pinned by this batch
          waits.push_back(e.ready);
          break;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    ResolvedPlan& r = R[i];
    if (!r.builds || !(plans[i].flags & PQ_PLAN_CACHE_DSET) || capturing) continue;
    DsetEntry e{};
    e.table_id = plans[i].D->id;
    e.row0 = r.d_row0;
    e.rows = r.n_d;
    e.pred = r.dev.pd;
    e.lf1024 = r.dev.lf1024;
    e.log2max = r.e_d;
    e.bm = r.dev.d_static != 0;  // built from the static range
    e.block = ctx->arena.alloc(dset_block_bytes(r.e_d));
    if (!e.block) continue;  // no room to cache: build in the workspace
    if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ctx->arena.release_now(e.block);
      continue;
    }
    e.keys = nullptr;  // laid out by dset_block_assign
    fresh.push_back(e);
    r.cache = &fresh.back();
    r.cache_new = true;
    r.dset_from = -3;  // builds into a new cache block
  }
  // Undo the cache bookkeeping of a batch that does not run.
  auto unwind = [&]() {
    std::list<DsetEntry> drop;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      for (DsetEntry* e : pinned)
        if (--e->pins == 0 && e->dead)
          for (auto it = ctx->dsets.begin(); it != ctx->dsets.end(); ++it)
            if (&*it == e) {
              drop.splice(drop.end(), ctx->dsets, it);
              break;
            }
    }
    for (auto& e : drop) dset_release(ctx, e, s);
    for (auto& e : fresh) {
      if (e.ready) cudaEventDestroy(e.ready), e.ready = nullptr;
      ctx->arena.release(e.block, s);
    }
    pinned.clear();
    fresh.clear();
  };
  // After the chain is queued: the new sets are ready after it, every entry
  // the batch touched records the batch's completion, the new entries join
  // the cache, and the least recently used unpinned entries beyond 64 leave it.
  auto commit = [&]() {
    for (auto& e : fresh) cudaEventRecord(e.ready, s);
    std::vector<std::pair<DsetEntry*, cudaEvent_t>> marks;
    auto mark = [&](DsetEntry* e) {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventRecord(ev, s) == cudaSuccess)
        marks.push_back({e, ev});
      else if (ev)
        cudaEventDestroy(ev);
      cudaGetLastError();
    };
    for (DsetEntry* e : pinned) mark(e);
    for (auto& e : fresh) mark(&e);
    std::list<DsetEntry> drop;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      for (auto& m : marks) m.first->users.push_back(m.second);
      for (auto& e : fresh) e.last_use = ++ctx->dset_tick;
      ctx->dsets.splice(ctx->dsets.end(), fresh);
      for (DsetEntry* e : pinned) e->pins--;
      for (auto it = ctx->dsets.begin(); it != ctx->dsets.end();) {
        auto nx = std::next(it);
        if (it->dead && it->pins == 0) drop.splice(drop.end(), ctx->dsets, it);
        it = nx;
      }
      while (ctx->dsets.size() > 64) {
        auto old = ctx->dsets.end();
        for (auto it = ctx->dsets.begin(); it != ctx->dsets.end(); ++it)
          if (it->pins == 0 && (old == ctx->dsets.end() || it->last_use < old->last_use)) old = it;
        if (old == ctx->dsets.end()) break;
        drop.splice(drop.end(), ctx->dsets, old);
      }
    }
    for (auto& e : drop) dset_release(ctx, e, s);
    pinned.clear();
  };

  const BatchLayout L = batch_layout(n);
  size_t total = L.end;
  std::vector<size_t> off(n);
  for (int i = 0; i < n; ++i) {
    off[i] = total;
    total += plan_bytes(R[i]);
  }
  char* ws = (char*)ctx->arena.alloc(total);
  if (!ws) {
    unwind();
    return fail(ctx, PQ_ERR_BUDGET, "batch of %d plans needs %zu bytes (largest free %zu)", n,
                total, ctx->arena.largest_free());
  }
  bool any_build = false, vec = true, list_d = false, list_m = false, bm_dm = true;
  bool any_part = false;
  std::vector<std::pair<void*, size_t>> clears;  // static D bitmaps to zero first
  std::vector<std::pair<void*, size_t>> m_clears;  // static M bitmaps: the D scan clears them
  i64 tmax[kPhaseTopk + 1] = {0};  // largest tile count of each phase
  std::vector<char> host(L.upload_bytes());
  PlanDev* descs = (PlanDev*)host.data();
  i64* tD = (i64*)(host.data() + (L.tD - L.desc));
  i64* tM = (i64*)(host.data() + (L.tM - L.desc));
  i64* tF = (i64*)(host.data() + (L.tF - L.desc));
  tD[0] = tM[0] = tF[0] = 0;
  QCtr* ctr = (QCtr*)(ws + L.ctr);
  pq_result* out = (pq_result*)(ws + L.out);
  for (int i = 0; i < n; ++i) {
    ResolvedPlan& r = R[i];
    plan_assign(r, ws + off[i]);
    PlanDev& d = r.dev;
    if (r.dset_from >= 0) {
      const PlanDev& src = R[r.dset_from].dev;
      d.dset_log2 = src.dset_log2;
      d.dset_tag = src.dset_tag;
    } else if (r.cache) {
      dset_block_assign((char*)r.cache->block, r.cache->log2max, d);
    }
    d.ctr = ctr + i;
    d.out = out + i;
    any_build = any_build || r.builds;
    vec = vec && d.vec;
    if (r.builds && d.d_static)
      clears.push_back({(char*)d.dset_tag + table_layout(r.e_d, false).keybm,
                        (size_t)((d.d_sb + 127) / 128 * 16)});
    if (d.m_static) m_clears.push_back({(void*)d.ht_tag, (size_t)dense_layout(0, d.m_sb).tdir});
    if (d.part_log2) {
      any_part = true;
      clears.push_back({(void*)d.part, (size_t)((1 << d.part_log2) + 1) * 8});
      tmax[kPhaseFpart] += (r.n_f + kPT - 1) / kPT;
      tmax[kPhaseFscatter] += (r.n_f + kPT - 1) / kPT;
      tmax[kPhaseFagg] += (r.n_f + 8 * kAT - 1) / (8 * kAT);
    }
    list_d = list_d || (r.builds && !d.d_static);
    list_m = list_m || !d.m_static;
    // The D-set is a bitmap for certain when it is built here from a static
    // range, or was built so (an earlier plan of the batch, or the cache).
    const bool d_bm = r.builds                ? d.d_static != 0
                      : r.dset_from >= 0      ? R[r.dset_from].builds && R[r.dset_from].dev.d_static
                      : r.cache != nullptr    ? r.cache->bm
                                              : false;
    bm_dm = bm_dm && d.m_static && d_bm;
    descs[i] = d;
    tD[i + 1] = tD[i] + (r.builds ? (r.n_d + r.dev.d_tile - 1) / r.dev.d_tile : 0);
    tM[i + 1] = tM[i] + (r.n_m + r.dev.m_tile - 1) / r.dev.m_tile;
    tF[i + 1] = tF[i] + (r.n_f + r.dev.f_tile - 1) / r.dev.f_tile;
    if (r.builds) {
      tmax[kPhaseDfill] += fill_tiles(r.e_d, false, 32ULL << r.e_d);
      tmax[kPhaseDbuild] += (r.n_d + kTB - 1) / kTB;
    }
    tmax[kPhaseMfill] += fill_tiles(r.e_m, true, 32ULL << r.e_m);
    tmax[kPhaseMbuild] += (r.n_m + kTB - 1) / kTB;
    const u64 mbits = d.m_static ? d.m_sb : (32ULL << r.e_m);  // bound on the M bitmap
    tmax[kPhaseMrank] += (i64)(((mbits + 511) / 512 + kRankTile - 1) / kRankTile);
    tmax[kPhaseMdup] += (r.n_m + kTB - 1) / kTB;
    tmax[kPhaseTopk] += topk_parts(r.e_m);
  }
  tmax[kPhaseD] = tD[n];
  tmax[kPhaseM] = tM[n];
  tmax[kPhaseFscan] = tF[n];
  tmax[kPhaseF] = 0;
  for (int i = 0; i < n; ++i) tmax[kPhaseF] += (R[i].n_f + 63) / 64;

  cudaError_t ue = cudaSuccess;
  for (auto ev : waits)
    if (ue == cudaSuccess) ue = cudaStreamWaitEvent(s, ev, 0);
  if (ue == cudaSuccess) ue = ctx->ring.upload(ws + L.desc, host.data(), host.size(), s);
  if (ue != cudaSuccess) {
    unwind();
    ctx->arena.release(ws, s);
    return cuda_fail(ctx, ue, "batch set-up");
  }
  Batch b = make_batch(ctx, ws, n, L);
  b.clear_m = any_build ? 1 : 0;  // else no D scan runs: the memsets clear them
  if (!any_build) clears.insert(clears.end(), m_clears.begin(), m_clears.end());

  // The chain of phases.  With a side stream (graph capture), the rank and
  // copy-count passes of the M dictionary run beside the F scan, which only
  // tests the M bitmap; the F probe waits for both.
  auto chain = [&](cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) -> pq_status {
    PQ_CUDA(ctx, cudaMemsetAsync(ws + L.work, 0, L.zero_bytes(), s));
    for (auto& c : clears) PQ_CUDA(ctx, cudaMemsetAsync(c.first, 0, c.second, s));
    // The first phase that reads the M dictionary's directories.
    const int first_probe = any_part ? kPhaseFpart : kPhaseF;
    for (int ph = any_build ? kPhaseD : kPhaseM; ph <= kPhaseTopk; ++ph) {
      // Phases only plans with key lists need.
      if (!list_d && (ph == kPhaseDfill || ph == kPhaseDbuild)) continue;
      if (!list_m && (ph == kPhaseMfill || ph == kPhaseMbuild)) continue;
      if (!any_part && part_phase(ph)) continue;
      cudaStream_t on = s;
      if (side && ph == kPhaseMrank) {
        PQ_CUDA(ctx, cudaEventRecord(fork, s));
        PQ_CUDA(ctx, cudaStreamWaitEvent(side, fork, 0));
      }
      if (side && (ph == kPhaseMrank || ph == kPhaseMdup)) on = side;
      if (side && ph == first_probe) PQ_CUDA(ctx, cudaStreamWaitEvent(s, join, 0));
      pq_status st = launch_phase(ctx, ph, b, vec, on, tmax[ph], list_m, bm_dm);
      if (st != PQ_OK) return st;
      if (side && ph == kPhaseMdup) PQ_CUDA(ctx, cudaEventRecord(join, side));
    }
    return PQ_OK;
  };

  pq_status st = PQ_OK;
  if (graphable) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    bool captured = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess &&
                    cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const int64_t launches0 = ctx->launches.load();
    if (captured) {
      st = chain(side, fork, join);
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      captured = st == PQ_OK && e == cudaSuccess &&
                 cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (side) cudaStreamDestroy(side);
    cudaGetLastError();
    if (captured) {
      GraphEntry e;
      e.key = gkey;
      e.tids[0] = plans[0].D->id;
      e.tids[1] = plans[0].M->id;
      e.tids[2] = plans[0].F->id;
      e.ws = ws;
      e.out = out;
      e.exec = exec;
      e.kernels = ctx->launches.load() - launches0;  // counted while capturing
      cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming);
      PQ_CUDA(ctx, cudaGraphLaunch(exec, s));
      PQ_CUDA(ctx, cudaEventRecord(e.done, s));
      ctx->plans++;
      std::vector<GraphEntry> evicted;  // least recently used beyond 16 graphs
      {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto& v = ctx->plan_cache->entries;
        if (v.size() >= 16) {
          auto old = std::min_element(v.begin(), v.end(), [](const GraphEntry& a,
                                                              const GraphEntry& c) {
            return a.last_use < c.last_use;
          });
          evicted.push_back(*old);
          v.erase(old);
        }
        e.last_use = ++ctx->plan_cache->tick;
        v.push_back(e);
      }
      for (auto& o : evicted) graph_release(ctx, o, s);
      return read_back(ctx, results, out, 1, s);
    }
    if (st != PQ_OK) {
      ctx->arena.release(ws, s);
      return st;
    }
  }
  st = chain(nullptr, nullptr, nullptr);
  if (st == PQ_OK) {
    commit();
    st = read_back(ctx, results, out, n, s);
    ctx->plans += n;
  } else {
    unwind();
  }
  ctx->arena.release(ws, s);
  return st;
}

// The results of the passes of an out-of-core plan (disjoint groups): top-k
// of their top-k lists, summed group and hit counts, the first error.
static void merge_passes(const std::vector<pq_result>& parts, int k, pq_result* out) {
  std::vector<std::pair<int64_t, int64_t>> all;  // (sum, key)
  pq_result r{};
  for (const pq_result& p : parts) {
    for (int64_t i = 0; i < p.n; ++i) all.push_back({p.sums[i], p.keys[i]});
    r.ngroups += p.ngroups;
    r.hits += p.hits;
    if (!r.status) r.status = p.status;
  }
  std::sort(all.begin(), all.end(), [](const std::pair<int64_t, int64_t>& a,
                                       const std::pair<int64_t, int64_t>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  });
  r.n = std::min<int64_t>(k, (int64_t)all.size());
  for (int64_t i = 0; i < r.n; ++i) r.sums[i] = all[i].first, r.keys[i] = all[i].second;
  *out = r;
}

// A join-first plan over resident (or mapped) tables.  When its workspace
// does not fit the arena and its M side is a static dense dictionary, the
// build side is radix-partitioned by key range (the M key column's
// histogram of kHistBuckets buckets) and the plan runs in passes, each over
// the consecutive buckets whose dictionary fits: the M scan keeps the
// members of the pass's key window and the F scan hits only their keys
// (Sec. 3.4: chunks keep memory bounded; Sec. 3.1: partition, then build
// and probe per partition).  The passes' groups are disjoint; their results
// are merged on the host, so such a call returns when the plan is done.
pq_status run_plan_resident(pq_ctx* ctx, const pq_plan& p, pq_result* result, cudaStream_t s) {
  pq_status st = run_batch_internal(ctx, &p, 1, result, s, true);
  if (st != PQ_ERR_BUDGET) return st;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (s) cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone) return st;
  ResolvedPlan r;
  if (resolve_plan(ctx, p, r, false) != PQ_OK) return st;
  plan_static(ctx, p, r, s, false);
  if (!r.dev.m_static || !ensure_key_hist(ctx, p.M, 0, s)) return st;
  const std::string why = ctx->last_error;
  const size_t head = batch_layout(1).end;
  const size_t budget = ctx->arena.largest_free();
  const KeyHist& h = p.M->cols[0].hist;
  const u64 umin = p.M->cols[0].range.umin, umax = p.M->cols[0].range.umax;
  auto window = [&](int b0, int b1) {  // buckets [b0, b1)
    MWindow w;
    w.lo = umin + ((u64)b0 << h.shift);
    const u64 hi = std::min<u64>(umax, umin + ((u64)b1 << h.shift) - 1);  // last key
    w.bits = hi - w.lo + 1;
    w.cap = 0;
    for (int b = b0; b < b1; ++b) w.cap += h.counts[b];
    return w;
  };
  auto fits = [&](const MWindow& w) {
    ResolvedPlan q = r;
    q.dev.m_sb = w.bits;
    q.m_cap = w.cap;
    return head + plan_bytes(q) <= budget;
  };
  const int nb = (int)std::min<u64>(kHistBuckets, ((umax - umin) >> h.shift) + 1);
  std::vector<MWindow> wins;
  for (int b0 = 0; b0 < nb;) {
    int b1 = b0 + 1;
    if (!fits(window(b0, b1)))
      return fail(ctx, PQ_ERR_BUDGET,
                  "%s; out of core, one key bucket of M (%lld rows) does not fit either",
                  why.c_str(), (long long)window(b0, b1).cap);
    while (b1 < nb && fits(window(b0, b1 + 1))) ++b1;
    wins.push_back(window(b0, b1));
    b0 = b1;
  }
  pq_result* parts = nullptr;
  PQ_CUDA(ctx, cudaHostAlloc((void**)&parts, sizeof(pq_result) * wins.size(), 0));
  st = PQ_OK;
  for (size_t i = 0; i < wins.size() && st == PQ_OK; ++i)
    st = run_batch_internal(ctx, &p, 1, &parts[i], s, false, &wins[i]);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == PQ_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "out-of-core plan");
  if (st == PQ_OK) {
    merge_passes(std::vector<pq_result>(parts, parts + wins.size()), p.k, result);
    ctx->plans -= (int64_t)wins.size() - 1;
    ctx->passes += (int64_t)wins.size();
  }
  cudaFreeHost(parts);
  return st;
}

}  // namespace pqh

extern "C" {

pq_status pq_run_plan(pq_ctx* ctx, const pq_plan* plan, pq_result* result, void* stream) {
  if (!ctx || !plan || !result) return PQ_ERR_INVALID_ARG;
  if (plan->flags & PQ_PLAN_AGG_FIRST)
    return pqh::run_plan_aggfirst(ctx, *plan, result, pqh::S(stream));
  pqh::ResolvedPlan r;
  pq_status st = pqh::resolve_plan(ctx, *plan, r, false);
  if (st != PQ_OK) return st;
  if (!r.resident[0] || !r.resident[1] || !r.resident[2])
    return pqh::run_plan_streaming(ctx, plan, result, pqh::S(stream));
  return pqh::run_plan_resident(ctx, *plan, result, pqh::S(stream));
}

pq_status pq_run_batch(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                       void* stream) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  return pqh::run_batch_internal(ctx, plans, n, results, pqh::S(stream), false);
}

}  // extern "C"
