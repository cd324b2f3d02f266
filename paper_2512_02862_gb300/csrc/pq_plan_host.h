// pq_plan_host.h -- host-side plan resolution and workspace layout shared by
// the resident (pq_plan.cu) and streaming (pq_stream.cu) plan drivers.
#pragma once
#include "pq_internal.h"
#include "pq_plan_kernels.cuh"

namespace pqh {

// A plan resolved against its tables: row ranges, predicates, sizes.
struct ResolvedPlan {
  pqk::PlanDev dev{};
  i64 n_d = 0, n_m = 0, n_f = 0;
  i64 d_row0 = 0, m_row0 = 0, f_row0 = 0;
  int e_d = 6, e_m = 6;   // log2 of the largest D-set / M-table slot counts
  i64 parts = 1;          // top-k tiles at most
  bool builds = true;     // fills its D-set in this batch
  int dset_from = -1;     // -1 own block, >= 0 builder index in the batch, -2 cache
  DsetEntry* cache = nullptr;
  bool cache_new = false;
  bool resident[3] = {false, false, false};
  i64 m_cap = -1;         // members the dense dictionary is sized for (-1: n_m)
};

// Validate `p`; fill predicates, sizes and (for resident tables) the column
// pointers of r.dev.  need_resident: every table must be resident.
pq_status resolve_plan(pq_ctx* ctx, const pq_plan& p, ResolvedPlan& r, bool need_resident);

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Rows per warp tile of a scan over n rows: the largest unit * 2^j, up to
// max_rows, that still gives each of `warps` resident warps two tiles.
inline int scan_tile(i64 n, int unit, int max_rows, i64 warps) {
  int t = max_rows;
  while (t > unit && (n + t - 1) / t < 2 * warps) t >>= 1;
  return t;
}
// Resident warps of plan kernel `occ_index` (see plan_kernels_init).
inline i64 resident_warps(const pq_ctx* ctx, int occ_index) {
  return (i64)ctx->num_sms * std::max(1, std::min(ctx->tune_bps, ctx->plan_occ[occ_index])) * 8;
}

// A D-set block of 2^e slots: a 256-byte header (the log2 of the slot count
// in use, then the key-range bitmap's base and bit count) followed by a key
// set laid out by pqk::table_layout.
inline size_t dset_block_bytes(int e) { return 256 + pqk::table_layout(e, false).total; }
inline void dset_block_assign(char* blk, int, pqk::PlanDev& d) {
  d.dset_log2 = (int*)blk;
  d.dset_tag = (unsigned short*)(blk + 256);
}

// An M table of 2^e slots with {key, sum} records (pqk::table_layout).
inline size_t mtable_bytes(int e) { return al256(pqk::table_layout(e, true).total); }
inline char* mtable_assign(char* p, int e, pqk::PlanDev& d) {
  d.ht_tag = (unsigned short*)p;
  return p + mtable_bytes(e);
}

// The key range of column c of a resident table (Column::umin/umax), measured
// on first use by one kernel and a read-back on stream s; false if the column
// is not on the device or the table is empty.
bool ensure_range(pq_ctx* ctx, const pq_table* t, int c, cudaStream_t s);

// The aggregate-first plan (PQ_PLAN_AGG_FIRST; pq_agg.cu).
pq_status run_plan_aggfirst(pq_ctx* ctx, const pq_plan& plan, pq_result* result, cudaStream_t s);
// Arena bytes an aggregate-first plan needs; an error if it cannot run
// (tables not resident, keys not dense).  Measures the key ranges on first use.
pq_status aggfirst_bytes(pq_ctx* ctx, const pq_plan& plan, size_t* bytes);

// Per-plan workspace bytes (excluding a cached D-set block).
size_t plan_bytes(const ResolvedPlan& r);

// Carve the plan's workspace pointers out of `base` (as sized by plan_bytes).
void plan_assign(ResolvedPlan& r, char* base);

// Batch header layout inside the workspace.
struct BatchLayout {
  size_t desc = 0, tD = 0, tM = 0, tF = 0, dyn = 0, work = 0, ctr = 0, out = 0, end = 0;
  // Descriptors + static tile prefixes.  The dynamic prefixes that follow are
  // written by the kernels and must never be overwritten by a re-upload.
  size_t upload_bytes() const { return dyn - desc; }
  size_t zero_bytes() const { return out - work; }     // tickets + per-plan counters
};
BatchLayout batch_layout(int nq);

// The batch argument of every plan kernel for a workspace at `ws`.
pqk::Batch make_batch(pq_ctx* ctx, char* ws, int nq, const BatchLayout& L);

// Launch one phase of the plan chain for the whole batch.  vec: every column
// pointer 16-byte aligned.  tiles_max: the phase's largest possible tile
// count (-1 unknown), which caps the grid.  list_m: some plan keeps an M key
// list (else the M scan without list code runs).  bm_dm: every plan has a
// static M bitmap and a D-set bitmap (the ring-free M scan runs).
pq_status launch_phase(pq_ctx* ctx, int phase, const pqk::Batch& b, bool vec, cudaStream_t s,
                       i64 tiles_max = -1, bool list_m = true, bool bm_dm = false);
// Kernel variants for the launches that follow on this thread: the F scan
// that buffers hits, the M scan of an out-of-core pass's key window.
void set_kernel_variants(bool buffered_hits, bool key_window);

// Phases in chain order.  Fpart, Fscatter and Fagg run only for batches
// with a partitioned plan; the F probe (kPhaseF) always runs, for the plans
// that are not partitioned, and its last block sizes the top-k for all.
enum { kPhaseD = 0, kPhaseDfill, kPhaseDbuild, kPhaseM, kPhaseMfill, kPhaseMbuild, kPhaseMrank,
       kPhaseMdup, kPhaseFscan, kPhaseFpart, kPhaseFscatter, kPhaseFagg, kPhaseF, kPhaseTopk };
inline bool part_phase(int ph) {
  return ph == kPhaseFpart || ph == kPhaseFscatter || ph == kPhaseFagg;
}

}  // namespace pqh
