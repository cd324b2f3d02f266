// pq_agg.cu -- the aggregate-first plan (PQ_PLAN_AGG_FIRST): a large
// materialised group-by filtered on its aggregate (the shape of the paper's
// Q18 remark, Sec. 6.3), on resident tables with dense keys.
//
//   D' bitmap  <- D rows with seg op_d c_d                  (k_agg_dbits)
//   M' bitmap  <- M rows with date op_m c_m, dref in D'      (k_agg_mbits)
//   G          <- F rows with date2 op_f c_f: sums[mkey] += price*(100-disc),
//                 a group per set flag of the F key range    (k_agg_fscan,
//                                                             k_agg_fixup)
//   candidates <- keys of M' whose group exists and has sum > having
//                                                            (k_agg_select)
//   result     <- top-k of the candidates (the top-k operator's kernel) and
//                 their number                               (k_agg_result)
//
// The group sums live in a dense array over the F key range (8 bytes per key
// of the range), so the plan needs keys whose range is at most a few times
// the F row count.  Consecutive rows of the same group are added up inside
// the warp first.  When F's keys come in a few non-decreasing segments
// (measured once per key column), each segment is scanned by its own launch
// and every group's total is stored once (k_agg_fixup finishes the runs that
// tile edges cut); otherwise each run's total is one reduction into a zeroed
// array.  int64 overflow: a group sum can only leave int64 if the magnitudes
// of all summed revenues reach 2^62, which the plan tracks (one atomic per
// warp) and reports as PQ_ERR_OVERFLOW; a single revenue is formed exactly.
#include <algorithm>
#include <vector>

#include "pq_plan_host.h"

using namespace pqk;

namespace pqh {

namespace {

// Sorted F: the parts of the runs that a tile's edges cut.  P: the tile's
// first run, when it continues a run of the tile before; L: its last run,
// when the run goes on into the next tile (with that run's key).
struct TileEdge {
  u64 psum, lsum;
  i64 lkey;
  u32 pcnt, lcnt;  // non-zero when the part has a passing row
};

struct AggPlan {
  const int* d_key;
  const signed char* d_seg;
  i64 n_d;
  Pred pd;
  u64 d_base, d_bits;
  u32* dbm;
  const i64* m_key;
  const int* m_dref;
  const int* m_date;
  i64 n_m;
  Pred32 pm;
  u64 m_base, m_bits;
  u32* mbm;
  const i64* f_mkey;
  const i64* f_price;
  const signed char* f_disc;
  const int* f_date;
  i64 n_f;
  Pred32 pf;
  u64 f_base, f_bits;
  i64* sums;
  unsigned char* hit;  // one flag byte per key of the F range (padded to 16)
  int vec;             // F columns 16-byte aligned (mkey, price, date2) and disc 4-byte
  int mvec;            // M date and dref 16-byte aligned
  int accum;           // sorted F, not the first segment: groups may exist already
  TileEdge* edge;      // sorted F: per tile, the parts of runs cut by its edges
  unsigned char* eflag;  // sorted F: per tile, kCin | kCout | kWhole
  i64 having;
  i64* cand_k;
  i64* cand_s;
  u64* ctr;  // [0] candidates, [1] sum of |revenue| (saturating at 2^62), [2] F rows,
             // [3] status; bytes 128-131: the top-k's ticket (all zeroed per run)
  DevStatus* st;  // the context's error latch (read by pq_sync)
};

constexpr u64 kMag = 1ULL << 62;
constexpr int kCin = 1, kCout = 2, kWhole = 4;

// Sorted F: a group's total within one non-decreasing segment of F, stored
// by its only writer (the segments run one after another).
__device__ __forceinline__ void store_group(const AggPlan& a, u64 idx, u64 sum) {
  if (a.accum && a.hit[idx]) {
    a.sums[idx] = (i64)((u64)a.sums[idx] + sum);
  } else {
    a.sums[idx] = (i64)sum;
    a.hit[idx] = 1;
  }
}

__global__ void __launch_bounds__(256) k_agg_dbits(AggPlan a) {
  chain_begin();
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_d; i += stride)
    if (pass(a.pd, a.d_seg[i])) bit_set(a.dbm, ukey((i64)a.d_key[i]) - a.d_base);
}

// M rows, 4 consecutive rows per thread (vector loads of date and dref
// when aligned), so that each thread has 4 independent chains of loads in
// flight: date -> D' bit -> key -> M' bit.
__global__ void __launch_bounds__(256) k_agg_mbits(AggPlan a) {
  chain_begin();
  const u64 keep = policy_keep(), pol = policy_stream();
  const i64 n4 = (a.n_m + 3) / 4;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
    const i64 r0 = 4 * t;
    int dt[4], dr[4];
    if (a.mvec && r0 + 4 <= a.n_m) {
      const int4 d4 = ld_stream_v4(a.m_date + r0, pol), r4 = ld_stream_v4(a.m_dref + r0, pol);
      dt[0] = d4.x, dt[1] = d4.y, dt[2] = d4.z, dt[3] = d4.w;
      dr[0] = r4.x, dr[1] = r4.y, dr[2] = r4.z, dr[3] = r4.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool in = r0 + j < a.n_m;
        dt[j] = in ? a.m_date[r0 + j] : 0;
        dr[j] = in ? a.m_dref[r0 + j] : 0;
      }
    }
    bool ok[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      ok[j] = r0 + j < a.n_m && pass32(a.pm, dt[j]);
      const u64 di = ukey((i64)dr[j]) - a.d_base;
      ok[j] = ok[j] && di < a.d_bits && bit_test(a.dbm, di, keep);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (ok[j]) bit_set(a.mbm, ukey(a.m_key[r0 + j]) - a.m_base);
  }
}

// F rows in warp tiles of 128 consecutive rows, 4 consecutive rows per lane
// (vector loads when the columns are 16-byte aligned).  F is typically
// clustered by mkey, so the tile's rows form runs of equal keys: a segmented
// scan over the warp adds up each run (rows that fail the filter count 0) and
// the lane holding a run's last row commits it, if the run holds a passing
// row.  SORTED (one non-decreasing segment of F): a run is its group's only
// writer, so the commit is a plain store of the sum and the hit flag; runs
// that a tile edge cuts leave their parts in the tile's edge record for
// k_agg_fixup.  Otherwise each run's total is reduced into the zeroed sum
// array (exact for any key order) and its hit flag stored.  Partial sums are
// formed in wrapping 64-bit arithmetic, exact while the magnitudes of all
// revenues stay below 2^62 (otherwise the plan reports PQ_ERR_OVERFLOW).
template <bool SORTED>
__global__ void __launch_bounds__(256) k_agg_fscan(AggPlan a) {
  chain_begin();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 pol = policy_stream();
  const i64 nw = (i64)gridDim.x * (blockDim.x >> 5);
  u64 mag = 0, rows = 0;
  bool ovf = false;
  for (i64 g = (i64)blockIdx.x * (blockDim.x >> 5) + warp; g * 128 < a.n_f; g += nw) {
    const i64 r0 = g * 128 + 4 * lane;
    i64 k[4], p[4];
    int dt[4], dc[4];
    if (a.vec && g * 128 + 128 <= a.n_f) {
      const int4 d4 = ld_stream_v4(a.f_date + r0, pol);
      const longlong2 k01 = ld_stream_v2(a.f_mkey + r0, pol), k23 = ld_stream_v2(a.f_mkey + r0 + 2, pol);
      const longlong2 p01 = ld_stream_v2(a.f_price + r0, pol), p23 = ld_stream_v2(a.f_price + r0 + 2, pol);
      const u32 c4 = __ldcs(reinterpret_cast<const unsigned int*>(a.f_disc + r0));
      dt[0] = d4.x, dt[1] = d4.y, dt[2] = d4.z, dt[3] = d4.w;
      k[0] = k01.x, k[1] = k01.y, k[2] = k23.x, k[3] = k23.y;
      p[0] = p01.x, p[1] = p01.y, p[2] = p23.x, p[3] = p23.y;
#pragma unroll
      for (int j = 0; j < 4; ++j) dc[j] = (int)(signed char)(c4 >> (8 * j));
    } else {
      // Rows past the end take the last row's key and count 0: they extend
      // its run without changing it.
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const i64 r = min(r0 + j, a.n_f - 1);
        k[j] = a.f_mkey[r];
        p[j] = a.f_price[r];
        dc[j] = a.f_disc[r];
        dt[j] = r0 + j < a.n_f ? a.f_date[r] : 0;
      }
    }
    // Revenues of the passing rows (0 for the others), bit j of pm set when
    // row j passes.  Prices that fit in 32 bits (the common case) give
    // revenues below 2^39: a 32 x 32 -> 64-bit product and one saturating
    // magnitude update per tile; larger ones take the exact 128-bit product.
    u64 v[4];
    u32 pm = 0;
    bool small = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pm |= (r0 + j < a.n_f && pass32(a.pf, dt[j]) ? 1u : 0u) << j;
      small = small && p[j] == (i64)(int)p[j];
    }
    if (small) {
      u64 tm = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const i64 r = (i64)(int)p[j] * (i64)(100 - dc[j]);
        const bool in = (pm >> j) & 1u;
        v[j] = in ? (u64)r : 0;
        tm += in ? (r < 0 ? (u64)0 - (u64)r : (u64)r) : 0;
      }
      mag = mag >= kMag ? kMag : min(kMag, mag + tm);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool in = (pm >> j) & 1u;
        const __int128 rev = (__int128)p[j] * (100 - dc[j]);
        const i64 r64 = (i64)rev;
        ovf = ovf || (in && rev != (__int128)r64);
        v[j] = in ? (u64)r64 : 0;
        const u64 m = r64 < 0 ? (u64)0 - (u64)r64 : (u64)r64;
        if (in) mag = mag >= kMag || m >= kMag ? kMag : min(kMag, mag + m);
      }
    }
    rows += __popc(pm);
    // Run heads: a row whose key differs from the row before it.
    const i64 prev = __shfl_up_sync(kFull, k[3], 1);
    bool head[4];
    head[0] = lane == 0 || k[0] != prev;
#pragma unroll
    for (int j = 1; j < 4; ++j) head[j] = k[j] != k[j - 1];
    // The lane's last run: its part inside the lane; fl bit 0: it starts in
    // this lane, bit 1: one of its rows passes.
    u64 ls = 0;
    u32 fl = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (head[j]) ls = 0, fl = 1;
      ls += v[j];
      fl |= ((pm >> j) & 1u) << 1;
    }
    // Segmented inclusive scan over lanes: the lane's last run summed back
    // to the lane where it starts.  It ends as soon as every lane has reached
    // its run's start (runs span few lanes: usually one or two steps).
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (__all_sync(kFull, fl & 1u)) break;
      const u64 us = __shfl_up_sync(kFull, ls, o);
      const u32 uf = __shfl_up_sync(kFull, fl, o);
      if (lane >= o) {
        if (!(fl & 1u)) ls += us, fl |= uf & 2u;
        fl |= uf & 1u;
      }
    }
    // The run entering the lane from the left, and whether the next lane
    // starts a new run.
    const u64 in_s = __shfl_up_sync(kFull, ls, 1);
    const u32 in_p = __shfl_up_sync(kFull, fl, 1) >> 1;
    const bool next_head = __shfl_down_sync(kFull, head[0], 1);
    // Sorted F: does the tile's first row continue the run of the row before
    // it (cin), its last row go on into the next tile (cout)?  A run is the
    // tile's first run if no head lies inside the tile before its end.
    bool cin = false, cout = false, first = false;
    u32 ih = 0;
    if (SORTED) {
      const i64 t0 = g * 128;
      bool e = false;
      if (lane == 0 && t0 > 0) e = a.f_mkey[t0 - 1] == k[0];
      if (lane == 31 && t0 + 128 < a.n_f) e = a.f_mkey[t0 + 128] == k[3];
      cin = __shfl_sync(kFull, e, 0);
      cout = __shfl_sync(kFull, e, 31);
      ih = __ballot_sync(kFull, head[1] || head[2] || head[3] || (lane > 0 && head[0]));
      first = (ih & lanemask_lt()) == 0 && !(lane > 0 && head[0]);
    }
    u64 acc = head[0] ? 0 : in_s;
    u32 cnt = head[0] ? 0 : in_p;  // non-zero when the run has a passing row
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j > 0 && head[j]) acc = 0, cnt = 0, first = false;
      acc += v[j];
      cnt |= (pm >> j) & 1u;
      const bool end = j < 3 ? head[j + 1] : (lane == 31 || next_head);
      if (!end) continue;
      const u64 idx = ukey(k[j]) - a.f_base;
      if (SORTED) {
        // A run that no tile edge cuts is this tile's alone: a plain store.
        const bool pcut = first && cin, lcut = lane == 31 && j == 3 && cout;
        if (pcut) a.edge[g].psum = acc, a.edge[g].pcnt = cnt;
        if (lcut) a.edge[g].lsum = acc, a.edge[g].lcnt = cnt, a.edge[g].lkey = k[j];
        if (!pcut && !lcut && cnt) store_group(a, idx, acc);
      } else if (cnt) {
        atomicAdd(reinterpret_cast<unsigned long long*>(a.sums + idx), (unsigned long long)acc);
        a.hit[idx] = 1;
      }
    }
    if (SORTED && lane == 0)
      a.eflag[g] = (unsigned char)((cin ? kCin : 0) | (cout ? kCout : 0) | (ih == 0 ? kWhole : 0));
  }
  // The warp's magnitude total (saturating) and row count: one atomic each.
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const u64 x = __shfl_xor_sync(kFull, mag, o);
    mag = mag >= kMag || x >= kMag ? kMag : min(kMag, mag + x);
    rows += __shfl_xor_sync(kFull, rows, o);
  }
  ovf = __any_sync(kFull, ovf);
  if (lane == 0) {
    if (rows) atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr + 2), rows);
    if (mag) {
      const u64 old = atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr + 1), mag);
      if (old >= kMag || old + mag >= kMag) ovf = true;
    }
    if (ovf) {
      atomicExch(reinterpret_cast<unsigned long long*>(a.ctr + 3), (u64)PQ_ERR_OVERFLOW);
      latch(a.st, PQ_ERR_OVERFLOW, (i64)rows);
    }
  }
}

// Sorted F: the runs that tile edges cut.  The tile holding a cut run's
// head (its last run goes on, and it is not a whole-tile piece of a run
// begun earlier) adds the next tiles' first-run parts while they are whole
// tiles that go on, then the part where the run ends, and stores the total.
__global__ void __launch_bounds__(256) k_agg_fixup(AggPlan a, i64 ntiles) {
  chain_begin();
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 g = (i64)blockIdx.x * blockDim.x + threadIdx.x; g < ntiles; g += stride) {
    const int f = a.eflag[g];
    if (!(f & kCout) || ((f & kWhole) && (f & kCin))) continue;
    u64 sum = a.edge[g].lsum;
    u64 cnt = a.edge[g].lcnt;
    const i64 key = a.edge[g].lkey;
    for (i64 h = g + 1; h < ntiles; ++h) {  // a tile with kCout has a next tile
      sum += a.edge[h].psum;
      cnt += a.edge[h].pcnt;
      const int fh = a.eflag[h];
      if (!((fh & kWhole) && (fh & kCout))) break;
    }
    if (cnt) store_group(a, ukey(key) - a.f_base, sum);
  }
}

// The semi-join, from the M' side: each set bit of the M' bitmap (a key of
// M') whose group exists (hit flag) and whose sum exceeds the threshold is
// appended as a (key, sum) candidate.  M' is usually far smaller than the
// group count, so only its groups read their flag and sum.
__global__ void __launch_bounds__(256) k_agg_select(AggPlan a) {
  chain_begin();
  const int lane = threadIdx.x & 31;
  const i64 words = (i64)((a.m_bits + 31) / 32);
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 w0 = (i64)blockIdx.x * blockDim.x; w0 < words; w0 += stride) {
    const i64 w = w0 + threadIdx.x;
    u32 bits = w < words ? __ldcs(a.mbm + w) : 0u;
    while (__any_sync(kFull, bits)) {
      bool take = false;
      i64 key = 0, sum = 0;
      if (bits) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1;
        const u64 uk = a.m_base + (u64)w * 32 + (u64)j;
        const u64 idx = uk - a.f_base;
        if (idx < a.f_bits && a.hit[idx]) {
          sum = a.sums[idx];
          key = (i64)(uk ^ (1ULL << 63));
          take = sum > a.having;
        }
      }
      const u32 m = __ballot_sync(kFull, take);
      if (!m) continue;
      u64 at = 0;
      if (lane == __ffs(m) - 1)
        at = atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr), (unsigned long long)__popc(m));
      at = __shfl_sync(kFull, at, __ffs(m) - 1) + __popc(m & lanemask_lt());
      if (take) a.cand_k[at] = key, a.cand_s[at] = sum;
    }
  }
}

__global__ void k_agg_result(const u64* ctr, const i64* keys, const i64* sums,
                             const i64* nout, int k, pq_result* out) {
  chain_begin();
  const int t = threadIdx.x;
  const i64 n = *nout;
  if (t < k && t < n) out->keys[t] = keys[t], out->sums[t] = sums[t];
  if (t == 0) {
    out->n = n;
    out->ngroups = (i64)ctr[0];
    out->status = (int)ctr[3];
    out->reserved = 0;
    out->hits = (i64)ctr[2];
  }
}

// Launch of a plan kernel; `chained`: programmatic dependent launch (the
// kernel waits for its predecessor at entry, so only the launch overlaps).
template <typename... P, typename... A>
cudaError_t launch(void (*k)(P...), int grid, int block, cudaStream_t s, bool chained, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Blocks of 256 threads of kernel k resident per SM (at least 1).
template <typename K>
int resident_blocks(K k) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return std::max(n, 1);
}

}  // namespace

namespace {

// Sizes of an aggregate-first plan's workspace, from the tables' key ranges
// and key order (measured once per key column).
struct AggShape {
  u64 d_bits = 0, m_bits = 0, f_bits = 0;
  size_t cap = 1;       // candidates: at most one per key of M' inside the F range
  bool sorted = false;  // F scanned as its non-decreasing segments
  std::vector<i64> seg;  // segment starts within the plan's F rows, then n_f
  i64 ntiles = 0;        // tiles of the longest segment
  size_t head = 0, sums_bytes = 0, zero = 0, edge_bytes = 0, cand_bytes = 0;
};

size_t words_bytes(u64 bits) { return (size_t)((bits + 31) / 32) * 4; }

pq_status agg_shape(pq_ctx* ctx, const pq_plan& plan, const ResolvedPlan& r, cudaStream_t s,
                    AggShape& g) {
  const pq_table* T[3] = {plan.D, plan.M, plan.F};
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (s) cudaStreamIsCapturing(s, &cap);
  for (int t = 0; t < 3; ++t) {
    if (T[t]->nrows <= 0 || T[t]->cols[0].range.known()) continue;
    if (cap != cudaStreamCaptureStatusNone)
      return fail(ctx, PQ_ERR_INVALID_ARG,
                  "aggregate-first plan: run it once before capturing a stream (key ranges)");
    if (!ensure_range(ctx, T[t], 0, s))
      return fail(ctx, PQ_ERR_CUDA, "aggregate-first plan: key range of table %d", t);
  }
  auto span = [&](int t) -> u64 {
    const KeyRange& c = T[t]->cols[0].range;
    return c.known() && c.umax >= c.umin ? c.umax - c.umin + 1 : 0;
  };
  g.d_bits = span(0), g.m_bits = span(1);
  g.f_bits = r.n_f > 0 ? span(2) : 0;  // no F rows: no group, nothing to scan
  // The sum array spans the F table's key range: dense keys are required.
  const u64 dense_cap = 4ULL * (u64)std::max<i64>(T[2]->nrows, 1) + 4096;
  if (g.f_bits > dense_cap || g.f_bits > kMaxBmBits || g.m_bits > kMaxBmBits ||
      g.d_bits > kMaxBmBits)
    return fail(ctx, PQ_ERR_INVALID_ARG,
                "aggregate-first plan: F keys span %llu values for %lld rows (dense keys needed)",
                (unsigned long long)g.f_bits, (long long)T[2]->nrows);
  g.cap = (size_t)std::max<u64>(std::min(g.f_bits, g.m_bits), 1);
  // F as its non-decreasing segments of keys: in a segment each group is one
  // run of rows, stored once, so the sum array needs no zeroing.  More than
  // kMaxDescents segments: reductions into a zeroed array.
  const KeyRange& fk = T[2]->cols[0].range;
  g.sorted = fk.ndesc >= 0;
  g.seg.assign(1, 0);
  if (g.sorted)
    for (int j = 0; j < fk.ndesc; ++j)
      if (fk.desc[j] > r.f_row0 && fk.desc[j] < r.f_row0 + r.n_f) g.seg.push_back(fk.desc[j] - r.f_row0);
  g.seg.push_back(r.n_f);
  for (size_t j = 0; j + 1 < g.seg.size(); ++j)
    g.ntiles = std::max(g.ntiles, (g.seg[j + 1] - g.seg[j] + 127) / 128);
  // Zeroed: counters, D' and M' bitmaps, hit flags (and the sums unless sorted).
  g.head = 256 + al256(words_bytes(g.d_bits)) + al256(words_bytes(g.m_bits)) +
           al256((size_t)(g.f_bits + 15) / 16 * 16);
  g.sums_bytes = al256(8 * (size_t)std::max<u64>(g.f_bits, 1));
  g.zero = g.head + (g.sorted ? 0 : g.sums_bytes);
  g.edge_bytes = g.sorted ? al256(sizeof(TileEdge) * g.ntiles) + al256(g.ntiles) : 0;
  // Candidates, the top-k output and count, the result record, the top-k's lists.
  g.cand_bytes = al256(16 * g.cap) + al256(16 * PQ_MAX_K) + 256 + al256(sizeof(pq_result)) +
                 al256(topk_scratch_bytes(ctx, (int64_t)g.cap, PQ_MAX_K));
  return PQ_OK;
}

}  // namespace

pq_status aggfirst_bytes(pq_ctx* ctx, const pq_plan& plan, size_t* bytes) {
  ResolvedPlan r;
  AggShape g;
  pq_status st = resolve_plan(ctx, plan, r, true);
  if (st == PQ_OK) st = agg_shape(ctx, plan, r, nullptr, g);
  if (st != PQ_OK) return st;
  *bytes = g.head + g.sums_bytes + g.edge_bytes + al256(g.cand_bytes) + 2 * 256;
  return PQ_OK;
}

pq_status run_plan_aggfirst(pq_ctx* ctx, const pq_plan& plan, pq_result* result, cudaStream_t s) {
  ResolvedPlan r;
  pq_status st = resolve_plan(ctx, plan, r, true);
  if (st != PQ_OK) return st;
  const PlanDev& d = r.dev;
  const pq_table* T[3] = {plan.D, plan.M, plan.F};
  AggShape g;
  st = agg_shape(ctx, plan, r, s, g);
  if (st != PQ_OK) return st;
  const u64 d_bits = g.d_bits, m_bits = g.m_bits, f_bits = g.f_bits;
  const size_t cap = g.cap;
  const bool sorted = g.sorted;
  const std::vector<i64>& seg = g.seg;
  const size_t head = g.head, sums_bytes = g.sums_bytes, zero = g.zero, edge_bytes = g.edge_bytes;
  const i64 ntiles = g.ntiles;
  Scratch scr(ctx, s);
  char* z = (char*)scr.get(head + sums_bytes + edge_bytes);
  char* c = (char*)scr.get(g.cand_bytes);
  if (!z || !c)
    return fail(ctx, PQ_ERR_BUDGET, "aggregate-first plan: %zu bytes",
                head + sums_bytes + edge_bytes + g.cand_bytes);
  AggPlan a{};
  a.ctr = (u64*)z;
  a.dbm = (u32*)(z + 256);
  a.mbm = (u32*)((char*)a.dbm + al256(words_bytes(d_bits)));
  a.hit = (unsigned char*)a.mbm + al256(words_bytes(m_bits));
  a.sums = (i64*)(z + head);
  if (sorted) {
    a.edge = (TileEdge*)(z + head + sums_bytes);
    a.eflag = (unsigned char*)a.edge + al256(sizeof(TileEdge) * ntiles);
  }
  a.cand_k = (i64*)c;
  a.cand_s = a.cand_k + cap;
  i64* ok = (i64*)(c + al256(16 * cap));
  i64* os = ok + PQ_MAX_K;
  i64* nout = (i64*)(c + al256(16 * cap) + al256(16 * PQ_MAX_K));
  pq_result* dres = (pq_result*)((char*)nout + 256);
  void* lists = (char*)dres + al256(sizeof(pq_result));
  a.d_key = d.d_key, a.d_seg = d.d_seg, a.n_d = r.n_d, a.pd = d.pd;
  a.d_base = T[0]->cols[0].range.umin, a.d_bits = d_bits;
  a.m_key = d.m_key, a.m_dref = d.m_dref, a.m_date = d.m_date, a.n_m = r.n_m, a.pm = to32(d.pm);
  a.m_base = T[1]->cols[0].range.umin, a.m_bits = m_bits;
  a.f_mkey = d.f_mkey, a.f_price = d.f_price, a.f_disc = d.f_disc, a.f_date = d.f_date;
  a.n_f = r.n_f, a.pf = to32(d.pf);
  a.mvec = (uintptr_t)a.m_date % 16 == 0 && (uintptr_t)a.m_dref % 16 == 0;
  a.f_base = T[2]->cols[0].range.umin, a.f_bits = f_bits;
  a.having = plan.having;
  a.st = ctx->d_status;
  PQ_CUDA(ctx, cudaMemsetAsync(z, 0, zero, s));
  const int sms = ctx->num_sms;
  auto grid = [&](i64 n, i64 per) {
    return (int)std::max<i64>(1, std::min<i64>((n + per - 1) / per, (i64)sms * 8));
  };
  // The F scans are persistent: one wave of as many blocks as fit.
  static const int occ[2] = {resident_blocks(k_agg_fscan<false>), resident_blocks(k_agg_fscan<true>)};
  auto fgrid = [&](i64 n, bool srt) {
    return (int)std::max<i64>(1, std::min<i64>((n + 1023) / 1024, (i64)sms * occ[srt ? 1 : 0]));
  };
  // A table with rows has a measured range, so every key of the plan's rows
  // indexes inside its bitmap or sum array.
  // Kernels after the first are chained (programmatic dependent launch).
  bool chained = false;
  int launches = 0;
  auto go = [&](cudaError_t e) {
    chained = true;
    ++launches;
    return e;
  };
  if (d_bits) PQ_CUDA(ctx, go(launch(k_agg_dbits, grid(r.n_d, 256), 256, s, chained, a)));
  if (d_bits && m_bits)
    PQ_CUDA(ctx, go(launch(k_agg_mbits, grid((r.n_m + 3) / 4, 256), 256, s, chained, a)));
  if (f_bits) {
    for (size_t j = 0; j + 1 < seg.size(); ++j) {
      AggPlan b = a;
      const i64 off = seg[j];
      b.f_mkey += off, b.f_price += off, b.f_disc += off, b.f_date += off;
      b.n_f = seg[j + 1] - off;
      b.vec = (uintptr_t)b.f_mkey % 16 == 0 && (uintptr_t)b.f_price % 16 == 0 &&
              (uintptr_t)b.f_date % 16 == 0 && (uintptr_t)b.f_disc % 4 == 0;
      b.accum = j > 0;
      if (b.n_f <= 0) continue;
      if (sorted) {
        const i64 nt = (b.n_f + 127) / 128;
        PQ_CUDA(ctx, go(launch(k_agg_fscan<true>, fgrid(b.n_f, true), 256, s, chained, b)));
        PQ_CUDA(ctx, go(launch(k_agg_fixup, grid(nt, 256), 256, s, chained, b, nt)));
      } else {
        PQ_CUDA(ctx, go(launch(k_agg_fscan<false>, fgrid(b.n_f, false), 256, s, chained, b)));
      }
    }
    if (m_bits)
      PQ_CUDA(ctx, go(launch(k_agg_select, grid((i64)(m_bits + 31) / 32, 256), 256, s, chained, a)));
  }
  ctx->launches += launches;
  // Top-k of the candidates (ticket zeroed with the counters), then the record.
  PQ_CUDA(ctx, topk_launch(ctx, (const int64_t*)a.cand_k, (const int64_t*)a.cand_s, (int64_t)cap,
                           (const int64_t*)a.ctr, d.k, (int64_t*)ok, (int64_t*)os, (int64_t*)nout,
                           (unsigned*)(z + 128), lists, chained, s));
  PQ_CUDA(ctx, launch(k_agg_result, 1, 64, s, true, (const u64*)a.ctr, (const i64*)ok,
                      (const i64*)os, (const i64*)nout, d.k, dres));
  ctx->launches += 1;
  ctx->plans++;
  return read_back(ctx, result, dres, 1, s);
}

}  // namespace pqh
