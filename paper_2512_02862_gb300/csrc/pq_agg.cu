// pq_agg.cu -- the aggregate-first plan (PQ_PLAN_AGG_FIRST): a large
// materialised group-by filtered on its aggregate (the shape of the paper's
// Q18 remark, Sec. 6.3), on resident tables with dense keys.
//
//   D' bitmap  <- D rows with seg op_d c_d                  (k_agg_dbits)
//   M' bitmap  <- M rows with date op_m c_m, dref in D'      (k_agg_mbits)
//   G          <- F rows with date2 op_f c_f: sums[slot(mkey)] +=
//                 price*(100-disc), a flag per group     (k_agg_fscan_t,
//                                                         k_agg_fscan,
//                                                         k_agg_fixup)
//   candidates <- keys of M' whose group exists and has sum > having
//                                                            (k_agg_select)
//   result     <- top-k of the candidates (the top-k operator's kernel,
//                 which also writes the result record)
//
// A group's slot is its key's rank among the F table's distinct keys (a
// presence bitmap of the F key column with a rank directory, measured once
// per table), so the sums and flags are dense; the key range must still be
// at most a few times the F row count (the presence bitmap spans it).
// Consecutive rows of the same group are added up inside the warp first.
// When F's keys come in a few non-decreasing segments (measured once per
// key column), each segment is scanned by its own launch and every group's
// total is stored once (k_agg_fixup finishes the runs that tile or unit
// edges cut); a gapless segment (its distinct keys consecutive among the
// table's) is streamed through shared memory by k_agg_fscan_t, with slots
// counted from one rank lookup per unit.  Otherwise each run's total is one
// reduction into a zeroed array.  int64 overflow: a group sum can only
// leave int64 if the magnitudes of all summed revenues reach 2^62, which
// the plan tracks (one atomic per warp) unless the price column's range
// bounds them, and reports as PQ_ERR_OVERFLOW; a single revenue is formed
// exactly.
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
  // Presence of the F table's keys with its rank directory: a group's slot
  // is its key's rank among the table's distinct keys (fslot).
  const u32* pbm;
  const u32* ptdir;
  const unsigned short* pwdir;
  int fill;            // every slot is written once by this plan (no zeroing)
  int gapless;         // k_agg_fscan_t: a gapless segment, edge records hold slots
  i64 unit;            // k_agg_fscan_t: rows per warp (a multiple of 128)
  i64 spin;            // polls of a stage's mbarrier before PQ_ERR_TIMEOUT
  i64* sums;           // one per slot
  unsigned char* hit;  // one flag byte per slot: the group has a passing row
  int vec;             // F columns 16-byte aligned (mkey, price, date2) and disc 4-byte;
                       // 2: mkey and price 32-byte aligned as well
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

// Slot of the F key with index idx in the F range (the key occurs in F): its
// rank among the F table's distinct keys.
__device__ __forceinline__ u64 fslot(const AggPlan& a, u64 idx) {
  const u64 wi = idx >> 5;
  return (u64)__ldg(a.ptdir + (idx >> 15)) + __ldg(a.pwdir + wi) +
         __popc(__ldg(a.pbm + wi) & ((1u << (idx & 31)) - 1u));
}

// Sorted F: a group's total within one non-decreasing segment of F, stored
// by its only writer (the segments run one after another).  cnt == 0: the
// key's rows all fail the filter; with `fill` its flag is written as 0 (the
// plan writes every slot, so nothing was zeroed).
__device__ __forceinline__ void store_slot(const AggPlan& a, u64 sl, u64 sum, u32 cnt) {
  if (!cnt) {
    if (a.fill) a.hit[sl] = 0;
    return;
  }
  if (a.accum && a.hit[sl]) {
    a.sums[sl] = (i64)((u64)a.sums[sl] + sum);
  } else {
    a.sums[sl] = (i64)sum;
    a.hit[sl] = 1;
  }
}

__device__ __forceinline__ void store_group(const AggPlan& a, u64 idx, u64 sum, u32 cnt) {
  if (cnt || a.fill) store_slot(a, fslot(a, idx), sum, cnt);
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
        if (!pcut && !lcut) store_group(a, idx, acc, cnt);
      } else if (cnt) {
        const u64 sl = fslot(a, idx);
        atomicAdd(reinterpret_cast<unsigned long long*>(a.sums + sl), (unsigned long long)acc);
        a.hit[sl] = 1;
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

// Gapless-segment scan: each warp owns one contiguous unit of rows (a
// multiple of kStep) and streams it through a ring of kAS stages of kStep
// rows in shared memory, filled by bulk copies (lane 0 issues them, an
// mbarrier per stage counts their bytes), so that the copies of the next
// stage are in flight while a step is reduced.  A lane takes kRPL
// consecutive rows of a step, so that the warp-wide work of a step (the
// scan over lanes, the ballots, the carry) is shared by 8 rows per lane.
constexpr int kRPL = 6;                   // rows per lane and step (even)
constexpr int kStep = 32 * kRPL;          // rows per step (and stage)
constexpr int kAS = 2;                    // stages per warp
constexpr int kStageBytes = kStep * 21;   // mkey 8 B, price 8 B, date2 4 B, disc 1 B per row
constexpr int kOffP = kStep * 8, kOffD = kStep * 16, kOffC = kStep * 20;
constexpr int kAggWarps = 4;              // warps per block (small blocks: 5 fit an SM)
constexpr int kAggRuns = kStep + 8;       // a step's stored runs: at most kStep + the carried one
static_assert(kAggRuns * 9 <= kStageBytes, "a step's runs are staged in its own stage");
constexpr size_t kAggSmem = (size_t)kAggWarps * kAS * (8 + kStageBytes);

// Sorted F, a gapless segment (its distinct keys hold consecutive slots).
// A step's runs are summed by a segmented scan over lanes; a run's slot is
// the slot of the unit's first key (one rank lookup per unit) plus the key
// changes before it, counted with four ballots.  The step's last run is
// carried into the next step in registers, so only the units' edges cut
// runs (edge records per unit, finished by k_agg_fixup with slots in place
// of keys).  BOUNDED: the price column's range bounds every revenue by 2^39
// and all of them together by 2^62, so no magnitude is tracked.  A stage
// whose copies do not complete within the spin limit latches
// PQ_ERR_TIMEOUT; the warp then waits (bounded) for its copies in flight
// and stops.
template <bool BOUNDED>
__global__ void __launch_bounds__(kAggWarps * 32, 6) k_agg_fscan_t(AggPlan a) {
  extern __shared__ __align__(128) unsigned char smem[];
  chain_begin();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64* bar = reinterpret_cast<u64*>(smem) + warp * kAS;
  unsigned char* ring = smem + kAggWarps * kAS * 8 + (size_t)warp * kAS * kStageBytes;
  const u32 fb = (u32)a.f_base, lt = lanemask_lt();
  const i64 u = (i64)blockIdx.x * kAggWarps + warp, u0 = u * a.unit;
  u64 mag = 0, rows = 0;
  bool ovf = false;
  if (u0 < a.n_f) {
    const i64 lim = min(a.unit, a.n_f - u0);
    const int steps = (int)((lim + kStep - 1) / kStep);
    if (lane == 0) {
      for (int s = 0; s < kAS; ++s) mbar_init(&bar[s], 1);
      fence_mbar_init();
    }
    __syncwarp();
    // Lane 0: the copies of step s into stage s % kAS (the whole 16-row
    // groups; a segment's last < 16 rows are read from global memory).
    auto issue = [&](int s) {
      if (lane != 0 || s >= steps) return;
      const i64 r = u0 + (i64)s * kStep;
      const u32 n = (u32)min((i64)kStep, a.n_f - r) & ~15u;
      unsigned char* st = ring + (s % kAS) * kStageBytes;
      u64* b = &bar[s % kAS];
      mbar_expect_tx(b, n * 21);
      if (n) {
        bulk_g2s(st, a.f_mkey + r, n * 8, b);
        bulk_g2s(st + kOffP, a.f_price + r, n * 8, b);
        bulk_g2s(st + kOffD, a.f_date + r, n * 4, b);
        bulk_g2s(st + kOffC, a.f_disc + r, n, b);
      }
    };
    for (int s = 0; s < kAS; ++s) issue(s);
    // Lane 0: the key of the row before the unit; lane 31: of the row after.
    i64 ek = 0;
    if (lane == 0 && u0 > 0) ek = __ldg(a.f_mkey + u0 - 1);
    if (lane == 31 && u0 + lim < a.n_f) ek = __ldg(a.f_mkey + u0 + lim);
    u32 cur_key = 0, cur_slot = 0, carry_c = 0, ubase = 0;
    u64 carry_s = 0;
    bool first_open = false, whole = true, cin = false, failed = false;
    i64 k_last = 0;  // lane 31: the unit's last key
    for (int s = 0; s < steps; ++s) {
      unsigned char* st = ring + (s % kAS) * kStageBytes;
      // The step's run totals, gathered in its own stage once its rows are
      // in registers, and stored as one contiguous range of slots (whole
      // sectors, not 8-byte pieces), unless the segment adds to groups of
      // earlier ones (accum: stored one by one).
      i64* ost = reinterpret_cast<i64*>(st);
      unsigned char* ohit = st + kAggRuns * 8;
      const bool ok = mbar_wait(&bar[s % kAS], (u32)((s / kAS) & 1), a.spin);
      if (!__all_sync(kFull, ok)) {
        if (lane == 0) latch(a.st, PQ_ERR_TIMEOUT, u0 + (i64)s * kStep);
        for (int t = s; t < steps && t < s + kAS; ++t)
          mbar_wait(&bar[t % kAS], (u32)((t / kAS) & 1), a.spin);
        failed = true;
        break;
      }
      const i64 s0 = u0 + (i64)s * kStep;
      const int nr = (int)min((i64)kStep, a.n_f - s0);
      i64 k[kRPL], p[kRPL];
      int dt[kRPL];
      u64 dc = 0;
      if (nr == kStep) {  // the lane's kRPL rows: 16-byte reads of keys and prices
        const longlong2* sk = reinterpret_cast<const longlong2*>(st) + (kRPL / 2) * lane;
        const longlong2* sp = reinterpret_cast<const longlong2*>(st + kOffP) + (kRPL / 2) * lane;
        const int2* sd = reinterpret_cast<const int2*>(st + kOffD) + (kRPL / 2) * lane;
        const unsigned short* sc = reinterpret_cast<const unsigned short*>(st + kOffC) + (kRPL / 2) * lane;
#pragma unroll
        for (int h = 0; h < kRPL / 2; ++h) {
          const longlong2 x = sk[h], y = sp[h];
          const int2 d = sd[h];
          k[2 * h] = x.x, k[2 * h + 1] = x.y, p[2 * h] = y.x, p[2 * h + 1] = y.y;
          dt[2 * h] = d.x, dt[2 * h + 1] = d.y;
          dc |= (u64)sc[h] << (16 * h);
        }
      } else {  // the segment's last step: rows past its end repeat the last row
        const int nc = nr & ~15;
#pragma unroll
        for (int j = 0; j < kRPL; ++j) {
          const int q = min(kRPL * lane + j, nr - 1);
          if (q < nc) {
            k[j] = reinterpret_cast<const i64*>(st)[q];
            p[j] = reinterpret_cast<const i64*>(st + kOffP)[q];
            dt[j] = reinterpret_cast<const int*>(st + kOffD)[q];
            dc |= (u64)st[kOffC + q] << (8 * j);
          } else {
            k[j] = a.f_mkey[s0 + q];
            p[j] = a.f_price[s0 + q];
            dt[j] = a.f_date[s0 + q];
            dc |= (u64)(unsigned char)a.f_disc[s0 + q] << (8 * j);
          }
        }
      }
      __syncwarp();  // the stage is read: it holds the run totals from here on
      u32 ix[kRPL];
#pragma unroll
      for (int j = 0; j < kRPL; ++j) ix[j] = (u32)k[j] - fb;
      if (s == 0) {  // the unit's first key: its slot, and whether its run began earlier
        if (lane == 0) ubase = (u32)fslot(a, ix[0]);
        cin = __shfl_sync(kFull, lane == 0 && u0 > 0 && ek == k[0], 0);
        first_open = cin;
      }
      if (lane == 31) k_last = k[kRPL - 1];
      const int nv = nr - kRPL * lane;  // the lane's rows inside the segment
      u32 pm = 0;
#pragma unroll
      for (int j = 0; j < kRPL; ++j) pm |= (j < nv && pass32(a.pf, dt[j]) ? 1u : 0u) << j;
      u64 v[kRPL];
      if (BOUNDED) {
#pragma unroll
        for (int j = 0; j < kRPL; ++j) {
          const i64 r = (i64)(int)p[j] * (i64)(100 - (int)(signed char)(dc >> (8 * j)));
          v[j] = (pm >> j) & 1u ? (u64)r : 0;
        }
      } else {
#pragma unroll
        for (int j = 0; j < kRPL; ++j) {
          const bool in = (pm >> j) & 1u;
          const __int128 rev = (__int128)p[j] * (100 - (int)(signed char)(dc >> (8 * j)));
          const i64 r64 = (i64)rev;
          ovf = ovf || (in && rev != (__int128)r64);
          v[j] = in ? (u64)r64 : 0;
          const u64 m = r64 < 0 ? (u64)0 - (u64)r64 : (u64)r64;
          if (in) mag = mag >= kMag || m >= kMag ? kMag : min(kMag, mag + m);
        }
      }
      rows += __popc(pm);
      // Key changes (bit j: row j holds another key than the row before it;
      // lane 0's row 0 compares with the previous step's last key, and
      // counts as a change at the unit's first step).
      const u32 prev = __shfl_up_sync(kFull, ix[kRPL - 1], 1);
      u32 hb = 0;
#pragma unroll
      for (int j = 1; j < kRPL; ++j) hb |= (ix[j] != ix[j - 1] ? 1u : 0u) << j;
      hb |= (lane ? ix[0] != prev : (s == 0 || ix[0] != cur_key)) ? 1u : 0u;
      const bool h0 = __shfl_sync(kFull, hb & 1u, 0);
      // The carried run: it ends before this step (committed with this
      // step's runs) or goes on into row 0 (its sum and pass flag join it).
      u32 pmc = pm;
      bool cc = false;
      if (s > 0) {
        if (h0) {
          if (lane == 0) {
            if (first_open)
              a.edge[u].psum = carry_s, a.edge[u].pcnt = carry_c;
            else if (a.accum)
              store_slot(a, cur_slot, carry_s, carry_c);
            else
              ost[0] = (i64)carry_s, ohit[0] = carry_c ? 1 : 0;
          }
          cc = !first_open && !a.accum;
          first_open = false, whole = false;
        } else if (lane == 0) {
          v[0] += carry_s, pmc |= carry_c ? 1u : 0u;
        }
      }
      // Segmented scan over lanes (lane 0 always starts one): the lane's
      // last run summed back to the lane where it starts.
      const u32 sh = hb | (lane == 0 ? 1u : 0u);
      u64 ls = 0;
      u32 fl = 0;
#pragma unroll
      for (int j = 0; j < kRPL; ++j) {
        if ((sh >> j) & 1u) ls = 0, fl = 1;
        ls += v[j];
        fl |= ((pmc >> j) & 1u) << 1;
      }
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
      const u64 in_s = __shfl_up_sync(kFull, ls, 1);
      const u32 in_p = __shfl_up_sync(kFull, fl, 1) >> 1;
      const bool next_head = __shfl_down_sync(kFull, sh & 1u, 1);
      // Slots: key changes after row 0 of the step, before each lane (four
      // ballots of the lanes' counts, 0..8) and in all.
      const u32 hx = lane ? hb : hb & ~1u;
      const u32 hc = __popc(hx);
      const u32 b0 = __ballot_sync(kFull, hc & 1u), b1 = __ballot_sync(kFull, hc & 2u),
                b2 = __ballot_sync(kFull, hc & 4u), b3 = __ballot_sync(kFull, hc & 8u);
      const u32 R = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
      const u32 sbase = s == 0 ? __shfl_sync(kFull, ubase, 0) : cur_slot + (h0 ? 1u : 0u);
      u32 ri = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) + 8 * __popc(b3 & lt);
      // Slots stored by this step: [lo, sbase + R): the carried run first
      // (cc), without the unit's first run when it began in an earlier unit.
      const u32 lo = cc ? sbase - 1 : sbase + (first_open && R ? 1u : 0u);
      u64 acc = (sh & 1u) ? 0 : in_s;
      u32 cnt = (sh & 1u) ? 0 : in_p;
#pragma unroll
      for (int j = 0; j < kRPL; ++j) {
        if (j > 0 && ((hb >> j) & 1u)) acc = 0, cnt = 0;
        ri += (hx >> j) & 1u;
        acc += v[j];
        cnt |= (pmc >> j) & 1u;
        const bool end = j < kRPL - 1 ? (hb >> (j + 1)) & 1u : (lane < 31 && next_head);
        if (!end) continue;
        if (first_open && ri == 0) {  // the unit's first run, begun in an earlier unit
          a.edge[u].psum = acc, a.edge[u].pcnt = cnt;
        } else if (a.accum) {
          store_slot(a, sbase + ri, acc, cnt);
        } else {
          const u32 o = sbase + ri - lo;
          ost[o] = (i64)acc, ohit[o] = cnt ? 1 : 0;
        }
      }
      if (!a.accum) {  // the range, stored by the warp
        __syncwarp();
        const int n = (int)(sbase + R - lo);
        for (int i = lane; i < n; i += 32) a.sums[lo + i] = ost[i], a.hit[lo + i] = ohit[i];
      }
      // Lane 0 refills the stage with step s + kAS.
      __syncwarp();
      if (lane == 0 && s + kAS < steps) fence_proxy_async_smem();
      issue(s + kAS);
      // The step's last run is carried on.
      carry_s = __shfl_sync(kFull, acc, 31);
      carry_c = __shfl_sync(kFull, cnt, 31);
      cur_slot = sbase + R;
      cur_key = __shfl_sync(kFull, ix[kRPL - 1], 31);
      if (R) first_open = false, whole = false;
    }
    // The unit's end: its last run is cut if the next row holds its key.
    if (!failed) {
      const bool cout = __shfl_sync(kFull, lane == 31 && u0 + lim < a.n_f && ek == k_last, 31);
      if (lane == 0) {
        if (cout) a.edge[u].lsum = carry_s, a.edge[u].lcnt = carry_c, a.edge[u].lkey = cur_slot;
        if (first_open)
          a.edge[u].psum = carry_s, a.edge[u].pcnt = carry_c;
        else if (!cout)
          store_slot(a, cur_slot, carry_s, carry_c);
        a.eflag[u] = (unsigned char)((cin ? kCin : 0) | (cout ? kCout : 0) | (whole ? kWhole : 0));
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    if (!BOUNDED) {
      const u64 x = __shfl_xor_sync(kFull, mag, o);
      mag = mag >= kMag || x >= kMag ? kMag : min(kMag, mag + x);
    }
    rows += __shfl_xor_sync(kFull, rows, o);
  }
  ovf = __any_sync(kFull, ovf);
  if (lane == 0) {
    if (rows) atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr + 2), rows);
    if (!BOUNDED && mag) {
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
    if (a.gapless)  // the edge record holds the run's slot
      store_slot(a, (u64)key, sum, (u32)cnt);
    else
      store_group(a, ukey(key) - a.f_base, sum, (u32)cnt);
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
        // The presence word and the rank directory are read together, then
        // the slot's flag and sum together (a sum without its flag is unused).
        if (idx < a.f_bits) {
          const u64 wi = idx >> 5;
          const u32 pw = __ldg(a.pbm + wi);
          const u64 sl = (u64)__ldg(a.ptdir + (idx >> 15)) + __ldg(a.pwdir + wi) +
                         __popc(pw & ((1u << (idx & 31)) - 1u));
          if ((pw >> (idx & 31)) & 1u) {
            const unsigned char h = a.hit[sl];
            sum = a.sums[sl];
            key = (i64)(uk ^ (1ULL << 63));
            take = h && sum > a.having;
          }
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

// Presence of an F key column's keys: one bit per key of its range.
__global__ void k_pres_bits(const i64* key, i64 n, u64 umin, u32* bm) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x)
    bit_set(bm, ukey(__ldg(key + i)) - umin);
}

// Rank directory of a presence bitmap (the dense dictionary's layout): one
// warp per tile of kRankTile 512-bit blocks writes each word's set bits
// before it within the tile and the tile's total (turned into tile prefixes
// afterwards).
__global__ void k_pres_rank(const uint4* bm, u64 blocks, u32* tdir, unsigned short* wdir) {
  const int lane = threadIdx.x & 31;
  const u64 tiles = (blocks + kRankTile - 1) / kRankTile;
  for (u64 t = (blockIdx.x * (u64)blockDim.x + threadIdx.x) >> 5; t < tiles;
       t += ((u64)gridDim.x * blockDim.x) >> 5) {
    const u64 b0 = t * kRankTile, b1 = min(blocks, b0 + kRankTile);
    u32 run = 0;
    for (u64 j0 = b0; j0 < b1; j0 += 32) {
      const u64 j = j0 + lane;
      u32 c[16], p = 0;
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        const uint4 v = j < b1 ? bm[j * 4 + qd] : make_uint4(0, 0, 0, 0);
        c[qd * 4] = __popc(v.x), c[qd * 4 + 1] = __popc(v.y);
        c[qd * 4 + 2] = __popc(v.z), c[qd * 4 + 3] = __popc(v.w);
        p += c[qd * 4] + c[qd * 4 + 1] + c[qd * 4 + 2] + c[qd * 4 + 3];
      }
      u32 incl = p;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      if (j < b1) {
        u32 pre = run + incl - p;
#pragma unroll
        for (int x = 0; x < 16; ++x) wdir[j * 16 + x] = (unsigned short)pre, pre += c[x];
      }
      run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) tdir[t] = run;
  }
}

// Segment starts of a key-ordered column (row 0, then its descents).
struct SegStarts {
  i64 at[kMaxDescents + 1];
  int n;
};

__device__ __forceinline__ int seg_of(const SegStarts& sb, i64 i) {
  int j = 0;
#pragma unroll
  for (int x = 1; x <= kMaxDescents; ++x) j += x < sb.n && i >= sb.at[x];
  return j;
}

// Rows that start a run of equal keys (row 0 and each row whose key differs
// from the row before), counted per segment: the segment's distinct keys.
__global__ void k_pres_heads(const i64* key, i64 n, SegStarts sb, unsigned long long* heads) {
  __shared__ unsigned long long sc[kMaxDescents + 1];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x <= kMaxDescents) sc[threadIdx.x] = 0;
  __syncthreads();
  for (i64 i0 = (i64)blockIdx.x * blockDim.x; i0 < n; i0 += (i64)gridDim.x * blockDim.x) {
    const i64 i = i0 + threadIdx.x;
    bool h = false;
    int j = 0;
    if (i < n) {
      h = i == 0 || key[i] != key[i - 1];
      j = seg_of(sb, i);
    }
    const int jl = __shfl_sync(kFull, j, 0);
    if (__all_sync(kFull, j == jl)) {
      const u32 b = __ballot_sync(kFull, h);
      if (lane == 0 && b) atomicAdd(&sc[jl], (unsigned long long)__popc(b));
    } else if (h) {
      atomicAdd(&sc[j], 1ULL);
    }
  }
  __syncthreads();
  if (threadIdx.x < sb.n && sc[threadIdx.x]) atomicAdd(heads + threadIdx.x, sc[threadIdx.x]);
}

// Segment j is gapless when the rank of its last key minus that of its first
// key, plus one, equals its count of distinct keys.  One warp; bit j of *mask.
__global__ void k_pres_gapless(const i64* key, i64 n, u64 umin, SegStarts sb, const u32* bm,
                               const u32* tdir, const unsigned short* wdir,
                               const unsigned long long* heads, u32* mask) {
  const int j = threadIdx.x;
  bool g = false;
  if (j < sb.n) {
    auto rank = [&](i64 row) -> u64 {
      const u64 idx = ukey(key[row]) - umin, wi = idx >> 5;
      return (u64)tdir[idx >> 15] + wdir[wi] + __popc(bm[wi] & ((1u << (idx & 31)) - 1u));
    };
    const i64 r1 = (j + 1 < sb.n ? sb.at[j + 1] : n) - 1;
    g = rank(r1) - rank(sb.at[j]) + 1 == heads[j];
  }
  const u32 b = __ballot_sync(kFull, g);
  if (j == 0) *mask = b;
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

// The same with `smem` bytes of dynamic shared memory.
template <typename... P, typename... A>
cudaError_t launch_smem(void (*k)(P...), int grid, int block, size_t smem, cudaStream_t s,
                        bool chained, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Blocks of 256 threads of kernel k resident per SM (at least 1), with
// `smem` bytes of dynamic shared memory (allowed for k first).
template <typename K>
int resident_blocks(K k, size_t smem = 0, int threads = 256) {
  int n = 0;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    cudaGetLastError();
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return std::max(n, 1);
}

}  // namespace

namespace {

// The presence bitmap and rank directory of the F key column c of table t
// (its range known), measured once and kept in an arena block the table
// owns: bits on the utility stream, word prefixes, then the tile prefixes
// scanned on the host (a few thousand tiles).  No lock is held across the
// waits; two threads measuring the same column publish the first result
// and the other releases its block.
static bool ensure_key_presence(pq_ctx* ctx, const pq_table* t, int c, cudaStream_t s) {
  const Column& col = t->cols[c];
  if (col.pres.known()) return true;
  if (!col.range.known() || !col.dev || t->nrows <= 0 || col.type != PQ_INT64) return false;
  const u64 bits = col.range.umax - col.range.umin + 1;
  if (bits > kMaxBmBits) return false;
  const DenseLayout L = dense_layout(0, bits);
  const u64 blocks = (bits + 511) / 512, tiles = (blocks + kRankTile - 1) / kRankTile;
  // After the bitmap and its directory: the segments' distinct-key counts
  // and the gapless mask (key-ordered columns).
  char* blk = (char*)ctx->arena.alloc(L.hit + 256);
  SegStarts sb{};
  sb.n = col.range.ndesc >= 0 ? col.range.ndesc + 1 : 0;
  for (int j = 1; j < sb.n; ++j) sb.at[j] = col.range.desc[j - 1];
  unsigned long long* heads = (unsigned long long*)(blk + L.hit);
  u32* gmask = (u32*)(blk + L.hit + 128);
  u32 gapless = 0;
  if (!blk) return false;
  cudaStream_t u = ctx->util_stream;
  std::vector<u32> td(tiles + 1);
  cudaEvent_t after = nullptr;
  bool ok = cudaEventCreateWithFlags(&after, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(after, s ? s : cudaStreamLegacy) == cudaSuccess &&
            cudaStreamWaitEvent(u, after, 0) == cudaSuccess &&
            cudaMemsetAsync(blk, 0, L.tdir, u) == cudaSuccess &&
            cudaMemsetAsync(blk + L.hit, 0, 256, u) == cudaSuccess;
  u32* tdir = (u32*)(blk + L.tdir);
  if (ok) {
    const int grid = (int)std::min<i64>((t->nrows + 255) / 256, (i64)ctx->num_sms * 8);
    k_pres_bits<<<grid, 256, 0, u>>>((const i64*)col.dev, t->nrows, col.range.umin, (u32*)blk);
    const int rgrid = (int)std::min<u64>((tiles * 32 + 255) / 256, (u64)ctx->num_sms * 8);
    k_pres_rank<<<rgrid, 256, 0, u>>>((const uint4*)blk, blocks, tdir,
                                      (unsigned short*)(blk + L.wdir));
    if (sb.n) {
      const int hgrid = (int)std::min<i64>((t->nrows + 255) / 256, (i64)ctx->num_sms * 8);
      k_pres_heads<<<hgrid, 256, 0, u>>>((const i64*)col.dev, t->nrows, sb, heads);
      ctx->launches += 1;
    }
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(td.data(), tdir, tiles * 4, cudaMemcpyDeviceToHost, u) == cudaSuccess &&
         cudaStreamSynchronize(u) == cudaSuccess;
    ctx->launches += 2;
  }
  u64 distinct = 0;
  if (ok) {  // tile totals -> prefixes, the total last
    for (u64 i = 0; i < tiles; ++i) {
      const u32 v = td[i];
      td[i] = (u32)distinct;
      distinct += v;
    }
    td[tiles] = (u32)distinct;
    ok = cudaMemcpyAsync(tdir, td.data(), (tiles + 1) * 4, cudaMemcpyHostToDevice, u) ==
         cudaSuccess;
    if (ok && sb.n) {
      k_pres_gapless<<<1, 32, 0, u>>>((const i64*)col.dev, t->nrows, col.range.umin, sb,
                                      (const u32*)blk, tdir, (const unsigned short*)(blk + L.wdir),
                                      heads, gmask);
      ok = cudaGetLastError() == cudaSuccess &&
           cudaMemcpyAsync(&gapless, gmask, 4, cudaMemcpyDeviceToHost, u) == cudaSuccess;
      ctx->launches += 1;
    }
    ok = ok && cudaStreamSynchronize(u) == cudaSuccess;
  }
  if (after) cudaEventDestroy(after);
  if (!ok) {
    cudaGetLastError();
    ctx->arena.release(blk, u);
    return false;
  }
  std::lock_guard<std::mutex> g(ctx->range_mu);
  if (col.pres.known()) {
    ctx->arena.release(blk, u);
    return true;
  }
  KeyPresence& kp = col.pres;
  kp.block = blk;
  kp.bits = bits;
  kp.distinct = distinct;
  kp.gapless = gapless;
  kp.ready.store(true, std::memory_order_release);
  return true;
}

// Sizes of an aggregate-first plan's workspace, from the tables' key ranges
// and key order (measured once per key column).
struct AggShape {
  u64 d_bits = 0, m_bits = 0, f_bits = 0;
  u64 f_slots = 0;      // distinct keys of the F table (the group slots)
  size_t cap = 1;       // candidates: at most one per key of M' inside the F range
  bool sorted = false;  // F scanned as its non-decreasing segments
  bool fill = false;    // one segment over the whole F table: every slot written once
  std::vector<i64> seg;  // segment starts within the plan's F rows, then n_f
  std::vector<char> gap;  // per segment: gapless (scanned by k_agg_fscan_u)
  u64 rev_max = 0;        // bound of one |revenue|, 0 when unknown
  i64 ntiles = 0;        // tiles of the longest segment
  size_t head = 0, hit_bytes = 0, sums_bytes = 0, zero = 0, edge_bytes = 0, cand_bytes = 0;
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
  // Bound of one revenue |price * (100 - disc)|: the price column's measured
  // range times 228, the largest |100 - disc| of an int8.
  if (T[2]->nrows > 0) {
    const KeyRange& pr = T[2]->cols[1].range;
    if (pr.known() || (cap == cudaStreamCaptureStatusNone && ensure_range(ctx, T[2], 1, s))) {
      const i64 lo = (i64)(pr.umin ^ (1ULL << 63)), hi = (i64)(pr.umax ^ (1ULL << 63));
      const unsigned __int128 amax =
          std::max(lo < 0 ? (unsigned __int128)(-(__int128)lo) : (unsigned __int128)lo,
                   hi < 0 ? (unsigned __int128)(-(__int128)hi) : (unsigned __int128)hi);
      if (amax * 228 < ((unsigned __int128)1 << 63)) g.rev_max = (u64)(amax * 228);
    }
  }
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
  if (g.f_bits) {  // group slots: ranks among the F table's distinct keys
    if (!T[2]->cols[0].pres.known()) {
      if (cap != cudaStreamCaptureStatusNone)
        return fail(ctx, PQ_ERR_INVALID_ARG,
                    "aggregate-first plan: run it once before capturing a stream (key presence)");
      if (!ensure_key_presence(ctx, T[2], 0, s))
        return fail(ctx, PQ_ERR_BUDGET, "aggregate-first plan: F key presence bitmap");
    }
    g.f_slots = T[2]->cols[0].pres.distinct;
  }
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
  // A plan segment is a clipped segment of the table (the first is the one
  // holding row f_row0): gapless if the table's segment is, and the slots
  // and key offsets fit in 32 bits.
  g.gap.assign(g.seg.size() - 1, 0);
  if (g.sorted && g.f_bits && g.f_bits <= (1ULL << 32)) {
    int j0 = 0;
    for (int j = 0; j < fk.ndesc; ++j) j0 += fk.desc[j] <= r.f_row0;
    const u32 gm = T[2]->cols[0].pres.gapless;
    for (size_t j = 0; j < g.gap.size(); ++j) g.gap[j] = (gm >> (j0 + j)) & 1u;
  }
  // Zeroed: counters, D' and M' bitmaps; the hit flags unless every slot is
  // written by the scan (one key-ordered segment over the whole F table);
  // the sums unless sorted (stores, not reductions).
  g.fill = g.sorted && g.seg.size() == 2 && r.f_row0 == 0 && r.n_f == T[2]->nrows;
  g.head = 256 + al256(words_bytes(g.d_bits)) + al256(words_bytes(g.m_bits));
  g.hit_bytes = al256((size_t)std::max<u64>(g.f_slots, 1));
  g.sums_bytes = al256(8 * (size_t)std::max<u64>(g.f_slots, 1));
  g.zero = g.head + (g.fill ? 0 : g.hit_bytes + (g.sorted ? 0 : g.sums_bytes));
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
  *bytes = g.head + g.hit_bytes + g.sums_bytes + g.edge_bytes + al256(g.cand_bytes) + 2 * 256;
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
  const size_t hit_bytes = g.hit_bytes;
  const i64 ntiles = g.ntiles;
  Scratch scr(ctx, s);
  char* z = (char*)scr.get(head + hit_bytes + sums_bytes + edge_bytes);
  char* c = (char*)scr.get(g.cand_bytes);
  if (!z || !c)
    return fail(ctx, PQ_ERR_BUDGET, "aggregate-first plan: %zu bytes",
                head + hit_bytes + sums_bytes + edge_bytes + g.cand_bytes);
  AggPlan a{};
  a.ctr = (u64*)z;
  a.dbm = (u32*)(z + 256);
  a.mbm = (u32*)((char*)a.dbm + al256(words_bytes(d_bits)));
  a.hit = (unsigned char*)(z + head);
  a.sums = (i64*)(z + head + hit_bytes);
  a.fill = g.fill ? 1 : 0;
  if (f_bits) {
    const KeyPresence& kp = T[2]->cols[0].pres;
    const DenseLayout PL = dense_layout(0, kp.bits);
    a.pbm = (const u32*)kp.block;
    a.ptdir = (const u32*)((const char*)kp.block + PL.tdir);
    a.pwdir = (const unsigned short*)((const char*)kp.block + PL.wdir);
  }
  if (sorted) {
    a.edge = (TileEdge*)(z + head + hit_bytes + sums_bytes);
    a.eflag = (unsigned char*)a.edge + al256(sizeof(TileEdge) * ntiles);
  }
  a.cand_k = (i64*)c;
  a.cand_s = a.cand_k + cap;
  pq_result* dres = (pq_result*)(c + al256(16 * cap) + al256(16 * PQ_MAX_K) + 256);
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
  static const int occ_t[2] = {resident_blocks(k_agg_fscan_t<false>, kAggSmem, kAggWarps * 32),
                               resident_blocks(k_agg_fscan_t<true>, kAggSmem, kAggWarps * 32)};
  // Bounded revenues: |price| < 2^31 and n_f * max|revenue| < 2^62, from the
  // price column's measured range (max |price| * 228).
  const bool bounded = g.rev_max > 0 && g.rev_max <= 228ULL * 0x7fffffffULL &&
                       (unsigned __int128)g.rev_max * (u64)std::max<i64>(r.n_f, 1) <
                           ((unsigned __int128)1 << 62);
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
      if (b.vec && (uintptr_t)b.f_mkey % 32 == 0 && (uintptr_t)b.f_price % 32 == 0) b.vec = 2;
      b.accum = j > 0;
      if (b.n_f <= 0) continue;
      // Bulk copies need 16-byte aligned segment starts in every column.
      const bool tma = (uintptr_t)b.f_mkey % 16 == 0 && (uintptr_t)b.f_price % 16 == 0 &&
                       (uintptr_t)b.f_date % 16 == 0 && (uintptr_t)b.f_disc % 16 == 0;
      if (sorted && g.gap[j] && tma) {
        // One unit per warp of one resident wave, in whole steps.
        const i64 warps = (i64)sms * occ_t[bounded] * kAggWarps;
        b.unit = std::max<i64>(1, (b.n_f + warps * kStep - 1) / (warps * kStep)) * kStep;
        const i64 nu = (b.n_f + b.unit - 1) / b.unit;
        b.gapless = 1;
        b.spin = ctx->opt.spin_limit;
        const int tg = (int)((nu + kAggWarps - 1) / kAggWarps);
        if (bounded)
          PQ_CUDA(ctx, go(launch_smem(k_agg_fscan_t<true>, tg, kAggWarps * 32, kAggSmem, s, chained,
                                      b)));
        else
          PQ_CUDA(ctx, go(launch_smem(k_agg_fscan_t<false>, tg, kAggWarps * 32, kAggSmem, s,
                                      chained, b)));
        PQ_CUDA(ctx, go(launch(k_agg_fixup, grid(nu, 256), 256, s, chained, b, nu)));
      } else if (sorted) {
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
  // Top-k of the candidates (ticket zeroed with the counters), written into
  // the result record with the plan's counters.
  PQ_CUDA(ctx, topk_launch(ctx, (const int64_t*)a.cand_k, (const int64_t*)a.cand_s, (int64_t)cap,
                           (const int64_t*)a.ctr, d.k, dres->keys, dres->sums, &dres->n,
                           (unsigned*)(z + 128), lists, chained, s, (const uint64_t*)a.ctr, dres));
  ctx->plans++;
  return read_back(ctx, result, dres, 1, s);
}

}  // namespace pqh
