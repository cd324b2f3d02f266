// pq_plan_kernels.cuh -- the kernels of the three-table plan, batched.
//
// One launch of each kernel serves every plan of a batch: persistent blocks
// claim tiles of a flattened work list (atomic tickets, work stealing) and map
// a tile to its plan by binary search in a tile prefix array.  A single plan
// is a batch of one.  Phases (each one kernel):
//   dscan   D rows: seg predicate -> append key to the plan's D list
//   fill    clear the D-set region (slot count from the device count)
//   dbuild  insert the D list into the D-set (open addressing, set semantics)
//   mscan   M rows: date predicate, dref in D-set -> append key to M list
//   fill    clear the M hash-table key region
//   mbuild  insert the M list (one slot per row; duplicates flagged)
//   fprobe  F rows: date2 predicate, probe M table, add price*(100-disc)
//           into the matched slot, record first-hit slots as groups
//   topk    per (plan, chunk of groups) block top-k, last block per plan merges
// The last block of dscan / mscan / fprobe sizes the next phases from the
// device counts (no host synchronisation: deferred synchronisation taken to
// its end, Sec. 3.3).
//
// The scans are warp-centric: a warp claims its own tile (no block barrier on
// the streaming path), reads 4 consecutive rows per lane with 128-bit loads
// software-pipelined two iterations ahead, and reads the wide columns (keys,
// references) only for 4-row groups whose predicate holds.  Passing rows are
// compacted into per-warp shared-memory rings so that every hash probe runs
// with all 32 lanes busy.  Scanned columns are loaded with an L2 evict-first
// policy and hash-table probes with evict-last, so the tables stay in L2
// while the columns stream past.
#pragma once
#include "../../include/pq.h"
#include "pq_dev.cuh"
#include "pq_topk.cuh"

namespace pqk {

constexpr int kTD = 4096;    // D rows per warp tile
constexpr int kTM = 2048;    // M rows per warp tile
constexpr int kTF = 4096;    // F rows per warp tile
constexpr int kTC = 16384;   // slots cleared per block tile
constexpr int kTB = 1024;    // list entries inserted per block tile
constexpr int kTK = 1024;    // groups per top-k block tile
constexpr int kQ = 256;      // entries of a warp's shared-memory ring

struct QCtr {
  u64 dcount, mcount, gcount;
  int dup;
  u32 tk_ticket;
  int status;
  int mlog2;
  u64 pad[2];
};

struct PlanDev {
  const int* d_key;
  const signed char* d_seg;
  i64 n_d;
  const i64* m_key;
  const int* m_dref;
  const int* m_date;
  i64 n_m;
  const i64* f_mkey;
  const i64* f_price;
  const signed char* f_disc;
  const int* f_date;
  i64 n_f;
  Pred pd, pm, pf;
  int k, lf1024;
  int build_dset;   // this plan fills its D-set in this batch
  int vec;          // every column pointer is 16-byte aligned
  i64* dlist;
  int* dset_log2;   // header word of the D-set block
  i64* dset;        // D-set keys
  unsigned short* dset_tag;  // D-set tags (0 = empty)
  i64* mlist;
  unsigned short* ht_tag;    // M table tags (0 = empty)
  i64* ht_keys;
  i64* ht_sums;
  u32* ht_cnt;
  u32* glist;
  i64* tk_k;
  i64* tk_s;
  int* tk_c;
  QCtr* ctr;
  pq_result* out;
};

// Chunk override for streaming plans: the scan phase of table `table`
// (1 = D, 2 = M, 3 = F) of plan 0 reads `n` rows from the column pointers
// `p` (in the table's column order) as `tiles` tiles, instead of the
// plan's resident columns.
struct Ovr {
  const void* p[4];
  i64 n;
  i64 tiles;
  int table;
  int pad;
};

struct Batch {
  PlanDev* q;
  int nq;
  int pad;
  const i64* tD;  // static tile prefixes [nq + 1]
  const i64* tM;
  const i64* tF;
  i64* dyn;       // dynamic prefixes [5][nq + 1]: dclear, dbuild, mclear, mbuild, topk
  u32* work;      // [8] work tickets, [8..16) done tickets
  DevStatus* st;
  i64 spin_limit;
  Ovr ov;
};

enum { kPhDscan = 0, kPhDfill, kPhDbuild, kPhMscan, kPhMfill, kPhMbuild, kPhFprobe, kPhTopk };

// The kernels below are defined in exactly one translation unit (pq_plan.cu),
// which defines PQ_DEFINE_PLAN_KERNELS before including this header.
#ifdef PQ_DEFINE_PLAN_KERNELS

__device__ __forceinline__ int find_q(const i64* pre, int nq, i64 t) {
  int lo = 0, hi = nq;  // invariant pre[lo] <= t < pre[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Claim the next tile of phase `ph` for the whole block.
__device__ __forceinline__ i64 claim(u32* work, int ph) {
  __shared__ i64 s_t;
  __syncthreads();
  if (threadIdx.x == 0) s_t = atomicAdd(&work[ph], 1u);
  __syncthreads();
  return s_t;
}

// Claim the next tile of phase `ph` for one warp (no block barrier).
__device__ __forceinline__ i64 warp_claim(u32* work, int ph) {
  u32 t = 0;
  if ((threadIdx.x & 31) == 0) t = atomicAdd(&work[ph], 1u);
  return (i64)__shfl_sync(kFull, t, 0);
}

// Returns true in the block that finishes last; that block also resets the
// phase's tickets so that the next launch starts from zero.
__device__ __forceinline__ bool finish(u32* work, int ph) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const u32 t = atomicAdd(&work[8 + ph], 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) {
      work[ph] = 0;
      work[8 + ph] = 0;
    }
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Block-wide exclusive scan over nq values produced by `f(q)`; writes
// pre[0..nq] (pre[nq] = total).  Run by one whole block.
template <typename F>
__device__ void block_prefix(i64* pre, int nq, F f) {
  __shared__ i64 s_w[32];
  __shared__ i64 s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int b = 0; b < nq; b += blockDim.x) {
    const int q = b + threadIdx.x;
    const i64 v = q < nq ? f(q) : 0;
    i64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      i64 y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      i64 c = lane < nw ? s_w[lane] : 0, y = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        i64 z = __shfl_up_sync(kFull, y, o);
        if (lane >= o) y += z;
      }
      if (lane < nw) s_w[lane] = y - c;
    }
    __syncthreads();
    const i64 carry = s_carry;
    if (q < nq) pre[q] = carry + s_w[warp] + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + s_w[warp] + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) pre[nq] = s_carry;
  __syncthreads();
}

__device__ __forceinline__ void q_latch(QCtr* c, DevStatus* st, int code, i64 detail) {
  atomicCAS(&c->status, 0, code);
  latch(st, code, detail);
}

// Geometry of a bucketized table of 2^e slots: bucket mask and the shift that
// takes a bucket index from the top of the Fibonacci product.
struct Geo {
  u64 bmask;
  int shiftb;
};
__device__ __forceinline__ Geo geo(int e) {
  Geo g;
  g.bmask = (1ULL << (e - 3)) - 1;
  g.shiftb = 64 - (e - 3);
  return g;
}

// Membership of k in a bucketized key set.
__device__ __forceinline__ bool set_contains(const unsigned short* tags, const i64* keys, Geo g,
                                             i64 k, u64 keep) {
  const BucketTag bt = bucket_tag(k, g.shiftb);
  const unsigned v2 = bt.tag * 0x10001u;
  u64 b = bt.bucket;
  for (u64 p = 0; p <= g.bmask; ++p) {
    const uint4 w = ld_keep_v4u(tags + b * 8, keep);
    Mask8 m = match8(w, v2);
    while (any8(m)) {
      const int j = first8(m);
      if (ld_keep(keys + b * 8 + j, keep) == k) return true;
      drop8(m, j);
    }
    if (any8(match8(w, 0u))) return false;
    b = (b + 1) & g.bmask;
  }
  return false;
}

// Insert k (one slot per insert, so duplicate keys take one slot each):
// claim the first free tag of the first non-full bucket with a 16-bit CAS,
// then write the key.  Returns the slot.
__device__ __forceinline__ u64 tagged_insert(unsigned short* tags, i64* keys, Geo g, i64 k) {
  const BucketTag bt = bucket_tag(k, g.shiftb);
  u64 b = bt.bucket;
  for (u64 p = 0; p <= g.bmask; ++p) {
    uint4 w;
    asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                 : "l"(tags + b * 8));
    Mask8 e = match8(w, 0u);
    while (any8(e)) {
      const int j = first8(e);
      if (atomicCAS(tags + b * 8 + j, (unsigned short)0, (unsigned short)bt.tag) == 0) {
        keys[b * 8 + j] = k;
        return b * 8 + j;
      }
      drop8(e, j);
    }
    b = (b + 1) & g.bmask;
  }
  return ~0ULL;  // unreachable: a table is never filled beyond its load factor
}

// Four consecutive int32 values starting at row e0; `rem` rows remain in the
// column from e0 (rows beyond read as 0).
template <bool VEC>
__device__ __forceinline__ int4 load_i32x4(const int* p, i64 e0, i64 rem, u64 pol) {
  if (VEC && rem >= 4) return ld_stream_v4(p + e0, pol);
  int4 v;
  v.x = rem > 0 ? ld_stream(p + e0) : 0;
  v.y = rem > 1 ? ld_stream(p + e0 + 1) : 0;
  v.z = rem > 2 ? ld_stream(p + e0 + 2) : 0;
  v.w = rem > 3 ? ld_stream(p + e0 + 3) : 0;
  return v;
}

// The int64 values of rows e0..e0+3 selected by `bits` (others unspecified).
template <bool VEC>
__device__ __forceinline__ void load_i64x4(const i64* p, i64 e0, i64 rem, u32 bits, u64 pol,
                                           i64 v[4]) {
  if (VEC && rem >= 4) {
    const longlong2 a = ld_stream_v2(p + e0, pol);
    const longlong2 c = ld_stream_v2(p + e0 + 2, pol);
    v[0] = a.x, v[1] = a.y, v[2] = c.x, v[3] = c.y;
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) v[s] = (bits >> s) & 1 ? ld_stream(p + e0 + s) : 0;
  }
}

// Predicate bits of 4 rows; rows at or beyond `rem` never pass.
__device__ __forceinline__ u32 pass4(const Pred32& p, int4 d, i64 rem) {
  const u32 live = rem >= 4 ? 0xFu : rem <= 0 ? 0u : (1u << rem) - 1u;
  return (pass32(p, d.x) | pass32(p, d.y) << 1 | pass32(p, d.z) << 2 | pass32(p, d.w) << 3) &
         live;
}

// Append the rows selected by `bits` (4 per lane) to a warp ring at `tail`:
// slot order is (row-in-lane, lane), fixed by four ballots.  Returns the
// number appended (warp-uniform).
template <typename W>
__device__ __forceinline__ u32 ring_append(u32 bits, u32 tail, W write) {
  const u32 lt = lanemask_lt();
  u32 base = tail;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const u32 m = __ballot_sync(kFull, (bits >> s) & 1u);
    if ((bits >> s) & 1u) write(s, base + __popc(m & lt));
    base += __popc(m);
  }
  return base - tail;
}

// ------------------------------------------------------------------ dscan ----
// Warp tile of 4096 D rows, 512 per iteration: lane l reads seg of rows
// 16l .. 16l+15 with one 128-bit load; keys only where seg passes.
template <bool VEC>
__global__ void __launch_bounds__(256) k_plan_dscan(Batch b) {
  const bool ov = b.ov.table == 1;
  const i64 total = ov ? b.ov.tiles : b.tD[b.nq];
  const int lane = threadIdx.x & 31;
  const u64 strm = policy_stream();
  while (true) {
    const i64 t = warp_claim(b.work, kPhDscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tD, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int* d_key = ov ? (const int*)b.ov.p[0] : q.d_key;
    const signed char* d_seg = ov ? (const signed char*)b.ov.p[1] : q.d_seg;
    const i64 n = ov ? b.ov.n : q.n_d;
    const i64 base = (t - (ov ? 0 : b.tD[qi])) * kTD;
    for (int it = 0; it < kTD / 512; ++it) {
      if (base + it * 512 >= n) break;
      const i64 e0 = base + it * 512 + lane * 16;
      u32 bits = 0;
      if (VEC && e0 + 16 <= n) {
        int4 v = ld_stream_v4(d_seg + e0, strm);
        const signed char* c = reinterpret_cast<const signed char*>(&v);
#pragma unroll
        for (int s = 0; s < 16; ++s) bits |= (u32)pass(q.pd, c[s]) << s;
      } else {
#pragma unroll
        for (int s = 0; s < 16; ++s)
          if (e0 + s < n) bits |= (u32)pass(q.pd, ld_stream(d_seg + e0 + s)) << s;
      }
      u64 at = warp_reserve(&q.ctr->dcount, (u32)__popc(bits));
      while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1;
        q.dlist[at++] = (i64)__ldg(d_key + e0 + s);
      }
    }
  }
  if (finish(b.work, kPhDscan)) {
    block_prefix(b.dyn, b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      if (!q.build_dset) return 0;
      const int e = cap_log2(ld_count(&q.ctr->dcount), q.lf1024);
      *q.dset_log2 = e;
      return (((i64)1 << e) + kTC - 1) / kTC;
    });
    block_prefix(b.dyn + (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      return q.build_dset ? (ld_count(&q.ctr->dcount) + kTB - 1) / kTB : 0;
    });
  }
}

// ------------------------------------------------------------------- fill ----
// Clear the tags (2 bytes per slot) of the D-set (which = 0) or the M table
// (which = 1); keys and sums are written by the inserting thread.
__global__ void __launch_bounds__(256) k_plan_fill(Batch b, int which) {
  const i64* pre = b.dyn + (which == 0 ? 0 : 2) * (b.nq + 1);
  const int ph = which == 0 ? kPhDfill : kPhMfill;
  const i64 total = pre[b.nq];
  while (true) {
    const i64 t = claim(b.work, ph);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int e = which == 0 ? *q.dset_log2 : q.ctr->mlog2;
    unsigned short* dst = which == 0 ? q.dset_tag : q.ht_tag;
    const i64 n = (i64)1 << e;
    const i64 s0 = (t - pre[qi]) * kTC;
    for (i64 i = s0 + threadIdx.x * 8; i < s0 + kTC && i < n; i += 256 * 8)
      *reinterpret_cast<int4*>(dst + i) = make_int4(0, 0, 0, 0);
  }
  finish(b.work, ph);
}

// ----------------------------------------------------------------- dbuild ----
__global__ void __launch_bounds__(256) k_plan_dbuild(Batch b) {
  const i64* pre = b.dyn + (b.nq + 1);
  const i64 total = pre[b.nq];
  while (true) {
    const i64 t = claim(b.work, kPhDbuild);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const Geo g = geo(*q.dset_log2);
    const i64 n = (i64)q.ctr->dcount;
    const i64 i0 = (t - pre[qi]) * kTB;
    for (i64 i = i0 + threadIdx.x; i < i0 + kTB && i < n; i += blockDim.x)
      tagged_insert(q.dset_tag, q.dset, g, q.dlist[i]);
  }
  finish(b.work, kPhDbuild);
}

// ------------------------------------------------------------------ mscan ----
// Warp tile of 2048 M rows, 128 per iteration (lane l: rows 4l .. 4l+3).
// date is read two iterations ahead and dref one ahead, only for 4-row groups
// with a date hit.  Date-passing (dref, row) pairs enter ring A and are
// probed against the D-set 32 at a time; the keys of the members (read only
// for them) enter ring B and leave for the M list in runs of 128 (one atomic
// reservation per run).
template <bool VEC>
__global__ void __launch_bounds__(256, 4) k_plan_mscan(Batch b) {
  __shared__ int s_ad[8][kQ];
  __shared__ u32 s_ar[8][kQ];
  __shared__ i64 s_rb[8][kQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* ad = s_ad[warp];
  u32* ar = s_ar[warp];
  i64* rb = s_rb[warp];
  const u64 keep = policy_keep(), strm = policy_stream();
  const bool ov = b.ov.table == 2;
  const i64 total = ov ? b.ov.tiles : b.tM[b.nq];
  while (true) {
    const i64 t = warp_claim(b.work, kPhMscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tM, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* m_key = ov ? (const i64*)b.ov.p[0] : q.m_key;
    const int* m_dref = ov ? (const int*)b.ov.p[1] : q.m_dref;
    const int* m_date = ov ? (const int*)b.ov.p[2] : q.m_date;
    const Geo dg = geo(*q.dset_log2);
    const Pred32 pm = to32(q.pm);
    const i64 n = ov ? b.ov.n : q.n_m;
    const i64 base = (t - (ov ? 0 : b.tM[qi])) * kTM;
    const i64 lim = min(n - base, (i64)kTM);
    const int iters = (int)((lim + 127) / 128);
    u32 ah = 0, at = 0, bh = 0, bt = 0;
    auto flush_b = [&](u32 cnt) {
      u64 o = 0;
      if (lane == 0) o = atomicAdd(&q.ctr->mcount, (u64)cnt);
      o = __shfl_sync(kFull, o, 0);
      for (u32 j = lane; j < cnt; j += 32) q.mlist[o + j] = rb[(bh + j) & (kQ - 1)];
      bh += cnt;
    };
    auto probe_a = [&](u32 cnt) {
      bool mem = false;
      i64 key = 0;
      if ((u32)lane < cnt) {
        const u32 j = (ah + lane) & (kQ - 1);
        mem = set_contains(q.dset_tag, q.dset, dg, ad[j], keep);
        if (mem) key = __ldg(m_key + base + ar[j]);
      }
      const u32 m = __ballot_sync(kFull, mem);
      if (mem) rb[(bt + __popc(m & lanemask_lt())) & (kQ - 1)] = key;
      bt += __popc(m);
      ah += cnt;
      __syncwarp();
      if (bt - bh >= 128) flush_b(128);
    };
    const i64 r0 = lane * 4;
    int4 dB = load_i32x4<VEC>(m_date, base + r0, lim - r0, strm);
    int4 dC = iters > 1 ? load_i32x4<VEC>(m_date, base + 128 + r0, lim - 128 - r0, strm)
                        : make_int4(0, 0, 0, 0);
    u32 hA = pass4(pm, dB, lim - r0);
    int4 rA = hA ? load_i32x4<VEC>(m_dref, base + r0, lim - r0, strm) : make_int4(0, 0, 0, 0);
    dB = dC;
    if (iters > 2) dC = load_i32x4<VEC>(m_date, base + 256 + r0, lim - 256 - r0, strm);
    for (int it = 0; it < iters; ++it) {
      const i64 rel1 = (it + 1) * 128 + r0;
      u32 hB = 0;
      int4 rB = make_int4(0, 0, 0, 0);
      if (it + 1 < iters) {
        hB = pass4(pm, dB, lim - rel1);
        if (hB) rB = load_i32x4<VEC>(m_dref, base + rel1, lim - rel1, strm);
      }
      dB = dC;
      if (it + 3 < iters) {
        const i64 rel3 = (it + 3) * 128 + r0;
        dC = load_i32x4<VEC>(m_date, base + rel3, lim - rel3, strm);
      }
      const int dr[4] = {rA.x, rA.y, rA.z, rA.w};
      __syncwarp();
      at += ring_append(hA, at, [&](int s, u32 pos) {
        ad[pos & (kQ - 1)] = dr[s];
        ar[pos & (kQ - 1)] = (u32)(it * 128 + r0 + s);
      });
      __syncwarp();
      while (at - ah >= 32) probe_a(32);
      hA = hB;
      rA = rB;
    }
    __syncwarp();
    if (at - ah) probe_a(at - ah);
    if (bt - bh) flush_b(bt - bh);
    __syncwarp();
  }
  if (finish(b.work, kPhMscan)) {
    block_prefix(b.dyn + 2 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      const int e = cap_log2(ld_count(&q.ctr->mcount), q.lf1024);
      q.ctr->mlog2 = e;
      return (((i64)1 << e) + kTC - 1) / kTC;
    });
    block_prefix(b.dyn + 3 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      return (ld_count(&b.q[qi].ctr->mcount) + kTB - 1) / kTB;
    });
  }
}

// ----------------------------------------------------------------- mbuild ----
__global__ void __launch_bounds__(256) k_plan_mbuild(Batch b) {
  const i64* pre = b.dyn + 3 * (b.nq + 1);
  const i64 total = pre[b.nq];
  while (true) {
    const i64 t = claim(b.work, kPhMbuild);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const Geo g = geo(q.ctr->mlog2);
    const i64 n = (i64)q.ctr->mcount;
    const i64 i0 = (t - pre[qi]) * kTB;
    for (i64 i = i0 + threadIdx.x; i < i0 + kTB && i < n; i += blockDim.x) {
      const i64 k = q.mlist[i];
      if (k == kEmpty) {
        q_latch(q.ctr, b.st, PQ_ERR_RESERVED_KEY, i);
        continue;
      }
      const u64 s = tagged_insert(q.ht_tag, q.ht_keys, g, k);
      q.ht_sums[s] = 0;
      q.ht_cnt[s] = 0;
    }
  }
  finish(b.work, kPhMbuild);
}

// ----------------------------------------------------------------- fprobe ----
struct ProbeCtx {
  const unsigned short* tags;
  const i64* keys;
  i64* sums;
  u32* cnt;
  u32* glist;
  QCtr* ctr;
  const i64* price;
  const signed char* disc;
  DevStatus* st;
  i64 base;
  u64 keep;
  Geo g;
};

// Finish the probe of key k (F row base + r) whose home bucket's tag word w
// has been read: count the slots holding k (its multiplicity in M', found in
// the home bucket and, while buckets are full, the next ones) and add the
// row's exact revenue times that count into the first of them, recording
// that slot as a group on its first hit.
__device__ __forceinline__ void probe_finish(const ProbeCtx& c, i64 k, u32 r, BucketTag bt,
                                             uint4 w) {
  i64 first = -1, mult = 0;
  const unsigned v2 = bt.tag * 0x10001u;
  u64 b = bt.bucket;
  for (u64 p = 0; p <= c.g.bmask; ++p) {
    Mask8 m = match8(w, v2);
    while (any8(m)) {
      const int j = first8(m);
      const u64 slot = b * 8 + j;
      if (ld_keep(c.keys + slot, c.keep) == k) {
        if (first < 0) first = (i64)slot;
        ++mult;
      }
      drop8(m, j);
    }
    if (any8(match8(w, 0u))) break;
    b = (b + 1) & c.g.bmask;
    w = ld_keep_v4u(c.tags + b * 8, c.keep);
  }
  if (first < 0) return;
  const i64 row = c.base + r;
  // Exact revenue: the product is formed in 128 bits so that a value outside
  // int64 is reported instead of wrapping.
  const __int128 v128 =
      (__int128)mult * ((__int128)__ldg(c.price + row) * (100 - (i64)__ldg(c.disc + row)));
  const i64 v = (i64)v128;
  if (v128 != (__int128)v) q_latch(c.ctr, c.st, PQ_ERR_OVERFLOW, k);
  const i64 old = (i64)atomicAdd((u64*)&c.sums[first], (u64)v);
  if ((v > 0 && old > INT64_MAX - v) || (v < 0 && old < INT64_MIN - v))
    q_latch(c.ctr, c.st, PQ_ERR_OVERFLOW, k);
  if (*(volatile u32*)&c.cnt[first] == 0 && atomicExch(&c.cnt[first], 1u) == 0u) {
    const u64 gi = atomicAdd(&c.ctr->gcount, 1ULL);
    c.glist[gi] = (u32)first;
  }
}

__device__ __forceinline__ void probe1(const ProbeCtx& c, i64 k, u32 r) {
  const BucketTag bt = bucket_tag(k, c.g.shiftb);
  probe_finish(c, k, r, bt, ld_keep_v4u(c.tags + bt.bucket * 8, c.keep));
}

// Two probes per lane with both home-bucket loads in flight together.
__device__ __forceinline__ void probe2(const ProbeCtx& c, i64 k0, u32 r0, i64 k1, u32 r1) {
  const BucketTag b0 = bucket_tag(k0, c.g.shiftb), b1 = bucket_tag(k1, c.g.shiftb);
  const uint4 w0 = ld_keep_v4u(c.tags + b0.bucket * 8, c.keep);
  const uint4 w1 = ld_keep_v4u(c.tags + b1.bucket * 8, c.keep);
  probe_finish(c, k0, r0, b0, w0);
  probe_finish(c, k1, r1, b1, w1);
}

// Warp tile of 4096 F rows, 128 per iteration (lane l: rows 4l .. 4l+3).
// date2 is read two iterations ahead and mkey one ahead, only for 4-row groups
// (one 32-byte sector) with a passing row.  Passing (key, row) pairs enter the
// warp's ring and are probed 64 at a time, two per lane.
template <bool VEC>
__global__ void __launch_bounds__(256, 4) k_plan_fprobe(Batch b) {
  __shared__ i64 s_qk[8][kQ];
  __shared__ u32 s_qr[8][kQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  i64* qk = s_qk[warp];
  u32* qr = s_qr[warp];
  const u64 keep = policy_keep(), strm = policy_stream();
  const bool ov = b.ov.table == 3;
  const i64 total = ov ? b.ov.tiles : b.tF[b.nq];
  while (true) {
    const i64 t = warp_claim(b.work, kPhFprobe);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tF, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* f_mkey = ov ? (const i64*)b.ov.p[0] : q.f_mkey;
    const int* f_date = ov ? (const int*)b.ov.p[3] : q.f_date;
    const i64 n = ov ? b.ov.n : q.n_f;
    const i64 base = (t - (ov ? 0 : b.tF[qi])) * kTF;
    ProbeCtx pc;
    pc.tags = q.ht_tag;
    pc.keys = q.ht_keys;
    pc.sums = q.ht_sums;
    pc.cnt = q.ht_cnt;
    pc.glist = q.glist;
    pc.ctr = q.ctr;
    pc.price = ov ? (const i64*)b.ov.p[1] : q.f_price;
    pc.disc = ov ? (const signed char*)b.ov.p[2] : q.f_disc;
    pc.st = b.st;
    pc.base = base;
    const int e = q.ctr->mlog2;
    pc.g = geo(e);
    pc.keep = keep;
    const Pred32 pf = to32(q.pf);
    const i64 lim = min(n - base, (i64)kTF);
    const int iters = (int)((lim + 127) / 128);
    const i64 r0 = lane * 4;
    u32 head = 0, tail = 0;
    int4 dB = load_i32x4<VEC>(f_date, base + r0, lim - r0, strm);
    int4 dC = iters > 1 ? load_i32x4<VEC>(f_date, base + 128 + r0, lim - 128 - r0, strm)
                        : make_int4(0, 0, 0, 0);
    u32 bA = pass4(pf, dB, lim - r0);
    i64 mA[4] = {0, 0, 0, 0};
    if (bA) load_i64x4<VEC>(f_mkey, base + r0, lim - r0, bA, strm, mA);
    dB = dC;
    if (iters > 2) dC = load_i32x4<VEC>(f_date, base + 256 + r0, lim - 256 - r0, strm);
    for (int it = 0; it < iters; ++it) {
      const i64 rel1 = (it + 1) * 128 + r0;
      u32 bB = 0;
      i64 mB[4] = {0, 0, 0, 0};
      if (it + 1 < iters) {
        bB = pass4(pf, dB, lim - rel1);
        if (bB) load_i64x4<VEC>(f_mkey, base + rel1, lim - rel1, bB, strm, mB);
      }
      dB = dC;
      if (it + 3 < iters) {
        const i64 rel3 = (it + 3) * 128 + r0;
        dC = load_i32x4<VEC>(f_date, base + rel3, lim - rel3, strm);
      }
      __syncwarp();
      tail += ring_append(bA, tail, [&](int s, u32 pos) {
        qk[pos & (kQ - 1)] = mA[s];
        qr[pos & (kQ - 1)] = (u32)(it * 128 + r0 + s);
      });
      __syncwarp();
      while (tail - head >= 64) {
        const u32 j0 = (head + lane) & (kQ - 1), j1 = (head + 32 + lane) & (kQ - 1);
        probe2(pc, qk[j0], qr[j0], qk[j1], qr[j1]);
        head += 64;
      }
      bA = bB;
#pragma unroll
      for (int s = 0; s < 4; ++s) mA[s] = mB[s];
    }
    __syncwarp();
    if (tail - head >= 32) {
      const u32 j = (head + lane) & (kQ - 1);
      probe1(pc, qk[j], qr[j]);
      head += 32;
    }
    if ((u32)lane < tail - head) {
      const u32 j = (head + lane) & (kQ - 1);
      probe1(pc, qk[j], qr[j]);
    }
    __syncwarp();
  }
  if (finish(b.work, kPhFprobe)) {
    block_prefix(b.dyn + 4 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      const i64 g = ld_count(&q.ctr->gcount);
      q.out->ngroups = g;
      q.out->status = q.ctr->status;
      q.out->reserved = 0;
      if (g == 0) q.out->n = 0;
      return (g + kTK - 1) / kTK;
    });
  }
}

// ------------------------------------------------------------------- topk ----
// Per (plan, 1024 groups) block top-k; the block that finishes a plan's last
// chunk merges the partial lists with all its warps, then warp 0 merges those.
__global__ void __launch_bounds__(256) k_plan_topk(Batch b) {
  __shared__ i64 sk[8 * kMaxK], ss[8 * kMaxK];
  __shared__ int sc[8];
  __shared__ bool s_last;
  const i64* pre = b.dyn + 4 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    const i64 t = claim(b.work, kPhTopk);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int K = q.k;
    const i64 n = (i64)q.ctr->gcount;
    const i64 lt = t - pre[qi];
    const i64 i0 = lt * kTK, i1 = min(n, i0 + kTK);
    TopList L;
    L.clear();
    for (i64 i = i0; i < i1; i += blockDim.x) {
      const i64 j = i + threadIdx.x;
      const bool v = j < i1;
      const u32 s = v ? q.glist[j] : 0u;
      L.offer(K, v, v ? q.ht_keys[s] : 0, v ? q.ht_sums[s] : 0);
    }
    tk_block_merge(L, K, sk, ss, sc);
    if (threadIdx.x < 32) {
      L.store(q.tk_k + lt * K, q.tk_s + lt * K);
      if (lane == 0) q.tk_c[lt] = L.cnt;
      __threadfence();
      u32 tk = 0;
      if (lane == 0) tk = atomicAdd(&q.ctr->tk_ticket, 1u);
      tk = __shfl_sync(kFull, tk, 0);
      const i64 parts = pre[qi + 1] - pre[qi];
      if (lane == 0) s_last = ((i64)tk == parts - 1);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      const i64 cand = (pre[qi + 1] - pre[qi]) * K;
      L.clear();
      for (i64 j = (i64)warp * 32; j < cand; j += blockDim.x) {
        const i64 e = j + lane;
        const bool v = e < cand && (int)(e % K) < *(volatile int*)&q.tk_c[e / K];
        L.offer(K, v, v ? *(volatile i64*)&q.tk_k[e] : 0, v ? *(volatile i64*)&q.tk_s[e] : 0);
      }
      tk_block_merge(L, K, sk, ss, sc);
      if (threadIdx.x < 32) {
        L.store((i64*)q.out->keys, (i64*)q.out->sums);
        if (lane == 0) q.out->n = L.cnt;
      }
    }
  }
  finish(b.work, kPhTopk);
}

#endif  // PQ_DEFINE_PLAN_KERNELS

}  // namespace pqk
