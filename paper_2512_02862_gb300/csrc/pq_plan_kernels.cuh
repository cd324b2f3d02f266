// pq_plan_kernels.cuh -- the kernels of the three-table plan, batched.
//
// One launch of each kernel serves every plan of a batch: persistent blocks
// claim tiles of a flattened work list (atomic ticket, work stealing) and map
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
#pragma once
#include "../../include/pq.h"
#include "pq_dev.cuh"
#include "pq_topk.cuh"

namespace pqk {

constexpr int kTD = 8192;   // D rows per tile
constexpr int kTM = 4096;   // M rows per tile
constexpr int kTF = 8192;   // F rows per tile
constexpr int kTC = 8192;   // slots cleared per tile
constexpr int kTB = 4096;   // list entries inserted per tile
constexpr int kTK = 4096;   // groups per top-k tile

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
  i64* dset;        // D-set slots
  i64* mlist;
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

// Claim the next tile of phase `ph` (block-wide).
__device__ __forceinline__ i64 claim(u32* work, int ph) {
  __shared__ i64 s_t;
  __syncthreads();
  if (threadIdx.x == 0) s_t = atomicAdd(&work[ph], 1u);
  __syncthreads();
  return s_t;
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

// Block-wide exclusive scan helper over nq values produced by `f(q)`; writes
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

__device__ __forceinline__ bool set_contains(const i64* set, u64 mask, i64 k) {
  u64 s = slot_hash(k) & mask;
  for (u64 p = 0; p <= mask; ++p) {
    const i64 kk = __ldg(set + s);
    if (kk == k) return true;
    if (kk == kEmpty) return false;
    s = (s + 1) & mask;
  }
  return false;
}

// ------------------------------------------------------------------ dscan ----
// Tile of 8192 D rows; thread t handles rows 16t .. 16t+15 of each half (one
// 128-bit load of seg = 16 int8 rows), keys are loaded only where seg passes.
template <bool VEC>
__global__ void __launch_bounds__(256) k_plan_dscan(Batch b) {
  const bool ov = b.ov.table == 1;
  const i64 total = ov ? b.ov.tiles : b.tD[b.nq];
  while (true) {
    const i64 t = claim(b.work, kPhDscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tD, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int* d_key = ov ? (const int*)b.ov.p[0] : q.d_key;
    const signed char* d_seg = ov ? (const signed char*)b.ov.p[1] : q.d_seg;
    const i64 n = ov ? b.ov.n : q.n_d;
    const i64 r0 = (t - (ov ? 0 : b.tD[qi])) * kTD;
    for (int half = 0; half < kTD / 4096; ++half) {
      const i64 e0 = r0 + half * 4096 + threadIdx.x * 16;
      u32 bits = 0;
      if (VEC && e0 + 16 <= n) {
        int4 v = ld_stream(reinterpret_cast<const int4*>(d_seg + e0));
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
// which = 0: D-set slots, 1: M table keys.
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
    i64* dst = which == 0 ? q.dset : q.ht_keys;
    const i64 n = (i64)1 << e;
    const i64 s0 = (t - pre[qi]) * kTC;
    for (i64 i = s0 + threadIdx.x * 2; i < s0 + kTC && i < n; i += 512)
      *reinterpret_cast<longlong2*>(dst + i) = make_longlong2(kEmpty, kEmpty);
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
    const u64 mask = (1ULL << *q.dset_log2) - 1;
    const i64 n = (i64)q.ctr->dcount;
    const i64 i0 = (t - pre[qi]) * kTB;
    for (i64 i = i0 + threadIdx.x; i < i0 + kTB && i < n; i += blockDim.x) {
      const i64 k = q.dlist[i];
      u64 s = slot_hash(k) & mask;
      for (u64 p = 0; p <= mask; ++p) {
        const i64 old = (i64)atomicCAS((u64*)&q.dset[s], (u64)kEmpty, (u64)k);
        if (old == kEmpty || old == k) break;
        s = (s + 1) & mask;
      }
    }
  }
  finish(b.work, kPhDbuild);
}

// ------------------------------------------------------------------ mscan ----
// Tile of 4096 M rows laid out like the filter: warp w, group g, lane l reads
// rows w*512 + g*128 + 4l .. +3.  dref is read only for groups with a date
// hit, the key only for groups with a D-set member.
template <bool VEC>
__global__ void __launch_bounds__(256) k_plan_mscan(Batch b) {
  const bool ov = b.ov.table == 2;
  const i64 total = ov ? b.ov.tiles : b.tM[b.nq];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    const i64 t = claim(b.work, kPhMscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tM, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* m_key = ov ? (const i64*)b.ov.p[0] : q.m_key;
    const int* m_dref = ov ? (const int*)b.ov.p[1] : q.m_dref;
    const int* m_date = ov ? (const int*)b.ov.p[2] : q.m_date;
    const u64 dmask = (1ULL << *q.dset_log2) - 1;
    const i64 r0 = (t - (ov ? 0 : b.tM[qi])) * kTM + warp * 512 + lane * 4;
    const i64 n = ov ? b.ov.n : q.n_m;
    u32 member = 0;
    i64 keys[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const i64 e0 = r0 + g * 128;
      int dt[4];
      if (VEC && e0 + 4 <= n) {
        int4 v = ld_stream(reinterpret_cast<const int4*>(m_date + e0));
        dt[0] = v.x, dt[1] = v.y, dt[2] = v.z, dt[3] = v.w;
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) dt[s] = e0 + s < n ? ld_stream(m_date + e0 + s) : 0;
      }
      u32 hit = 0;
#pragma unroll
      for (int s = 0; s < 4; ++s) hit |= (u32)(e0 + s < n && pass(q.pm, dt[s])) << s;
      if (hit) {
        int dr[4];
        if (VEC && e0 + 4 <= n) {
          int4 v = ld_stream(reinterpret_cast<const int4*>(m_dref + e0));
          dr[0] = v.x, dr[1] = v.y, dr[2] = v.z, dr[3] = v.w;
        } else {
#pragma unroll
          for (int s = 0; s < 4; ++s) dr[s] = (hit >> s) & 1 ? ld_stream(m_dref + e0 + s) : 0;
        }
        u32 mem = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if ((hit >> s) & 1) mem |= (u32)set_contains(q.dset, dmask, dr[s]) << s;
        if (mem) {
          if (VEC && e0 + 4 <= n) {
            longlong2 a = ld_stream(reinterpret_cast<const longlong2*>(m_key + e0));
            longlong2 c = ld_stream(reinterpret_cast<const longlong2*>(m_key + e0 + 2));
            keys[g * 4 + 0] = a.x, keys[g * 4 + 1] = a.y, keys[g * 4 + 2] = c.x,
                         keys[g * 4 + 3] = c.y;
          } else {
#pragma unroll
            for (int s = 0; s < 4; ++s)
              keys[g * 4 + s] = (mem >> s) & 1 ? ld_stream(m_key + e0 + s) : 0;
          }
        }
        member |= mem << (4 * g);
      }
    }
    u64 at = warp_reserve(&q.ctr->mcount, (u32)__popc(member));
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if ((member >> j) & 1) q.mlist[at++] = keys[j];
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
    const u64 mask = (1ULL << q.ctr->mlog2) - 1;
    const i64 n = (i64)q.ctr->mcount;
    const i64 i0 = (t - pre[qi]) * kTB;
    for (i64 i = i0 + threadIdx.x; i < i0 + kTB && i < n; i += blockDim.x) {
      const i64 k = q.mlist[i];
      if (k == kEmpty) {
        q_latch(q.ctr, b.st, PQ_ERR_RESERVED_KEY, i);
        continue;
      }
      u64 s = slot_hash(k) & mask;
      for (u64 p = 0; p <= mask; ++p) {
        const i64 old = (i64)atomicCAS((u64*)&q.ht_keys[s], (u64)kEmpty, (u64)k);
        if (old == kEmpty) {
          q.ht_sums[s] = 0;
          q.ht_cnt[s] = 0;
          break;
        }
        if (old == k) q.ctr->dup = 1;
        s = (s + 1) & mask;
      }
    }
  }
  finish(b.work, kPhMbuild);
}

// ----------------------------------------------------------------- fprobe ----
// Tile of 8192 F rows in 8 groups of 1024 (thread t: rows 4t .. 4t+3 of each
// group).  All date2 loads of the tile are issued before any is used; mkey is
// read only for groups with a passing row; price and disc only on a hit.
template <bool VEC>
__global__ void __launch_bounds__(256) k_plan_fprobe(Batch b) {
  const bool ov = b.ov.table == 3;
  const i64 total = ov ? b.ov.tiles : b.tF[b.nq];
  while (true) {
    const i64 t = claim(b.work, kPhFprobe);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tF, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* f_mkey = ov ? (const i64*)b.ov.p[0] : q.f_mkey;
    const i64* f_price = ov ? (const i64*)b.ov.p[1] : q.f_price;
    const signed char* f_disc = ov ? (const signed char*)b.ov.p[2] : q.f_disc;
    const int* f_date = ov ? (const int*)b.ov.p[3] : q.f_date;
    const int e = q.ctr->mlog2;
    const u64 mask = (1ULL << e) - 1;
    const bool dup = q.ctr->dup != 0;
    const i64 n = ov ? b.ov.n : q.n_f;
    const i64 r0 = (t - (ov ? 0 : b.tF[qi])) * kTF + threadIdx.x * 4;
    int dt[8][4];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const i64 e0 = r0 + g * 1024;
      if (VEC && e0 + 4 <= n) {
        int4 v = ld_stream(reinterpret_cast<const int4*>(f_date + e0));
        dt[g][0] = v.x, dt[g][1] = v.y, dt[g][2] = v.z, dt[g][3] = v.w;
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) dt[g][s] = e0 + s < n ? ld_stream(f_date + e0 + s) : 0;
      }
    }
    u32 hit = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g)
#pragma unroll
      for (int s = 0; s < 4; ++s)
        hit |= (u32)(r0 + g * 1024 + s < n && pass(q.pf, dt[g][s])) << (g * 4 + s);
    if (!hit) continue;
    i64 mk[8][4];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const i64 e0 = r0 + g * 1024;
      const u32 hg = (hit >> (4 * g)) & 0xFu;
      if (!hg) continue;
      if (VEC && e0 + 4 <= n) {
        longlong2 a = ld_stream(reinterpret_cast<const longlong2*>(f_mkey + e0));
        longlong2 c = ld_stream(reinterpret_cast<const longlong2*>(f_mkey + e0 + 2));
        mk[g][0] = a.x, mk[g][1] = a.y, mk[g][2] = c.x, mk[g][3] = c.y;
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) mk[g][s] = (hg >> s) & 1 ? ld_stream(f_mkey + e0 + s) : 0;
      }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (!((hit >> (g * 4 + s)) & 1)) continue;
        const i64 row = r0 + g * 1024 + s;
        const i64 k = mk[g][s];
        u64 slot = slot_hash(k) & mask;
        i64 first = -1, mult = 0;
        for (u64 p = 0; p <= mask; ++p) {
          const i64 kk = __ldg(q.ht_keys + slot);
          if (kk == kEmpty) break;
          if (kk == k) {
            if (first < 0) first = (i64)slot;
            ++mult;
            if (!dup) break;
          }
          slot = (slot + 1) & mask;
        }
        if (first < 0) continue;
        // Exact revenue: the product is formed in 128 bits so that a value
        // outside int64 is reported instead of wrapping.
        const __int128 v128 =
            (__int128)mult * ((__int128)__ldg(f_price + row) * (100 - (i64)__ldg(f_disc + row)));
        const i64 v = (i64)v128;
        if (v128 != (__int128)v) q_latch(q.ctr, b.st, PQ_ERR_OVERFLOW, k);
        const i64 old = (i64)atomicAdd((u64*)&q.ht_sums[first], (u64)v);
        if ((v > 0 && old > INT64_MAX - v) || (v < 0 && old < INT64_MIN - v))
          q_latch(q.ctr, b.st, PQ_ERR_OVERFLOW, k);
        if (*(volatile u32*)&q.ht_cnt[first] == 0 && atomicExch(&q.ht_cnt[first], 1u) == 0u) {
          const u64 gi = atomicAdd(&q.ctr->gcount, 1ULL);
          q.glist[gi] = (u32)first;
        }
      }
    }
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
__global__ void __launch_bounds__(256) k_plan_topk(Batch b) {
  __shared__ i64 sk[8 * kMaxK], ss[8 * kMaxK];
  __shared__ int sc[8];
  __shared__ bool s_last;
  const i64* pre = b.dyn + 4 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31;
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
    if (s_last && threadIdx.x < 32) {
      __threadfence();
      const i64 parts = pre[qi + 1] - pre[qi];
      L.clear();
      for (i64 j = 0; j < parts * K; j += 32) {
        const i64 e = j + lane;
        const bool v = e < parts * K && (int)(e % K) < *(volatile int*)&q.tk_c[e / K];
        L.offer(K, v, v ? *(volatile i64*)&q.tk_k[e] : 0, v ? *(volatile i64*)&q.tk_s[e] : 0);
      }
      L.store((i64*)q.out->keys, (i64*)q.out->sums);
      if (lane == 0) q.out->n = L.cnt;
    }
  }
  finish(b.work, kPhTopk);
}

#endif  // PQ_DEFINE_PLAN_KERNELS

}  // namespace pqk
