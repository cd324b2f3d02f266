// pq_agg.cu -- the aggregate-first plan (PQ_PLAN_AGG_FIRST): a large
// materialised group-by filtered on its aggregate (the shape of the paper's
// Q18 remark, Sec. 6.3), on resident tables with dense keys.
//
//   D' bitmap  <- D rows with seg op_d c_d                  (k_agg_dbits)
//   M' bitmap  <- M rows with date op_m c_m, dref in D'      (k_agg_mbits)
//   G          <- F rows with date2 op_f c_f: sums[mkey] += price*(100-disc),
//                 a group per set bit of the F key range     (k_agg_fscan)
//   candidates <- groups with sum > having and key in M'     (k_agg_select)
//   result     <- top-k of the candidates (the top-k operator's kernel) and
//                 their number                               (k_agg_result)
//
// The group sums live in a dense array over the F key range (8 bytes per key
// of the range), so the plan needs keys whose range is at most a few times
// the F row count.  Lanes that hit the same group combine their revenues
// first (exact 128-bit sum); the group's sum is then one reduction nobody
// waits for.  int64 overflow: each revenue is formed in 128 bits; a group sum
// can only leave int64 if the magnitudes of all summed revenues exceed 2^62,
// which the plan tracks (one atomic per warp) and reports as PQ_ERR_OVERFLOW.
#include <algorithm>

#include "pq_plan_host.h"

using namespace pqk;

namespace pqh {

namespace {

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
  u32* hit;
  i64 having;
  i64* cand_k;
  i64* cand_s;
  u64* ctr;  // [0] candidates, [1] sum of |revenue| (saturating at 2^62), [2] F rows, [3] status
  DevStatus* st;  // the context's error latch (read by pq_sync)
};

constexpr u64 kMag = 1ULL << 62;

__global__ void __launch_bounds__(256) k_agg_dbits(AggPlan a) {
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_d; i += stride)
    if (pass(a.pd, a.d_seg[i])) bit_set(a.dbm, ukey((i64)a.d_key[i]) - a.d_base);
}

__global__ void __launch_bounds__(256) k_agg_mbits(AggPlan a) {
  const u64 keep = policy_keep();
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_m; i += stride) {
    if (!pass32(a.pm, a.m_date[i])) continue;
    const u64 di = ukey((i64)a.m_dref[i]) - a.d_base;
    if (di < a.d_bits && bit_test(a.dbm, di, keep))
      bit_set(a.mbm, ukey(a.m_key[i]) - a.m_base);
  }
}

// F rows: each lane takes 4 consecutive rows per step; for each of its rows
// the lanes of the warp holding the same group add up their revenues and the
// lowest of them commits the total.
__global__ void __launch_bounds__(256) k_agg_fscan(AggPlan a) {
  __shared__ i64 s_v[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  i64* sv = s_v[warp];
  const i64 nw = (i64)gridDim.x * (blockDim.x >> 5);
  u64 mag = 0, rows = 0;
  bool ovf = false;
  for (i64 g = (i64)blockIdx.x * (blockDim.x >> 5) + warp; g * 128 < a.n_f; g += nw) {
    const i64 r0 = g * 128 + 4 * lane;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const i64 r = r0 + s;
      bool act = false;
      u64 idx = ~0ULL;
      i64 v = 0;
      if (r < a.n_f && pass32(a.pf, __ldg(a.f_date + r))) {
        idx = ukey(__ldg(a.f_mkey + r)) - a.f_base;
        const __int128 rev = (__int128)__ldg(a.f_price + r) * (100 - (int)a.f_disc[r]);
        v = (i64)rev;
        ovf = ovf || rev != (__int128)v;
        act = true;
        ++rows;
        const u64 m = v < 0 ? (u64)0 - (u64)v : (u64)v;
        mag = mag >= kMag || m >= kMag ? kMag : min(kMag, mag + m);
      }
      const u32 peers = __match_any_sync(kFull, idx);
      const bool lead = act && __ffs(peers) - 1 == lane;
      sv[lane] = v;
      __syncwarp();
      if (lead) {
        __int128 acc = 0;
        for (u32 p = peers; p; p &= p - 1) acc += sv[__ffs(p) - 1];
        const i64 tot = (i64)acc;
        ovf = ovf || acc != (__int128)tot;
        atomicAdd(reinterpret_cast<unsigned long long*>(a.sums + idx), (unsigned long long)tot);
        atomicOr(a.hit + (idx >> 5), 1u << (idx & 31));
      }
      __syncwarp();
    }
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

// Groups (set bits of the F key range) whose sum exceeds the threshold and
// whose key is in M', appended as (key, sum) candidates.
__global__ void __launch_bounds__(256) k_agg_select(AggPlan a) {
  const u64 keep = policy_keep();
  const int lane = threadIdx.x & 31;
  const i64 words = (i64)((a.f_bits + 31) / 32);
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 w0 = (i64)blockIdx.x * blockDim.x; w0 < words; w0 += stride) {
    const i64 w = w0 + threadIdx.x;
    u32 bits = w < words ? a.hit[w] : 0u;
    while (__any_sync(kFull, bits)) {
      bool take = false;
      i64 key = 0, sum = 0;
      if (bits) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1;
        const u64 idx = (u64)w * 32 + (u64)j;
        sum = a.sums[idx];
        const u64 uk = a.f_base + idx;
        const u64 mi = uk - a.m_base;
        key = (i64)(uk ^ (1ULL << 63));
        take = sum > a.having && mi < a.m_bits && bit_test(a.mbm, mi, keep);
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

}  // namespace

pq_status run_plan_aggfirst(pq_ctx* ctx, const pq_plan& plan, pq_result* result, cudaStream_t s) {
  ResolvedPlan r;
  pq_status st = resolve_plan(ctx, plan, r, true);
  if (st != PQ_OK) return st;
  const PlanDev& d = r.dev;
  // Key ranges of the whole tables, measured once per column.
  const pq_table* T[3] = {plan.D, plan.M, plan.F};
  for (int t = 0; t < 3; ++t)
    if (T[t]->nrows > 0 && !ensure_range(ctx, T[t], 0, s))
      return fail(ctx, PQ_ERR_CUDA, "aggregate-first plan: key range of table %d", t);
  auto span = [&](int t) -> u64 {
    const Column& c = T[t]->cols[0];
    return c.has_range && c.umax >= c.umin ? c.umax - c.umin + 1 : 0;
  };
  const u64 d_bits = span(0), m_bits = span(1), f_bits = span(2);
  const u64 dense_cap = 4ULL * (u64)std::max<i64>(r.n_f, 1) + 4096;
  if (f_bits > dense_cap || f_bits > kMaxBmBits || m_bits > kMaxBmBits || d_bits > kMaxBmBits)
    return fail(ctx, PQ_ERR_INVALID_ARG,
                "aggregate-first plan: F keys span %llu values for %lld rows (dense keys needed)",
                (unsigned long long)f_bits, (long long)r.n_f);
  const size_t cap = (size_t)std::max<u64>(f_bits, 1);  // candidates: at most one per key
  auto words = [](u64 bits) { return (size_t)((bits + 31) / 32) * 4; };
  Scratch scr(ctx, s);
  const size_t zero = 256 + al256(words(d_bits)) + al256(words(m_bits)) + al256(words(f_bits)) +
                      al256(8 * cap);
  char* z = (char*)scr.get(zero);
  char* c = (char*)scr.get(al256(16 * cap) + al256(16 * PQ_MAX_K) + 256 + sizeof(pq_result));
  if (!z || !c) return fail(ctx, PQ_ERR_BUDGET, "aggregate-first plan: %zu bytes", zero + 16 * cap);
  AggPlan a{};
  a.ctr = (u64*)z;
  a.dbm = (u32*)(z + 256);
  a.mbm = (u32*)((char*)a.dbm + al256(words(d_bits)));
  a.hit = (u32*)((char*)a.mbm + al256(words(m_bits)));
  a.sums = (i64*)((char*)a.hit + al256(words(f_bits)));
  a.cand_k = (i64*)c;
  a.cand_s = a.cand_k + cap;
  i64* ok = (i64*)(c + al256(16 * cap));
  i64* os = ok + PQ_MAX_K;
  i64* nout = (i64*)(c + al256(16 * cap) + al256(16 * PQ_MAX_K));
  pq_result* dres = (pq_result*)((char*)nout + 256);
  a.d_key = d.d_key, a.d_seg = d.d_seg, a.n_d = r.n_d, a.pd = d.pd;
  a.d_base = T[0]->cols[0].umin, a.d_bits = d_bits;
  a.m_key = d.m_key, a.m_dref = d.m_dref, a.m_date = d.m_date, a.n_m = r.n_m, a.pm = to32(d.pm);
  a.m_base = T[1]->cols[0].umin, a.m_bits = m_bits;
  a.f_mkey = d.f_mkey, a.f_price = d.f_price, a.f_disc = d.f_disc, a.f_date = d.f_date;
  a.n_f = r.n_f, a.pf = to32(d.pf);
  a.f_base = T[2]->cols[0].umin, a.f_bits = f_bits;
  a.having = plan.having;
  a.st = ctx->d_status;
  PQ_CUDA(ctx, cudaMemsetAsync(z, 0, zero, s));
  const int sms = ctx->num_sms;
  auto grid = [&](i64 n, i64 per) {
    return (int)std::max<i64>(1, std::min<i64>((n + per - 1) / per, (i64)sms * 8));
  };
  // A table with rows has a measured range, so every key of the plan's rows
  // indexes inside its bitmap or sum array.
  if (d_bits) k_agg_dbits<<<grid(r.n_d, 256), 256, 0, s>>>(a);
  if (d_bits && m_bits) k_agg_mbits<<<grid(r.n_m, 256), 256, 0, s>>>(a);
  if (f_bits) {
    k_agg_fscan<<<grid(r.n_f, 8 * 128), 256, 0, s>>>(a);
    k_agg_select<<<grid((i64)(f_bits + 31) / 32, 256), 256, 0, s>>>(a);
  }
  PQ_CUDA(ctx, cudaGetLastError());
  ctx->launches += 4;
  st = pq_topk(ctx, (const int64_t*)a.cand_k, (const int64_t*)a.cand_s, (int64_t)cap,
               (const int64_t*)a.ctr, d.k, (int64_t*)ok, (int64_t*)os, (int64_t*)nout, s);
  if (st != PQ_OK) return st;
  k_agg_result<<<1, 64, 0, s>>>(a.ctr, ok, os, nout, d.k, dres);
  PQ_CUDA(ctx, cudaGetLastError());
  ctx->launches += 1;
  ctx->plans++;
  return read_back(ctx, result, dres, 1, s);
}

}  // namespace pqh
