// pq_topk.cuh -- warp-register top-k list used by pq_topk and the plan.
//
// Order: larger sum first, ties by smaller key (ORDER BY sum DESC, key ASC).
// A warp keeps its best K <= 64 entries sorted in registers: lane j holds
// entries j and 32 + j.  Candidates are tested 32 at a time against the
// current K-th entry, so after the list fills most candidates cost one
// comparison.  For K <= 32 the candidates that beat it enter together, by
// rank: the list and the candidates are written to a per-warp shared-memory
// scratch, each entry counts what precedes it in the merged order, and the
// first K land in place (no chain of shuffles).  For larger K they enter one
// by one with a warp-wide shift.
#pragma once
#include "pq_dev.cuh"

namespace pqk {

constexpr int kTopScr = 128;  // i64 entries of a warp's TopList scratch

__device__ __forceinline__ bool tk_before(i64 ka, i64 sa, i64 kb, i64 sb) {
  return sa > sb || (sa == sb && ka < kb);
}
// The same order with validity: valid entries first.
__device__ __forceinline__ bool tk_before_v(i64 ka, i64 sa, bool va, i64 kb, i64 sb, bool vb) {
  return va && (!vb || tk_before(ka, sa, kb, sb));
}

// One step of a bitonic network across the warp: exchange with lane ^ stride
// and keep the earlier entry at the lower lane of a pair when `first` (the
// pair's block is ordered earliest first), else the later one.
__device__ __forceinline__ void tk_cmpx(i64& k, i64& s, bool& v, int stride, bool first) {
  const int lane = threadIdx.x & 31;
  const i64 ok = __shfl_xor_sync(kFull, k, stride), os = __shfl_xor_sync(kFull, s, stride);
  const bool ov = __shfl_xor_sync(kFull, v ? 1 : 0, stride) != 0;
  const bool lower = (lane & stride) == 0;
  const bool take = lower == first ? tk_before_v(ok, os, ov, k, s, v)
                                   : tk_before_v(k, s, v, ok, os, ov);
  if (take) k = ok, s = os, v = ov;
}

// Bitonic sort of one entry per lane: lane 0 gets the earliest.
__device__ __forceinline__ void tk_sort32(i64& k, i64& s, bool& v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1)
      tk_cmpx(k, s, v, stride, (lane & size) == 0 || size == 32);
}

struct TopList {
  i64 k0, s0, k1, s1;  // entries lane and 32 + lane
  int cnt;             // warp-uniform number of valid entries
  i64* scr;            // the warp's scratch (kTopScr entries): keys at [0, 64), sums at
                       // [64, 128); list entries at [0, 32), candidates at [32, 64)

  __device__ void clear() {
    k0 = k1 = 0;
    s0 = s1 = 0;
    cnt = 0;
  }
  __device__ void bind(i64* scratch) { scr = scratch; }

  // Entry K-1 (the admission threshold), valid when cnt == K.
  __device__ __forceinline__ void last(int K, i64& k, i64& s) const {
    const int idx = K - 1;
    i64 a = idx < 32 ? k0 : k1, b = idx < 32 ? s0 : s1;
    k = __shfl_sync(kFull, a, idx & 31);
    s = __shfl_sync(kFull, b, idx & 31);
  }

  // Warp-uniform insert of the broadcast candidate (ck, cs).
  __device__ __forceinline__ void insert(int K, i64 ck, i64 cs) {
    const int lane = threadIdx.x & 31;
    const bool b0 = lane < cnt && tk_before(k0, s0, ck, cs);
    const bool b1 = 32 + lane < cnt && tk_before(k1, s1, ck, cs);
    const int pos = __popc(__ballot_sync(kFull, b0)) + __popc(__ballot_sync(kFull, b1));
    if (pos >= K) return;
    const i64 upk0 = __shfl_up_sync(kFull, k0, 1), ups0 = __shfl_up_sync(kFull, s0, 1);
    const i64 upk1 = __shfl_up_sync(kFull, k1, 1), ups1 = __shfl_up_sync(kFull, s1, 1);
    const i64 lk0 = __shfl_sync(kFull, k0, 31), ls0 = __shfl_sync(kFull, s0, 31);
    const int i1 = 32 + lane;
    if (i1 > pos) {
      k1 = lane == 0 ? lk0 : upk1;
      s1 = lane == 0 ? ls0 : ups1;
    } else if (i1 == pos) {
      k1 = ck;
      s1 = cs;
    }
    if (lane > pos) {
      k0 = upk0;
      s0 = ups0;
    } else if (lane == pos) {
      k0 = ck;
      s0 = cs;
    }
    cnt = cnt + 1 < K ? cnt + 1 : K;
  }

  // Merge the candidates of the lanes in m (K <= 32) by rank: the list and
  // the candidates go to shared memory, every list entry and candidate
  // counts the entries that precede it in the merged order (broadcast reads,
  // independent of one another), and the first K land in place.  The merged
  // order is (sum desc, key asc), then list entries before equal
  // candidates, then candidates by lane, so every rank is distinct.
  __device__ __forceinline__ void merge_rank(int K, u32 m, bool want, i64 ck, i64 cs) {
    const int lane = threadIdx.x & 31;
    i64* sk = scr;
    i64* ss = scr + 64;
    sk[lane] = k0, ss[lane] = s0;
    sk[32 + lane] = ck, ss[32 + lane] = cs;
    __syncwarp();
    const bool has = lane < cnt;
    int re = lane;  // rank of this lane's list entry
    int rc = 0;     // rank of this lane's candidate
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      if (!((m >> j) & 1u)) continue;  // m is warp-uniform
      const i64 bk = sk[32 + j], bs = ss[32 + j];
      re += has && tk_before(bk, bs, k0, s0);
      rc += want && j != lane && (tk_before(bk, bs, ck, cs) || (!tk_before(ck, cs, bk, bs) && j < lane));
    }
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) rc += want && !tk_before(ck, cs, sk[j], ss[j]);
    __syncwarp();
    if (has && re < K) sk[re] = k0, ss[re] = s0;
    if (want && rc < K) sk[rc] = ck, ss[rc] = cs;
    __syncwarp();
    const int nc = min(K, cnt + __popc(m));
    if (lane < nc) k0 = sk[lane], s0 = ss[lane];
    __syncwarp();
    cnt = nc;
  }

  // Merge a list of c <= 32 entries (lane j holds entry j; K <= 32).
  __device__ __forceinline__ void merge_list(int K, int c, i64 ck, i64 cs) {
    const int lane = threadIdx.x & 31;
    merge_rank(K, c >= 32 ? kFull : (1u << c) - 1u, lane < c, ck, cs);
  }

  // Offer one candidate per lane (valid lanes only); warp-uniform call.
  __device__ __forceinline__ void offer(int K, bool valid, i64 ck, i64 cs) {
    bool want = valid;
    if (cnt == K) {
      i64 tk, ts;
      last(K, tk, ts);
      want = valid && tk_before(ck, cs, tk, ts);
    }
    u32 m = __ballot_sync(kFull, want);
    if (!m) return;
    if (K <= 32) {
      merge_rank(K, m, want, ck, cs);
      return;
    }
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const i64 k = __shfl_sync(kFull, ck, src), s = __shfl_sync(kFull, cs, src);
      insert(K, k, s);
    }
  }

  // Write entries [0, cnt) to keys/sums (one warp).
  __device__ __forceinline__ void store(i64* keys, i64* sums) const {
    const int lane = threadIdx.x & 31;
    if (lane < cnt) keys[lane] = k0, sums[lane] = s0;
    if (32 + lane < cnt) keys[32 + lane] = k1, sums[32 + lane] = s1;
  }
};

// Branch-free record order (a before b) for the rank counts below.
__device__ __forceinline__ int ks_bef(i64 ak, i64 as, i64 bk, i64 bs) {
  return (int)(as > bs) | ((int)(as == bs) & (int)(ak < bk));
}
// Rank of record x (at index xi) among n records in shared memory (keys k,
// sums s): the records before it, and the equal ones at a lower index, so
// that the ranks of n records are distinct even with repeated records.
// Four independent sums per step, so that the reads overlap.
__device__ __forceinline__ int rank_among(const i64* k, const i64* s, int n, i64 xk, i64 xs,
                                          int xi) {
  int r0 = 0, r1 = 0, r2 = 0, r3 = 0, j = 0;
  auto at = [&](int i) {
    return ks_bef(k[i], s[i], xk, xs) | ((int)(i < xi) & (int)(k[i] == xk) & (int)(s[i] == xs));
  };
  for (; j + 4 <= n; j += 4) r0 += at(j), r1 += at(j + 1), r2 += at(j + 2), r3 += at(j + 3);
  for (; j < n; ++j) r0 += at(j);
  return r0 + r1 + r2 + r3;
}

// A thread's best kLL records, sorted (registers), and the best record it
// dropped.
constexpr int kLL = 4;
struct LaneTop {
  i64 k[kLL], s[kLL];
  int n;
  i64 dk, ds;
  bool dv;
  __device__ __forceinline__ void clear() { n = 0, dv = false, dk = ds = 0; }
  __device__ __forceinline__ void drop(i64 xk, i64 xs) {
    if (!dv || ks_bef(xk, xs, dk, ds)) dk = xk, ds = xs, dv = true;
  }
  __device__ __forceinline__ void insert(i64 xk, i64 xs) {
    if (n == kLL) {
      if (!ks_bef(xk, xs, k[kLL - 1], s[kLL - 1])) {
        drop(xk, xs);
        return;
      }
      drop(k[kLL - 1], s[kLL - 1]);
    } else {
      ++n;
    }
    // The new record at position n - 1, then one bubble pass upwards.
#pragma unroll
    for (int i = 0; i < kLL; ++i)
      if (i == n - 1) k[i] = xk, s[i] = xs;
#pragma unroll
    for (int i = kLL - 1; i > 0; --i)
      if (i < n && ks_bef(k[i], s[i], k[i - 1], s[i - 1])) {
        const i64 tk = k[i], ts = s[i];
        k[i] = k[i - 1], s[i] = s[i - 1];
        k[i - 1] = tk, s[i - 1] = ts;
      }
  }
};

// Shared memory of tk_lane_rank for blocks of up to NT threads.
template <int NT>
struct LaneRankSmem {
  i64 hk[NT], hs[NT];              // the threads' list heads
  i64 ck[kLL * 32], cs[kLL * 32];  // the records not after the threshold
  i64 thk, ths, kk, ks;            // the threshold, the K-th result
  int nh, nc, found;
};

// The block's top K (K <= 32) from its threads' lists T: thr = the K-th best
// of the lists' heads.  At least K records are then not after thr, so every
// record of the result is not after it: only those (at most kLL from each of
// the K lists whose head is not after thr) are ranked, among themselves.
// Writes the first min(K, their number) to out_k / out_s in order and
// returns that number, or -1 (block-uniform) when the result may be
// incomplete: a thread dropped a record that is not after the K-th result,
// or repeated records left more than kLL * 32 candidates.  Every thread of
// the block calls it.
template <int NT>
__device__ __forceinline__ int tk_lane_rank(const LaneTop& T, int K, LaneRankSmem<NT>& m,
                                            i64* out_k, i64* out_s) {
  constexpr int kCap = kLL * 32;
  if (threadIdx.x == 0) m.nh = 0, m.nc = 0, m.found = 0;
  __syncthreads();
  int h = -1;
  if (T.n) {
    h = atomicAdd(&m.nh, 1);
    m.hk[h] = T.k[0], m.hs[h] = T.s[0];
  }
  __syncthreads();
  if (T.n && rank_among(m.hk, m.hs, m.nh, T.k[0], T.s[0], h) == K - 1)
    m.thk = T.k[0], m.ths = T.s[0], m.found = 1;
  __syncthreads();
  const bool every = m.found == 0;
  const i64 thk = m.thk, ths = m.ths;
#pragma unroll
  for (int i = 0; i < kLL; ++i)
    if (i < T.n && (every || !ks_bef(thk, ths, T.k[i], T.s[i]))) {
      const int c = atomicAdd(&m.nc, 1);
      if (c < kCap) m.ck[c] = T.k[i], m.cs[c] = T.s[i];
    }
  __syncthreads();
  const int nc = m.nc;
  if (nc > kCap) return -1;  // block-uniform
  const int nres = min(K, nc);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const i64 xk = m.ck[c], xs = m.cs[c];
    const int r = rank_among(m.ck, m.cs, nc, xk, xs, c);
    if (r < K) out_k[r] = xk, out_s[r] = xs;
    if (r == K - 1) m.kk = xk, m.ks = xs;
  }
  __syncthreads();
  const bool bad = T.dv && !(nres == K && ks_bef(m.kk, m.ks, T.dk, T.ds));
  return __syncthreads_or(bad) ? -1 : nres;
}

// Merge the per-warp lists of one block into warp 0's list through shared
// memory (`sk`, `ss`: nwarps * K entries, `sc`: nwarps counts).  K <= 32: a
// tree (warp w takes the list of warp w + d at distance d = 1, 2, 4, ...,
// one bitonic merge of sorted lists per level); larger K: warp 0 offers the
// other lists' entries.
__device__ __forceinline__ void tk_block_merge(TopList& L, int K, i64* sk, i64* ss, int* sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (K <= 32) {
    for (int d = 1; d < nw; d <<= 1) {
      const bool give = warp % (2 * d) == d, take = warp % (2 * d) == 0 && warp + d < nw;
      if (give) {
        L.store(sk + warp * K, ss + warp * K);
        if (lane == 0) sc[warp] = L.cnt;
      }
      __syncthreads();
      if (take) {
        const int w = warp + d, c = sc[w];
        const bool v = lane < c;
        L.merge_list(K, c, v ? sk[w * K + lane] : 0, v ? ss[w * K + lane] : 0);
      }
      __syncthreads();
    }
    return;
  }
  if (warp > 0) {
    L.store(sk + warp * K, ss + warp * K);
    if (lane == 0) sc[warp] = L.cnt;
  }
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < nw; ++w) {
      const int c = sc[w];
      for (int j = 0; j < c; j += 32) {
        const bool v = j + lane < c;
        const i64 k = v ? sk[w * K + j + lane] : 0, s = v ? ss[w * K + j + lane] : 0;
        L.offer(K, v, k, s);
      }
    }
  }
  __syncthreads();
}


// Merge the lists of all nw warps of the block into warp 0's list: every
// warp stores its list in shared memory (sk, ss: nw * K entries, sc: nw
// counts), then warp 0 offers all stored entries, 32 per call.
__device__ __forceinline__ void tk_block_merge_all(TopList& L, int K, i64* sk, i64* ss, int* sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (K <= 32) {
    tk_block_merge(L, K, sk, ss, sc);
    return;
  }
  L.store(sk + warp * K, ss + warp * K);
  if (lane == 0) sc[warp] = L.cnt;
  __syncthreads();
  if (warp == 0) {
    L.clear();
    const int total = nw * K;
    for (int j = 0; j < total; j += 32) {
      const int e = j + lane;
      const int p = e / K;
      const bool v = e < total && e - p * K < sc[p];
      L.offer(K, v, v ? sk[e] : 0, v ? ss[e] : 0);
    }
  }
  __syncthreads();
}

}  // namespace pqk
