// pq_ops.cu -- standalone operators: filter, radix partition, hash-join
// build/probe, group-by SUM, top-k.
#include <algorithm>
#include <mutex>

#include "pq_internal.h"
#include "pq_topk.cuh"

using namespace pqk;
using pqh::S;

namespace {

// ============================================================== filter ====
// Tile of 4096 elements: 8 warps x 512; lane l of warp w reads elements
// w*512 + g*128 + 4l + {0..3} for g = 0..3 (row order = element order), so a
// warp-wide load instruction covers 512 contiguous bytes of an int32 column.
constexpr int kFilterTile = 4096;

template <typename T, bool VEC>
__device__ __forceinline__ void load4(const T* __restrict__ col, i64 e0, i64 n, i64 v[4]) {
  if (VEC && e0 + 4 <= n) {
    if constexpr (sizeof(T) == 4) {
      int4 q = ld_stream(reinterpret_cast<const int4*>(col + e0));
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else if constexpr (sizeof(T) == 8) {
      longlong2 a = ld_stream(reinterpret_cast<const longlong2*>(col + e0));
      longlong2 b = ld_stream(reinterpret_cast<const longlong2*>(col + e0 + 2));
      v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else {
      char4 q = ld_stream(reinterpret_cast<const char4*>(col + e0));
      v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) v[s] = e0 + s < n ? (i64)ld_stream(col + e0 + s) : 0;
  }
}

template <typename T, bool SEL, bool VEC>
__global__ void __launch_bounds__(256) k_filter(const T* __restrict__ col,
                                                const i64* __restrict__ sel_in, i64 n_cap,
                                                const i64* d_n, Pred p, i64* __restrict__ out,
                                                i64* d_count, u64* state, u32* tile_ctr,
                                                i64 spin_limit, DevStatus* st) {
  __shared__ i64 s_tile;
  __shared__ u32 s_w[8];
  __shared__ i64 s_prefix;
  const i64 n = d_n ? min(*d_n, n_cap) : n_cap;
  const i64 ntiles = (n + kFilterTile - 1) / kFilterTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const i64 tile = s_tile;
    if (tile >= ntiles) break;
    const i64 wbase = tile * kFilterTile + warp * 512;
    u32 bits = 0;
    i64 rows[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const i64 e0 = wbase + g * 128 + lane * 4;
      i64 v[4];
      if (SEL) {
        i64 r[4];
        load4<i64, VEC>(sel_in, e0, n, r);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          rows[g * 4 + s] = r[s];
          v[s] = e0 + s < n ? (i64)__ldg(col + r[s]) : 0;
        }
      } else {
        load4<T, VEC>(col, e0, n, v);
#pragma unroll
        for (int s = 0; s < 4; ++s) rows[g * 4 + s] = e0 + s;
      }
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (e0 + s < n && pass(p, v[s])) bits |= 1u << (g * 4 + s);
    }
    // Per-group counts packed in 16-bit fields: one warp scan covers 4 groups.
    u64 packed = 0;
#pragma unroll
    for (int g = 0; g < 4; ++g) packed |= (u64)__popc((bits >> (4 * g)) & 0xFu) << (16 * g);
    u64 incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const u64 wt = __shfl_sync(kFull, incl, 31);
    const u64 excl = incl - packed;
    if (lane == 0)
      s_w[warp] = (u32)((wt & 0xFFFF) + ((wt >> 16) & 0xFFFF) + ((wt >> 32) & 0xFFFF) + (wt >> 48));
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      u32 c = lane < nw ? s_w[lane] : 0, x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      const u32 total = __shfl_sync(kFull, x, 31);
      const i64 prefix = lookback_prefix(state, tile, total, spin_limit, st);
      if (lane < nw) s_w[lane] = x - c;
      if (lane == 0) {
        s_prefix = prefix;
        if (tile == ntiles - 1) *d_count = prefix + total;
      }
    }
    __syncthreads();
    i64 pos = s_prefix + s_w[warp];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const u32 bg = (bits >> (4 * g)) & 0xFu;
      i64 at = pos + (i64)((excl >> (16 * g)) & 0xFFFF);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (bg & (1u << s)) {
          if (at < n_cap) out[at] = rows[g * 4 + s];
          ++at;
        }
      pos += (i64)((wt >> (16 * g)) & 0xFFFF);
    }
    __syncthreads();
  }
}

__global__ void k_fill(i64* __restrict__ p, i64 n, i64 v) {
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

// =========================================================== partition ====
// 8192 rows per tile; warp w owns rows w*1024 .. w*1024+1023 of the tile and
// walks them in 32 steps of 32 rows, so ranks assigned in step order keep the
// input order inside every bucket.
constexpr int kPartTile = 8192;

template <typename T>
__global__ void __launch_bounds__(256) k_part_hist(const T* __restrict__ key, i64 n, int log2P,
                                                   u32* __restrict__ hist, i64 ntiles) {
  extern __shared__ u32 sh[];
  const int P = 1 << log2P;
  for (int b = threadIdx.x; b < P; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const i64 tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 base = tile * kPartTile + warp * 1024;
  for (int s = 0; s < 32; ++s) {
    const i64 r = base + s * 32 + lane;
    const bool valid = r < n;
    const u32 b = valid ? fib_bucket((i64)__ldg(key + r), log2P) : 0xFFFFFFFFu;
    const u32 peers = __match_any_sync(kFull, b);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&sh[b], (u32)__popc(peers));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < P; b += blockDim.x) hist[(i64)b * ntiles + tile] = sh[b];
}

// Exclusive scan of a u32 array into i64 (single pass, decoupled look-back).
__global__ void __launch_bounds__(256) k_scan_u32(const u32* __restrict__ in, i64 n,
                                                  i64* __restrict__ out, u64* state,
                                                  u32* tile_ctr, i64 spin_limit, DevStatus* st) {
  __shared__ i64 s_tile;
  __shared__ i64 s_w[8];
  __shared__ i64 s_prefix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 ntiles = (n + 4095) / 4096;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const i64 tile = s_tile;
    if (tile >= ntiles) break;
    const i64 e0 = tile * 4096 + threadIdx.x * 16;
    u32 v[16];
    i64 sum = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      v[j] = e0 + j < n ? in[e0 + j] : 0u;
      sum += v[j];
    }
    i64 x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      i64 y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      i64 c = lane < nw ? s_w[lane] : 0, y = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        i64 z = __shfl_up_sync(kFull, y, o);
        if (lane >= o) y += z;
      }
      const i64 total = __shfl_sync(kFull, y, 31);
      const i64 prefix = lookback_prefix(state, tile, total, spin_limit, st);
      if (lane < nw) s_w[lane] = y - c;
      if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    i64 run = s_prefix + s_w[warp] + (x - sum);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (e0 + j < n) out[e0 + j] = run;
      run += v[j];
    }
    __syncthreads();
  }
}

struct PayArgs {
  const void* src[PQ_MAX_PAYLOAD];
  void* dst[PQ_MAX_PAYLOAD];
  int type[PQ_MAX_PAYLOAD];
  int n;
};

__device__ __forceinline__ void copy_elem(int type, const void* src, void* dst, i64 from, i64 to) {
  if (type == PQ_INT64) ((i64*)dst)[to] = __ldg((const i64*)src + from);
  else if (type == PQ_INT32) ((int*)dst)[to] = __ldg((const int*)src + from);
  else ((signed char*)dst)[to] = __ldg((const signed char*)src + from);
}

template <typename T>
__global__ void __launch_bounds__(256) k_part_scatter(const T* __restrict__ key, i64 n, int log2P,
                                                      const i64* __restrict__ gofs, i64 ntiles,
                                                      PayArgs pa, T* __restrict__ out_key,
                                                      i64* d_offsets) {
  extern __shared__ u32 wc[];  // [8][P]: per-warp counts, then per-warp bases
  const int P = 1 << log2P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = threadIdx.x; b < nw * P; b += blockDim.x) wc[b] = 0;
  __syncthreads();
  const i64 tile = blockIdx.x;
  const i64 base = tile * kPartTile + warp * 1024;
  for (int s = 0; s < 32; ++s) {
    const i64 r = base + s * 32 + lane;
    const bool valid = r < n;
    const u32 b = valid ? fib_bucket((i64)__ldg(key + r), log2P) : 0xFFFFFFFFu;
    const u32 peers = __match_any_sync(kFull, b);
    if (valid && lane == __ffs(peers) - 1) wc[warp * P + b] += (u32)__popc(peers);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < P; b += blockDim.x) {
    u32 run = 0;
    for (int w = 0; w < nw; ++w) {
      const u32 c = wc[w * P + b];
      wc[w * P + b] = run;
      run += c;
    }
    if (tile == 0) d_offsets[b] = gofs[(i64)b * ntiles];
  }
  if (tile == 0 && threadIdx.x == 0) d_offsets[P] = n;
  __syncthreads();
  for (int s = 0; s < 32; ++s) {
    const i64 r = base + s * 32 + lane;
    const bool valid = r < n;
    const T k = valid ? __ldg(key + r) : T(0);
    const u32 b = valid ? fib_bucket((i64)k, log2P) : 0xFFFFFFFFu;
    const u32 peers = __match_any_sync(kFull, b);
    if (valid) {
      const i64 pos = __ldg(gofs + (i64)b * ntiles + tile) + wc[warp * P + b] +
                      __popc(peers & lanemask_lt());
      if (pos >= n) continue;  // only after a timed-out scan; never in a correct run
      out_key[pos] = k;
      for (int j = 0; j < pa.n; ++j) copy_elem(pa.type[j], pa.src[j], pa.dst[j], r, pos);
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wc[warp * P + b] += (u32)__popc(peers);
    __syncwarp();
  }
}

// ========================================================== hash join ====
template <typename TK, typename TV>
__global__ void k_ht_build(const TK* __restrict__ key, const TV* __restrict__ val, i64 n,
                           i64* __restrict__ keys, i64* __restrict__ vals, int log2cap, i64* meta,
                           DevStatus* st) {
  const u64 mask = (1ULL << log2cap) - 1;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const i64 k = (i64)__ldg(key + i);
    if (k == kEmpty) {
      latch(st, PQ_ERR_RESERVED_KEY, i);
      continue;
    }
    const i64 v = val ? (i64)__ldg(val + i) : i;
    u64 s = slot_hash(k) & mask;
    u64 probes = 0;
    for (; probes <= mask; ++probes) {
      const i64 old = (i64)atomicCAS((u64*)&keys[s], (u64)kEmpty, (u64)k);
      if (old == kEmpty) {
        vals[s] = v;
        break;
      }
      if (old == k) meta[0] = 1;
      s = (s + 1) & mask;
    }
    if (probes > mask) latch(st, PQ_ERR_CAPACITY, i);
  }
}

template <typename TK>
__global__ void k_ht_probe(const TK* __restrict__ pkey, i64 n, const i64* __restrict__ keys,
                           const i64* __restrict__ vals, int log2cap, const i64* meta,
                           i64* __restrict__ out_row, i64* __restrict__ out_val, i64 cap,
                           u64* d_count) {
  const u64 mask = (1ULL << log2cap) - 1;
  const bool dup = meta[0] != 0;
  const int lane = threadIdx.x & 31;
  const i64 gw = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nwarps = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 wb = gw * 32; wb < n; wb += nwarps * 32) {
    const i64 i = wb + lane;
    bool active = i < n;
    const i64 k = active ? (i64)__ldg(pkey + i) : 0;
    if (k == kEmpty) active = false;
    u64 s = slot_hash(k) & mask;
    while (__any_sync(kFull, active)) {
      bool emit = false;
      i64 v = 0;
      if (active) {
        const i64 kk = __ldg(keys + s);
        if (kk == kEmpty) {
          active = false;
        } else {
          if (kk == k) {
            emit = true;
            v = __ldg(vals + s);
            if (!dup) active = false;
          }
          s = (s + 1) & mask;
        }
      }
      const u64 pos = warp_reserve(d_count, emit ? 1u : 0u);
      if (emit && pos < (u64)cap) {
        out_row[pos] = i;
        out_val[pos] = v;
      }
    }
  }
}

__global__ void k_check_cap(const i64* d_count, i64 cap, DevStatus* st) {
  if (*d_count > cap) latch(st, PQ_ERR_CAPACITY, *d_count);
}

// ============================================================= group-by ====
template <typename TK, typename TV>
__global__ void k_gb_insert(const TK* __restrict__ key, const TV* __restrict__ val, i64 n,
                            i64* __restrict__ keys, i64* __restrict__ sums, int log2cap,
                            DevStatus* st) {
  const u64 mask = (1ULL << log2cap) - 1;
  const int lane = threadIdx.x & 31;
  const i64 gw = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nwarps = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 wb = gw * 32; wb < n; wb += nwarps * 32) {
    const i64 i = wb + lane;
    bool active = i < n;
    i64 k = active ? (i64)__ldg(key + i) : kEmpty;
    i64 v = active ? (i64)__ldg(val + i) : 0;
    if (active && k == kEmpty) {
      latch(st, PQ_ERR_RESERVED_KEY, i);
      active = false;
    }
    // Warp pre-aggregation: one atomic per distinct key per warp (hot keys).
    const u32 peers = __match_any_sync(kFull, (u64)(active ? k : kEmpty));
    if (__any_sync(kFull, __popc(peers) > 1)) {
      i64 agg = 0;
      for (int src = 0; src < 32; ++src) {
        const i64 x = __shfl_sync(kFull, v, src);
        if ((peers >> src) & 1u) agg += x;
      }
      v = agg;
    }
    if (!active || lane != __ffs(peers) - 1) continue;
    u64 s = slot_hash(k) & mask;
    u64 probes = 0;
    for (; probes <= mask; ++probes) {
      i64 cur = *(volatile i64*)&keys[s];
      if (cur == kEmpty) cur = (i64)atomicCAS((u64*)&keys[s], (u64)kEmpty, (u64)k);
      if (cur == kEmpty || cur == k) break;
      s = (s + 1) & mask;
    }
    if (probes > mask) {
      latch(st, PQ_ERR_CAPACITY, -1);
      continue;
    }
    atomicAdd((u64*)&sums[s], (u64)v);
  }
}

__global__ void k_gb_emit(const i64* __restrict__ keys, const i64* __restrict__ sums, i64 slots,
                          i64* __restrict__ out_keys, i64* __restrict__ out_sums, i64 cap,
                          u64* d_ngroups) {
  const int lane = threadIdx.x & 31;
  const i64 gw = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nwarps = ((i64)gridDim.x * blockDim.x) >> 5;
  (void)lane;
  for (i64 wb = gw * 32; wb < slots; wb += nwarps * 32) {
    const i64 s = wb + (threadIdx.x & 31);
    const bool has = s < slots && keys[s] != kEmpty;
    const u64 pos = warp_reserve(d_ngroups, has ? 1u : 0u);
    if (has && pos < (u64)cap) {
      out_keys[pos] = keys[s];
      out_sums[pos] = sums[s];
    }
  }
}

// ================================================================ top-k ====
__global__ void __launch_bounds__(256) k_topk(const i64* __restrict__ keys,
                                              const i64* __restrict__ sums, i64 n_cap,
                                              const i64* d_n, int K, i64* part_k, i64* part_s,
                                              int* part_c, u32* ticket, i64* out_keys,
                                              i64* out_sums, i64* d_nout) {
  __shared__ i64 sk[8 * kMaxK], ss[8 * kMaxK];
  __shared__ int sc[8];
  __shared__ bool s_last;
  __shared__ i64 s_scr[8][64];
  chain_begin();
  const i64 n = d_n ? min(*d_n, n_cap) : n_cap;
  // Only the first nb blocks take pairs (at least 2048 each), so that a
  // small count read on the device leaves few lists to merge.
  const int nb = (int)max((i64)1, min((i64)gridDim.x, (n + 2047) / 2048));
  const i64 per = (n + nb - 1) / nb;
  const i64 lo = min(n, per * blockIdx.x), hi = min(n, lo + per);
  TopList L;
  L.bind(s_scr[threadIdx.x >> 5]);
  L.clear();
  for (i64 b = lo; b < hi; b += blockDim.x) {
    const i64 i = b + threadIdx.x;
    const bool v = i < hi;
    L.offer(K, v, v ? keys[i] : 0, v ? sums[i] : 0);
  }
  tk_block_merge(L, K, sk, ss, sc);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    L.store(part_k + (i64)blockIdx.x * K, part_s + (i64)blockIdx.x * K);
    if (lane == 0) part_c[blockIdx.x] = L.cnt;
    __threadfence();
    u32 t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1u);
    t = __shfl_sync(kFull, t, 0);
    if (lane == 0) s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  // The last block merges the blocks' lists: each warp offers 32 entries
  // of the grid * K list slots per round; an entry, its slot's list count
  // and its value are independent loads (L2, not L1: other blocks wrote
  // them), so a round costs one memory latency.  Slots past a list's count
  // are in the buffer but unused.
  __threadfence();
  L.clear();
  const int total = nb * K;
  for (int base = (threadIdx.x >> 5) * 32; base < total; base += blockDim.x) {
    const int e = base + lane;
    bool v = false;
    i64 k = 0, s = 0;
    if (e < total) {
      const int b = e / K;
      const int c = __ldcg(part_c + b);
      k = __ldcg(part_k + e);
      s = __ldcg(part_s + e);
      v = e - b * K < c;
    }
    L.offer(K, v, k, s);
  }
  tk_block_merge(L, K, sk, ss, sc);
  if (threadIdx.x < 32) {
    L.store(out_keys, out_sums);
    if (lane == 0) *d_nout = L.cnt;
  }
}

template <typename T>
int filter_grid(pq_ctx* ctx, i64 n) {
  i64 tiles = (n + kFilterTile - 1) / kFilterTile;
  return (int)std::max<i64>(1, std::min<i64>(tiles, (i64)ctx->num_sms * 4));
}

template <typename T, bool SEL, bool VEC>
void launch_filter(pq_ctx* ctx, int grid, cudaStream_t s, const void* col, const i64* sel,
                   i64 n_cap, const i64* d_n, Pred p, i64* out, i64* d_count, u64* state,
                   u32* ctr) {
  k_filter<T, SEL, VEC><<<grid, 256, 0, s>>>((const T*)col, sel, n_cap, d_n, p, out, d_count,
                                             state, ctr, ctx->opt.spin_limit, ctx->d_status);
}

template <typename T, bool SEL>
void launch_filter_v(pq_ctx* ctx, bool vec, int grid, cudaStream_t s, const void* col,
                     const i64* sel, i64 n_cap, const i64* d_n, Pred p, i64* out, i64* d_count,
                     u64* state, u32* ctr) {
  if (vec) launch_filter<T, SEL, true>(ctx, grid, s, col, sel, n_cap, d_n, p, out, d_count, state, ctr);
  else launch_filter<T, SEL, false>(ctx, grid, s, col, sel, n_cap, d_n, p, out, d_count, state, ctr);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

namespace pqh {
namespace {
int topk_grid(pq_ctx* ctx, i64 n) {
  return (int)std::max<i64>(1, std::min<i64>((n + 2047) / 2048, (i64)ctx->num_sms * 2));
}
}  // namespace

size_t topk_scratch_bytes(pq_ctx* ctx, int64_t n, int k) {
  const int grid = topk_grid(ctx, n);
  return (size_t)grid * k * 16 + (size_t)grid * 4;
}

cudaError_t topk_launch(pq_ctx* ctx, const int64_t* keys, const int64_t* sums, int64_t n,
                        const int64_t* d_n, int k, int64_t* out_keys, int64_t* out_sums,
                        int64_t* d_nout, unsigned* ticket, void* lists, bool chained,
                        cudaStream_t s) {
  const int grid = topk_grid(ctx, n);
  i64* pk = (i64*)lists;
  i64* ps = pk + (i64)grid * k;
  int* pc = (int*)(ps + (i64)grid * k);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chained ? 1 : 0;
  ctx->launches++;
  return cudaLaunchKernelEx(&cfg, k_topk, (const i64*)keys, (const i64*)sums, (i64)n,
                            (const i64*)d_n, k, pk, ps, pc, (u32*)ticket, (i64*)out_keys,
                            (i64*)out_sums, (i64*)d_nout);
}

pq_status fill_i64(pq_ctx* ctx, i64* p, int64_t n, i64 v, cudaStream_t s) {
  if (n <= 0) return PQ_OK;
  int grid = (int)std::min<i64>((n + 255) / 256, (i64)ctx->num_sms * 8);
  k_fill<<<grid, 256, 0, s>>>(p, n, v);
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}
}  // namespace pqh

#define PQ_DISPATCH_T(type, T, ...)              \
  switch (type) {                                \
    case PQ_INT8: { typedef signed char T; __VA_ARGS__; break; } \
    case PQ_INT32: { typedef int T; __VA_ARGS__; break; }        \
    default: { typedef long long T; __VA_ARGS__; break; }        \
  }

extern "C" {

pq_status pq_filter(pq_ctx* ctx, pq_col col, int op, int64_t c, const int64_t* sel_in,
                    int64_t n_in, const int64_t* d_n_in, int64_t* sel_out, int64_t* d_count,
                    void* stream) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  bool ok;
  Pred p = pqh::make_pred(op, c, &ok);
  if (!ok || !pqh::valid_dtype(col.type) || col.n < 0 || !d_count || col.reserved != 0)
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_filter: bad arguments");
  const bool sel = sel_in != nullptr;
  const i64 n_cap = sel ? n_in : col.n;
  if (n_cap < 0 || (n_cap > 0 && (!sel_out || (!col.data && col.n > 0))))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_filter: bad arguments");
  if (d_n_in && !sel) return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_filter: d_n_in needs sel_in");
  cudaStream_t s = S(stream);
  PQ_CUDA(ctx, cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
  if (n_cap == 0) return PQ_OK;
  const i64 ntiles = (n_cap + kFilterTile - 1) / kFilterTile;
  pqh::Scratch scr(ctx, s);
  char* w = (char*)scr.get(ntiles * 8 + 256);
  if (!w) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_filter: no scratch");
  u64* state = (u64*)(w + 256);
  u32* ctr = (u32*)w;
  PQ_CUDA(ctx, cudaMemsetAsync(w, 0, ntiles * 8 + 256, s));
  const bool vec = sel ? aligned16(sel_in) : aligned16(col.data);
  const int grid = filter_grid<int>(ctx, n_cap);
  PQ_DISPATCH_T(col.type, T, {
    if (sel)
      launch_filter_v<T, true>(ctx, vec, grid, s, col.data, (const i64*)sel_in, n_cap,
                               (const i64*)d_n_in, p, (i64*)sel_out, (i64*)d_count, state, ctr);
    else
      launch_filter_v<T, false>(ctx, vec, grid, s, col.data, nullptr, n_cap, nullptr, p,
                                (i64*)sel_out, (i64*)d_count, state, ctr);
  });
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}

pq_status pq_partition(pq_ctx* ctx, pq_col key, const pq_col* payload, int npay, int log2P,
                       void* out_key, void* const* out_payload, int64_t* d_offsets,
                       void* stream) {
  if (!ctx) return PQ_ERR_INVALID_ARG;
  if (log2P < 0 || log2P > PQ_MAX_LOG2P || npay < 0 || npay > PQ_MAX_PAYLOAD || !d_offsets ||
      (key.type != PQ_INT32 && key.type != PQ_INT64) || key.n < 0 || key.reserved != 0 ||
      (npay > 0 && (!payload || !out_payload)))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_partition: bad arguments");
  PayArgs pa{};
  pa.n = npay;
  for (int j = 0; j < npay; ++j) {
    if (!pqh::valid_dtype(payload[j].type) || payload[j].n != key.n ||
        (key.n && (!payload[j].data || !out_payload[j])))
      return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_partition: payload %d", j);
    pa.src[j] = payload[j].data;
    pa.dst[j] = out_payload[j];
    pa.type[j] = payload[j].type;
  }
  cudaStream_t s = S(stream);
  const i64 n = key.n;
  const int P = 1 << log2P;
  if (n == 0) {
    PQ_CUDA(ctx, cudaMemsetAsync(d_offsets, 0, (P + 1) * sizeof(int64_t), s));
    return PQ_OK;
  }
  if (!key.data || !out_key) return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_partition: null key");
  const i64 ntiles = (n + kPartTile - 1) / kPartTile;
  const i64 m = ntiles * P;
  const i64 stiles = (m + 4095) / 4096;
  pqh::Scratch scr(ctx, s);
  u32* hist = (u32*)scr.get(m * 4);
  i64* gofs = (i64*)scr.get(m * 8);
  char* w = (char*)scr.get(stiles * 8 + 256);
  if (!hist || !gofs || !w) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_partition: no scratch");
  PQ_CUDA(ctx, cudaMemsetAsync(w, 0, stiles * 8 + 256, s));
  const size_t smem_hist = (size_t)P * 4, smem_scatter = (size_t)8 * P * 4;
  PQ_DISPATCH_T(key.type, T, {
    if (smem_scatter > 48 * 1024)
      cudaFuncSetAttribute(k_part_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_scatter);
    k_part_hist<T><<<(unsigned)ntiles, 256, smem_hist, s>>>((const T*)key.data, n, log2P, hist,
                                                            ntiles);
    PQ_LAUNCHED(ctx);
    k_scan_u32<<<(unsigned)std::min<i64>(stiles, (i64)ctx->num_sms * 4), 256, 0, s>>>(
        hist, m, gofs, (u64*)(w + 256), (u32*)w, ctx->opt.spin_limit, ctx->d_status);
    PQ_LAUNCHED(ctx);
    k_part_scatter<T><<<(unsigned)ntiles, 256, smem_scatter, s>>>(
        (const T*)key.data, n, log2P, gofs, ntiles, pa, (T*)out_key, (i64*)d_offsets);
  });
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}

pq_status pq_join_build(pq_ctx* ctx, pq_col key, pq_col val, float load_factor, pq_ht** out,
                        void* stream) {
  if (!ctx || !out) return PQ_ERR_INVALID_ARG;
  *out = nullptr;
  if (load_factor <= 0) load_factor = ctx->opt.load_factor;
  if (!pqh::valid_dtype(key.type) || key.n < 0 || (key.n && !key.data) || load_factor < 0.05f ||
      load_factor > 0.9f || (val.data && (!pqh::valid_dtype(val.type) || val.n != key.n)))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_join_build: bad arguments");
  cudaStream_t s = S(stream);
  const int lf = (int)(load_factor * 1024 + 0.5f);
  const int log2cap = cap_log2(key.n, lf);
  const i64 cap = (i64)1 << log2cap;
  auto* ht = new pq_ht();
  ht->block = ctx->arena.alloc((size_t)cap * 16 + 256);
  if (!ht->block) {
    delete ht;
    return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_join_build: table of %lld slots", (long long)cap);
  }
  ht->meta = (i64*)ht->block;
  ht->keys = (i64*)((char*)ht->block + 256);
  ht->vals = ht->keys + cap;
  ht->log2cap = log2cap;
  ht->n = key.n;
  pq_status st = pqh::fill_i64(ctx, ht->keys, cap, kEmpty, s);
  if (st == PQ_OK && cudaMemsetAsync(ht->meta, 0, 256, s) != cudaSuccess)
    st = pqh::fail(ctx, PQ_ERR_CUDA, "memset");
  if (st == PQ_OK && key.n > 0) {
    const int grid = (int)std::min<i64>((key.n + 255) / 256, (i64)ctx->num_sms * 8);
    PQ_DISPATCH_T(key.type, TK, {
      if (!val.data) {
        k_ht_build<TK, long long><<<grid, 256, 0, s>>>((const TK*)key.data, nullptr, key.n,
                                                       ht->keys, ht->vals, log2cap, ht->meta,
                                                       ctx->d_status);
      } else {
        PQ_DISPATCH_T(val.type, TV, {
          k_ht_build<TK, TV><<<grid, 256, 0, s>>>((const TK*)key.data, (const TV*)val.data,
                                                  key.n, ht->keys, ht->vals, log2cap, ht->meta,
                                                  ctx->d_status);
        });
      }
    });
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) st = pqh::fail(ctx, PQ_ERR_CUDA, "k_ht_build launch");
  }
  if (st != PQ_OK) {
    ctx->arena.release(ht->block, s);
    delete ht;
    return st;
  }
  *out = ht;
  return PQ_OK;
}

pq_status pq_join_probe(pq_ctx* ctx, const pq_ht* ht, pq_col probe_key, int64_t* out_probe_row,
                        int64_t* out_build_val, int64_t cap, int64_t* d_count, void* stream) {
  if (!ctx || !ht || !d_count || cap < 0 || !pqh::valid_dtype(probe_key.type) ||
      probe_key.n < 0 || (probe_key.n && !probe_key.data) ||
      (cap > 0 && (!out_probe_row || !out_build_val)))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_join_probe: bad arguments");
  cudaStream_t s = S(stream);
  PQ_CUDA(ctx, cudaMemsetAsync(d_count, 0, sizeof(int64_t), s));
  if (probe_key.n == 0) return PQ_OK;
  const int grid = (int)std::min<i64>((probe_key.n + 255) / 256, (i64)ctx->num_sms * 8);
  PQ_DISPATCH_T(probe_key.type, TK, {
    k_ht_probe<TK><<<grid, 256, 0, s>>>((const TK*)probe_key.data, probe_key.n, ht->keys,
                                        ht->vals, ht->log2cap, ht->meta, (i64*)out_probe_row,
                                        (i64*)out_build_val, cap, (u64*)d_count);
  });
  PQ_LAUNCHED(ctx);
  k_check_cap<<<1, 1, 0, s>>>((const i64*)d_count, cap, ctx->d_status);
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}

pq_status pq_groupby_sum(pq_ctx* ctx, pq_col key, pq_col val, int64_t* out_keys,
                         int64_t* out_sums, int64_t cap, int64_t* d_ngroups, void* stream) {
  if (!ctx || !d_ngroups || cap < 0 || !pqh::valid_dtype(key.type) || !pqh::valid_dtype(val.type) ||
      key.n < 0 || val.n != key.n || (key.n && (!key.data || !val.data)) ||
      (cap > 0 && (!out_keys || !out_sums)))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_groupby_sum: bad arguments");
  cudaStream_t s = S(stream);
  PQ_CUDA(ctx, cudaMemsetAsync(d_ngroups, 0, sizeof(int64_t), s));
  if (key.n == 0) return PQ_OK;
  const int lf = (int)(ctx->opt.load_factor * 1024 + 0.5f);
  const int log2cap = cap_log2(std::min<i64>(key.n, std::max<i64>(cap, 1)), lf);
  const i64 slots = (i64)1 << log2cap;
  pqh::Scratch scr(ctx, s);
  i64* keys = (i64*)scr.get((size_t)slots * 16);
  if (!keys) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_groupby_sum: table of %lld slots",
                              (long long)slots);
  i64* sums = keys + slots;
  pq_status st = pqh::fill_i64(ctx, keys, slots, kEmpty, s);
  if (st != PQ_OK) return st;
  PQ_CUDA(ctx, cudaMemsetAsync(sums, 0, slots * 8, s));
  const int grid = (int)std::min<i64>((key.n + 255) / 256, (i64)ctx->num_sms * 8);
  PQ_DISPATCH_T(key.type, TK, {
    PQ_DISPATCH_T(val.type, TV, {
      k_gb_insert<TK, TV><<<grid, 256, 0, s>>>((const TK*)key.data, (const TV*)val.data, key.n,
                                               keys, sums, log2cap, ctx->d_status);
    });
  });
  PQ_LAUNCHED(ctx);
  const int grid2 = (int)std::min<i64>((slots + 255) / 256, (i64)ctx->num_sms * 8);
  k_gb_emit<<<grid2, 256, 0, s>>>(keys, sums, slots, (i64*)out_keys, (i64*)out_sums, cap,
                                   (u64*)d_ngroups);
  PQ_LAUNCHED(ctx);
  k_check_cap<<<1, 1, 0, s>>>((const i64*)d_ngroups, cap, ctx->d_status);
  PQ_LAUNCHED(ctx);
  return PQ_OK;
}

pq_status pq_topk(pq_ctx* ctx, const int64_t* keys, const int64_t* sums, int64_t n,
                  const int64_t* d_n, int k, int64_t* out_keys, int64_t* out_sums,
                  int64_t* d_nout, void* stream) {
  if (!ctx || k < 1 || k > PQ_MAX_K || n < 0 || !d_nout || !out_keys || !out_sums ||
      (n > 0 && (!keys || !sums)))
    return pqh::fail(ctx, PQ_ERR_INVALID_ARG, "pq_topk: bad arguments");
  cudaStream_t s = S(stream);
  PQ_CUDA(ctx, cudaMemsetAsync(d_nout, 0, sizeof(int64_t), s));
  if (n == 0) return PQ_OK;
  pqh::Scratch scr(ctx, s);
  char* w = (char*)scr.get(pqh::topk_scratch_bytes(ctx, n, k) + 256);
  if (!w) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_topk: no scratch");
  PQ_CUDA(ctx, cudaMemsetAsync(w, 0, 256, s));
  PQ_CUDA(ctx, pqh::topk_launch(ctx, keys, sums, n, d_n, k, out_keys, out_sums, d_nout,
                                (unsigned*)w, w + 256, false, s));
  return PQ_OK;
}

}  // extern "C"

// ===================================================== allocation-free filter ====
// pq_filter needs scratch for its single-pass tile prefixes, normally carved
// from the context's arena.  Some callers cannot allocate device memory at all
// (for example code that runs while a CUDA graph is being captured, or inside
// a runtime that owns every allocation and forbids others), and they may not
// have a context either.  For them the same kernel runs with its scratch in
// this file-scope device array: a fixed 1 MiB of tile states plus a small
// header, which every GPU that loads the library keeps until the process
// exits.  All calls share the array, so calls that overlap on the GPU race;
// each call clears the part it uses before its kernel runs.
namespace {

constexpr i64 kNoAllocTiles = 1 << 17;                  // 131072 tiles
constexpr i64 kNoAllocRows = kNoAllocTiles * kFilterTile;  // 536,870,912 rows
constexpr int kNoAllocHeader = 32;                      // words: ticket, status

__device__ __align__(256) u64 g_noalloc_scratch[kNoAllocHeader + kNoAllocTiles];

struct NoAllocDevice {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  u64* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
};
NoAllocDevice g_noalloc_dev[256];

// Per-device set-up, run once with that device current: the host cannot use
// the array's name as a device address, so it asks the runtime for it.
cudaError_t noalloc_setup(int dev, NoAllocDevice** out) {
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  NoAllocDevice& d = g_noalloc_dev[dev];
  std::call_once(d.once, [&d, dev] {
    d.err = cudaGetSymbolAddress((void**)&d.scratch, g_noalloc_scratch);
    if (d.err == cudaSuccess)
      d.err = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  });
  *out = &d;
  return d.err;
}

}  // namespace

extern "C" pq_status pq_filter_noalloc(pq_col col, int op, int64_t c, const int64_t* sel_in,
                                       int64_t n_in, int64_t* sel_out, int64_t* d_count,
                                       int32_t* d_error, void* stream) {
  bool ok;
  Pred p = pqh::make_pred(op, c, &ok);
  if (!ok || !pqh::valid_dtype(col.type) || col.n < 0 || !d_count || col.reserved != 0)
    return PQ_ERR_INVALID_ARG;
  const bool sel = sel_in != nullptr;
  const i64 n_cap = sel ? n_in : col.n;
  if (n_cap < 0 || (n_cap > 0 && (!sel_out || (!col.data && col.n > 0))))
    return PQ_ERR_INVALID_ARG;
  if (n_cap > kNoAllocRows) return PQ_ERR_CAPACITY;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PQ_ERR_CUDA;
  NoAllocDevice* d = nullptr;
  if (noalloc_setup(dev, &d) != cudaSuccess) return PQ_ERR_CUDA;
  cudaStream_t s = S(stream);
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), s) != cudaSuccess) return PQ_ERR_CUDA;
  if (d_error && cudaMemsetAsync(d_error, 0, sizeof(int32_t), s) != cudaSuccess)
    return PQ_ERR_CUDA;
  if (n_cap == 0) return PQ_OK;
  const i64 ntiles = (n_cap + kFilterTile - 1) / kFilterTile;
  u64* hdr = d->scratch;
  if (cudaMemsetAsync(hdr, 0, (kNoAllocHeader + ntiles) * sizeof(u64), s) != cudaSuccess)
    return PQ_ERR_CUDA;
  u32* ticket = (u32*)hdr;
  DevStatus* status = (DevStatus*)(hdr + 2);
  u64* state = hdr + kNoAllocHeader;
  const bool vec = sel ? aligned16(sel_in) : aligned16(col.data);
  const int grid = (int)std::max<i64>(1, std::min<i64>(ntiles, (i64)d->sms * 4));
  const i64 spin = 1ll << 22;
  PQ_DISPATCH_T(col.type, T, {
    if (sel) {
      if (vec)
        k_filter<T, true, true><<<grid, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in,
                                                     n_cap, nullptr, p, (i64*)sel_out,
                                                     (i64*)d_count, state, ticket, spin, status);
      else
        k_filter<T, true, false><<<grid, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in,
                                                      n_cap, nullptr, p, (i64*)sel_out,
                                                      (i64*)d_count, state, ticket, spin, status);
    } else {
      if (vec)
        k_filter<T, false, true><<<grid, 256, 0, s>>>((const T*)col.data, nullptr, n_cap,
                                                      nullptr, p, (i64*)sel_out, (i64*)d_count,
                                                      state, ticket, spin, status);
      else
        k_filter<T, false, false><<<grid, 256, 0, s>>>((const T*)col.data, nullptr, n_cap,
                                                       nullptr, p, (i64*)sel_out, (i64*)d_count,
                                                       state, ticket, spin, status);
    }
  });
  if (cudaGetLastError() != cudaSuccess) return PQ_ERR_CUDA;
  if (d_error &&
      cudaMemcpyAsync(d_error, &status->code, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return PQ_ERR_CUDA;
  return PQ_OK;
}
