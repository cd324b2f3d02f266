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

// Large inputs: two passes with no chain between tiles.  Pass 1 counts the
// passing rows of every kFilterTile tile (tiles spread over the grid, all
// loads independent); a scan of the counts gives each tile's offset; pass 2
// reads the column again and writes each tile's rows at its offset.  The
// column is read twice, but no tile waits for another.
template <typename T, bool SEL, bool VEC>
__device__ __forceinline__ u32 filter_tile_bits(const T* __restrict__ col,
                                                const i64* __restrict__ sel_in, i64 n, Pred p,
                                                i64 tile, i64 (&rows)[16]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 wbase = tile * kFilterTile + warp * 512;
  i64 v[16];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const i64 e0 = wbase + g * 128 + lane * 4;
    if (SEL) {
      i64 r[4];
      load4<i64, VEC>(sel_in, e0, n, r);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        rows[g * 4 + s] = r[s];
        v[g * 4 + s] = e0 + s < n ? (i64)__ldg(col + r[s]) : 0;
      }
    } else {
      i64 x[4];
      load4<T, VEC>(col, e0, n, x);
#pragma unroll
      for (int s = 0; s < 4; ++s) v[g * 4 + s] = x[s], rows[g * 4 + s] = e0 + s;
    }
  }
  u32 bits = 0;
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (wbase + g * 128 + lane * 4 + s < n && pass(p, v[g * 4 + s])) bits |= 1u << (g * 4 + s);
  return bits;
}

template <typename T, bool SEL, bool VEC>
__global__ void __launch_bounds__(256) k_filter_count(const T* __restrict__ col,
                                                      const i64* __restrict__ sel_in, i64 n_cap,
                                                      const i64* d_n, Pred p, u32* counts) {
  __shared__ u32 s_w[8];
  const i64 n = d_n ? min(*d_n, n_cap) : n_cap;
  const i64 ntiles = (n + kFilterTile - 1) / kFilterTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (i64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    i64 rows[16];
    const u32 bits = filter_tile_bits<T, SEL, VEC>(col, sel_in, n, p, tile, rows);
    const u32 c = __reduce_add_sync(kFull, (u32)__popc(bits));
    if (lane == 0) s_w[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
      counts[tile] = t;
    }
    __syncthreads();
  }
}

template <typename T, bool SEL, bool VEC>
__global__ void __launch_bounds__(256) k_filter_write(const T* __restrict__ col,
                                                      const i64* __restrict__ sel_in, i64 n_cap,
                                                      const i64* d_n, Pred p,
                                                      const i64* __restrict__ offs,
                                                      const u32* __restrict__ counts,
                                                      i64* __restrict__ out, i64* d_count) {
  __shared__ u32 s_w[8];
  const i64 n = d_n ? min(*d_n, n_cap) : n_cap;
  const i64 ntiles = (n + kFilterTile - 1) / kFilterTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (i64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    i64 rows[16];
    const i64 toff = __ldg(offs + tile);
    const u32 bits = filter_tile_bits<T, SEL, VEC>(col, sel_in, n, p, tile, rows);
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
    i64 pos = toff;
    for (int w = 0; w < warp; ++w) pos += s_w[w];
    if (tile == ntiles - 1 && threadIdx.x == 0) *d_count = toff + __ldg(counts + tile);
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

// ------------------------------------------------- staged partition ----
// For fan-outs up to 2^kStagedMaxLog2: persistent blocks, block k taking the
// contiguous rows [k * n / G, (k + 1) * n / G).  The histogram is then one
// count per (bucket, block), so the scan and the per-bucket cursor reads are
// small.  Each block walks its rows in sub-tiles of kSub: warp w takes rows
// w * kSubWarpRows .. of the sub-tile in steps of 32, which fixes every
// row's place in the sub-tile sorted by (bucket, input order); each
// column is then staged in shared memory in that order and every bucket's
// run is written with consecutive threads on consecutive rows.  Within a
// bucket the order is input order: blocks in block order, sub-tiles in
// order, warps in order, steps in order, lanes in order.
constexpr int kStagedMaxLog2 = 10;
constexpr int kSub = 2048;
constexpr int kSubWarpRows = kSub / 8;     // rows of a warp in a sub-tile
constexpr int kSubSteps = kSubWarpRows / 32;

// Lanes of the warp whose bucket equals this lane's, from one ballot per
// bucket bit (all lanes taking part): cheaper than a general match for small
// bucket ids.  nbits = log2P when every lane holds a row; otherwise
// log2P + 1, an invalid lane passing a bucket of its own, 2^log2P.
__device__ __forceinline__ u32 bucket_peers(u32 b, int nbits) {
  u32 peers = kFull;
#pragma unroll
  for (int k = 0; k <= kStagedMaxLog2; ++k) {
    if (k >= nbits) break;  // warp-uniform
    const u32 m = __ballot_sync(kFull, (b >> k) & 1u);
    peers &= (b >> k) & 1u ? m : ~m;
  }
  return peers;
}

// First row of block k's chunk: a multiple of 16 rows (so that every column's
// slice starts on a 16-byte boundary for the bulk copies), n for k = g.
__host__ __device__ inline i64 chunk_begin(i64 n, i64 g, i64 k) {
  if (k >= g) return n;
  const i64 r = (i64)((__int128)n * k / g + 15) & ~(i64)15;
  return r < n ? r : n;
}

// Histogram of the scatter's chunks: hsplit blocks per chunk (chunk k =
// blockIdx.x / hsplit), each counting a share of the chunk's rows and adding
// its counts into hist[b * g + k] (zeroed before).
template <typename T>
__global__ void __launch_bounds__(256, 8) k_part_hist_blk(const T* __restrict__ key, i64 n,
                                                          int log2P, u32* __restrict__ hist,
                                                          i64 g, int hsplit) {
  extern __shared__ u32 sh[];
  const int P = 1 << log2P;
  for (int b = threadIdx.x; b < P; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const i64 k = blockIdx.x / hsplit, h = blockIdx.x % hsplit;
  const i64 c0 = chunk_begin(n, g, k), c1 = chunk_begin(n, g, k + 1);
  auto cut = [&](i64 x) { return x >= hsplit ? c1 : min(c1, c0 + (((c1 - c0) * x / hsplit + 15) & ~15LL)); };
  const i64 r0 = cut(h), r1 = cut(h + 1);  // 16-row aligned shares
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerVec = 16 / sizeof(T);    // keys per 16-byte load
  constexpr int kLd = 4;                     // 16-byte loads per lane per step
  constexpr int kRows = kLd * 32 * kPerVec;  // rows of a warp step
  // Whole warp steps (kRows consecutive rows: kLd loads of 16 bytes per
  // lane, issued together, then counted with no bounds tests) while the
  // share's start is 16-byte aligned; the rest row by row.
  const bool vec = ((uintptr_t)(key + r0) & 15) == 0;
  const i64 steps = vec ? (r1 - r0) / kRows : 0;
  for (i64 st = warp; st < steps; st += 8) {  // warp-uniform
    const uint4* p = reinterpret_cast<const uint4*>(key + r0 + st * kRows);
    uint4 x[kLd];
#pragma unroll
    for (int j = 0; j < kLd; ++j) x[j] = __ldcs(p + j * 32 + lane);
#pragma unroll
    for (int j = 0; j < kLd; ++j) {
      T v[kPerVec];
      memcpy(v, &x[j], 16);
#pragma unroll
      for (int e = 0; e < kPerVec; ++e) atomicAdd(&sh[fib_bucket((i64)v[e], log2P)], 1u);
    }
  }
  for (i64 i = r0 + steps * kRows + threadIdx.x; i < r1; i += blockDim.x)
    atomicAdd(&sh[fib_bucket((i64)__ldg(key + i), log2P)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < P; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[(i64)b * g + k], sh[b]);
}

// Shared memory of the staged scatter for P buckets (bytes).
__host__ __device__ inline size_t staged_smem(int P) {
  return (size_t)P * 8        // s_gb: global cursor per bucket
         + (size_t)8 * P * 4  // s_cnt: per-warp counts, then per-warp offsets
         + (size_t)P * 4      // s_run: run start of each bucket in the sub-tile
         + (size_t)P * 4      // s_tot: the sub-tile's rows per bucket
         + (size_t)kSub * 8   // s_stage: one column of the sub-tile, sorted
         + (size_t)kSub * 2   // s_lpos: sorted place of each row
         + (size_t)kSub * 2;  // s_sbk: bucket of each sorted place
}

// One column of a sub-tile: each thread issues its 16 loads before it uses
// any of them, places the values in sorted order in shared memory, then
// writes sorted places i = thread, thread + 256, ... to their runs.
template <typename V>
__device__ __forceinline__ void stage_column(const V* __restrict__ src, V* __restrict__ dst,
                                             i64 r, int cnt, const unsigned short* s_lpos,
                                             const unsigned short* s_sbk, const u32* s_run,
                                             const i64* s_gb, V* s_stage) {
  constexpr int kPer = kSub / 256;
  V v[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = j * 256 + (int)threadIdx.x;
    v[j] = i < cnt ? __ldcs(src + r + i) : V(0);
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = j * 256 + (int)threadIdx.x;
    if (i < cnt) s_stage[s_lpos[i]] = v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = j * 256 + (int)threadIdx.x;
    if (i < cnt) {
      const u32 b = s_sbk[i];
      __stcs(dst + s_gb[b] + (i - (i64)s_run[b]), s_stage[i]);
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_part_scatter_blk(const T* __restrict__ key, i64 n,
                                                          int log2P, const i64* __restrict__ gofs,
                                                          PayArgs pa, T* __restrict__ out_key,
                                                          i64* d_offsets) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int P = 1 << log2P;
  i64* s_gb = reinterpret_cast<i64*>(smem);
  u32* s_cnt = reinterpret_cast<u32*>(s_gb + P);
  u32* s_run = s_cnt + 8 * P;
  u32* s_tot = s_run + P;
  u64* s_stage = reinterpret_cast<u64*>(s_tot + P);
  unsigned short* s_lpos = reinterpret_cast<unsigned short*>(s_stage + kSub);
  unsigned short* s_sbk = s_lpos + kSub;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 g = gridDim.x, k = blockIdx.x;
  const i64 r0 = chunk_begin(n, g, k), r1 = chunk_begin(n, g, k + 1);
  for (int b = threadIdx.x; b < P; b += blockDim.x) {
    s_gb[b] = gofs[(i64)b * g + k];
    if (k == 0) d_offsets[b] = s_gb[b];
  }
  if (k == 0 && threadIdx.x == 0) d_offsets[P] = n;
  for (i64 r = r0; r < r1; r += kSub) {
    const int cnt = (int)min((i64)kSub, r1 - r);
    for (int b = threadIdx.x; b < 8 * P; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    // Bucket and place within the warp's rows of each of the lane's rows
    // (the keys loaded first, so that their loads are in flight together).
    const int nbits = cnt == kSub ? log2P : log2P + 1;  // every lane holds a row?
    u32 bp[kSubSteps];  // bucket << 9 | place among the warp's rows of that bucket
#pragma unroll
    for (int st = 0; st < kSubSteps; ++st) {
      const int i = warp * kSubWarpRows + st * 32 + lane;
      bp[st] = i < cnt ? fib_bucket((i64)__ldg(key + r + i), log2P) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int st = 0; st < kSubSteps; ++st) {
      const bool valid = bp[st] != 0xFFFFFFFFu;
      const u32 b = bp[st];
      const u32 peers = bucket_peers(valid ? b : (1u << log2P), nbits);
      u32 place = 0;
      if (valid) place = s_cnt[warp * P + b] + __popc(peers & lanemask_lt());
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) s_cnt[warp * P + b] += (u32)__popc(peers);
      __syncwarp();
      bp[st] = valid ? b << 9 | place : 0xFFFFFFFFu;
    }
    __syncthreads();
    static_assert(kSubWarpRows <= 512, "place takes 9 bits");
    // Per bucket: offsets of the warps' rows, the sub-tile's total.
    for (int b = threadIdx.x; b < P; b += blockDim.x) {
      u32 run = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 c = s_cnt[w * P + b];
        s_cnt[w * P + b] = run;
        run += c;
      }
      s_tot[b] = run;
    }
    __syncthreads();
    {  // run starts: exclusive scan of the totals (P <= 4 * 256)
      static_assert((1 << kStagedMaxLog2) <= 4 * 256, "four buckets per thread");
      u32 v[4], sum = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = (int)threadIdx.x * 4 + j;
        v[j] = b < P ? s_tot[b] : 0u;
        sum += v[j];
      }
      u32 run = block_exclusive_sum(sum);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = (int)threadIdx.x * 4 + j;
        if (b < P) s_run[b] = run;
        run += v[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int st = 0; st < kSubSteps; ++st) {
      if (bp[st] == 0xFFFFFFFFu) continue;
      const u32 b = bp[st] >> 9;
      const int i = warp * kSubWarpRows + st * 32 + lane;
      const u32 at = s_run[b] + s_cnt[warp * P + b] + (bp[st] & 511u);
      s_lpos[i] = (unsigned short)at;
      s_sbk[at] = (unsigned short)b;
    }
    __syncthreads();
    stage_column<T>(key, out_key, r, cnt, s_lpos, s_sbk, s_run, s_gb,
                    reinterpret_cast<T*>(s_stage));
    for (int j = 0; j < pa.n; ++j) {
      if (pa.type[j] == PQ_INT64)
        stage_column<i64>((const i64*)pa.src[j], (i64*)pa.dst[j], r, cnt, s_lpos, s_sbk, s_run,
                          s_gb, reinterpret_cast<i64*>(s_stage));
      else if (pa.type[j] == PQ_INT32)
        stage_column<int>((const int*)pa.src[j], (int*)pa.dst[j], r, cnt, s_lpos, s_sbk, s_run,
                          s_gb, reinterpret_cast<int*>(s_stage));
      else
        stage_column<signed char>((const signed char*)pa.src[j], (signed char*)pa.dst[j], r, cnt,
                                  s_lpos, s_sbk, s_run, s_gb,
                                  reinterpret_cast<signed char*>(s_stage));
    }
    for (int b = threadIdx.x; b < P; b += blockDim.x) s_gb[b] += s_tot[b];
    __syncthreads();
  }
}

// The staged scatter with its sub-tiles brought into shared memory by bulk
// copies (TMA), double-buffered: while the block orders and writes sub-tile
// j, the copies of sub-tile j + 1 are in flight.  The columns of a sub-tile
// sit one after another in its buffer (kSub elements each, raw row order);
// after the places are fixed, s_inv[i] holds the row of sorted place i, and
// each column is written by gathering through it.  Used when every column
// is 16-byte aligned and the buffers fit in shared memory.
struct TmaCols {
  const void* src[1 + PQ_MAX_PAYLOAD];
  void* dst[1 + PQ_MAX_PAYLOAD];
  int es[1 + PQ_MAX_PAYLOAD];   // element bytes
  int off[1 + PQ_MAX_PAYLOAD];  // byte offset of the column in a buffer
  int n;                        // columns, the key first
  int buf_bytes;                // bytes of one buffer
};

// SUB: rows of a sub-tile (2048, or 4096 where many buckets would leave
// runs of about two rows per bucket and sub-tile).
__host__ __device__ inline size_t tma_smem(int P, int buf_bytes, int sub) {
  return 16                          // two mbarriers
         + 2 * (size_t)buf_bytes     // double-buffered sub-tile
         + (size_t)P * 8             // s_gb
         + (size_t)8 * P * 2         // s_cnt (u16: at most sub / 8 per warp)
         + (size_t)P * 2 * 2         // s_run, s_tot (u16)
         + (size_t)sub * 2 * 2;      // s_inv, s_sbk
}

// One column of a sub-tile of SUB rows, written in sorted order: sorted
// place i = j * 256 + thread takes the buffered row src[j] to output row
// drow[j] (both worked out once for all columns).
template <typename V, int SUB>
__device__ __forceinline__ void gather_column(const char* buf, int off, V* __restrict__ dst,
                                              int cnt, const unsigned short* src,
                                              const i64* drow) {
  const V* col = reinterpret_cast<const V*>(buf + off);
  constexpr int kPer = SUB / 256;
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    if (j * 256 + (int)threadIdx.x < cnt) __stcs(dst + drow[j], col[src[j]]);
}

template <typename T, int SUB>
__global__ void __launch_bounds__(256) k_part_scatter_tma(i64 n, int log2P,
                                                          const i64* __restrict__ gofs,
                                                          TmaCols tc, i64* d_offsets,
                                                          i64 spin_limit, DevStatus* st) {
  constexpr int kWRows = SUB / 8;  // rows of a warp in a sub-tile
  constexpr int kSteps = kWRows / 32;
  static_assert(kWRows <= 512, "place takes 9 bits");
  extern __shared__ __align__(16) unsigned char smem[];
  const int P = 1 << log2P;
  u64* bar = reinterpret_cast<u64*>(smem);
  char* bufs = reinterpret_cast<char*>(smem + 16);
  i64* s_gb = reinterpret_cast<i64*>(bufs + 2 * (size_t)tc.buf_bytes);
  unsigned short* s_cnt = reinterpret_cast<unsigned short*>(s_gb + P);
  unsigned short* s_run = s_cnt + 8 * P;
  unsigned short* s_tot = s_run + P;
  unsigned short* s_inv = s_tot + P;
  unsigned short* s_sbk = s_inv + SUB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 g = gridDim.x, k = blockIdx.x;
  const i64 r0 = chunk_begin(n, g, k), r1 = chunk_begin(n, g, k + 1);
  const i64 nsub = (r1 - r0 + SUB - 1) / SUB;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  for (int b = threadIdx.x; b < P; b += blockDim.x) {
    s_gb[b] = gofs[(i64)b * g + k];
    if (k == 0) d_offsets[b] = s_gb[b];
  }
  if (k == 0 && threadIdx.x == 0) d_offsets[P] = n;
  __syncthreads();
  // Thread 0 starts the copies of sub-tile j into buffer j & 1: the part of
  // each column slice that is a whole number of 16-byte units (all of it but
  // possibly the last sub-tile's tail, which the block loads itself).
  auto issue = [&](i64 j) {
    if (threadIdx.x != 0 || j >= nsub) return;
    const i64 r = r0 + j * SUB;
    const i64 cnt = min((i64)SUB, r1 - r);
    char* buf = bufs + (j & 1) * (size_t)tc.buf_bytes;
    u32 total = 0;
    for (int c = 0; c < tc.n; ++c) total += (u32)((cnt * tc.es[c]) & ~15LL);
    mbar_expect_tx(&bar[j & 1], total);
    for (int c = 0; c < tc.n; ++c) {
      const u32 bytes = (u32)((cnt * tc.es[c]) & ~15LL);
      if (bytes)
        bulk_g2s(buf + tc.off[c], static_cast<const char*>(tc.src[c]) + r * tc.es[c], bytes,
                 &bar[j & 1]);
    }
  };
  issue(0);
  issue(1);
  for (i64 j = 0; j < nsub; ++j) {
    const i64 r = r0 + j * SUB;
    const int cnt = (int)min((i64)SUB, r1 - r);
    char* buf = bufs + (j & 1) * (size_t)tc.buf_bytes;
    const bool arrived = mbar_wait(&bar[j & 1], (u32)((j >> 1) & 1), spin_limit);
    if (__syncthreads_or(!arrived)) {  // block-uniform
      // The copies did not complete: report, give them a second bounded wait
      // (they write this block's shared memory) and stop.
      if (threadIdx.x == 0) latch(st, PQ_ERR_TIMEOUT, r);
      mbar_wait(&bar[j & 1], (u32)((j >> 1) & 1), spin_limit);
      if (j + 1 < nsub) mbar_wait(&bar[(j + 1) & 1], (u32)(((j + 1) >> 1) & 1), spin_limit);
      return;
    }
    // The tail that is not a whole 16-byte unit (last sub-tile only).
    for (int c = 0; cnt < SUB && c < tc.n; ++c) {
      const int es = tc.es[c];
      const int done = (int)(((i64)cnt * es) & ~15LL) / es;
      for (int i = done + (int)threadIdx.x; i < cnt; i += blockDim.x) {
        const char* src = static_cast<const char*>(tc.src[c]) + (r + i) * es;
        char* d = buf + tc.off[c] + (size_t)i * es;
        if (es == 8) *reinterpret_cast<i64*>(d) = *reinterpret_cast<const i64*>(src);
        else if (es == 4) *reinterpret_cast<int*>(d) = *reinterpret_cast<const int*>(src);
        else *d = *src;
      }
    }
    for (int b = threadIdx.x; b < 8 * P; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    const T* s_key = reinterpret_cast<const T*>(buf + tc.off[0]);
    const int nbits = cnt == SUB ? log2P : log2P + 1;  // every lane holds a row?
    u32 bp[kSteps];  // bucket << 9 | place among the warp's rows of that bucket
#pragma unroll
    for (int q = 0; q < kSteps; ++q) {
      const int i = warp * kWRows + q * 32 + lane;
      bp[q] = i < cnt ? fib_bucket((i64)s_key[i], log2P) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int q = 0; q < kSteps; ++q) {
      const bool valid = bp[q] != 0xFFFFFFFFu;
      const u32 b = bp[q];
      const u32 peers = bucket_peers(valid ? b : (1u << log2P), nbits);
      u32 place = 0;
      if (valid) place = s_cnt[warp * P + b] + __popc(peers & lanemask_lt());
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1)
        s_cnt[warp * P + b] = (unsigned short)(s_cnt[warp * P + b] + __popc(peers));
      __syncwarp();
      bp[q] = valid ? b << 9 | place : 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < P; b += blockDim.x) {
      u32 run = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const u32 c = s_cnt[w * P + b];
        s_cnt[w * P + b] = (unsigned short)run;
        run += c;
      }
      s_tot[b] = (unsigned short)run;
    }
    __syncthreads();
    {
      u32 v[4], sum = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = (int)threadIdx.x * 4 + q;
        v[q] = b < P ? s_tot[b] : 0u;
        sum += v[q];
      }
      u32 run = block_exclusive_sum(sum);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = (int)threadIdx.x * 4 + q;
        if (b < P) s_run[b] = (unsigned short)run;
        run += v[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSteps; ++q) {
      if (bp[q] == 0xFFFFFFFFu) continue;
      const u32 b = bp[q] >> 9;
      const int i = warp * kWRows + q * 32 + lane;
      const u32 at = s_run[b] + s_cnt[warp * P + b] + (bp[q] & 511u);
      s_inv[at] = (unsigned short)i;
      s_sbk[at] = (unsigned short)b;
    }
    __syncthreads();
    // This thread's sorted places: their rows in the buffer and output rows.
    constexpr int kPer = SUB / 256;
    unsigned short src[kPer];
    i64 drow[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = q * 256 + (int)threadIdx.x;
      src[q] = 0, drow[q] = 0;
      if (i < cnt) {
        const u32 b = s_sbk[i];
        src[q] = s_inv[i];
        drow[q] = s_gb[b] + (i - (i64)s_run[b]);
      }
    }
    for (int c = 0; c < tc.n; ++c) {
      if (tc.es[c] == 8)
        gather_column<i64, SUB>(buf, tc.off[c], static_cast<i64*>(tc.dst[c]), cnt, src, drow);
      else if (tc.es[c] == 4)
        gather_column<int, SUB>(buf, tc.off[c], static_cast<int*>(tc.dst[c]), cnt, src, drow);
      else
        gather_column<signed char, SUB>(buf, tc.off[c], static_cast<signed char*>(tc.dst[c]), cnt,
                                   src, drow);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < P; b += blockDim.x) s_gb[b] += s_tot[b];
    // Every thread's reads of this buffer are done: the next copies into it
    // may start (ordered after the reads for the copy engine).
    fence_proxy_async_smem();
    __syncthreads();
    issue(j + 2);
  }
}

// ========================================================== hash join ====
// The join's hash table: 2^log2cap slots of 16 bytes, {key, value} side by
// side, so that an insert and a match each touch one sector.
template <typename TK, typename TV>
__global__ void k_ht_build(const TK* __restrict__ key, const TV* __restrict__ val, i64 n,
                           i64* __restrict__ slots, int log2cap, i64* meta, DevStatus* st) {
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
      const i64 old = (i64)atomicCAS((u64*)&slots[2 * s], (u64)kEmpty, (u64)k);
      if (old == kEmpty) {
        slots[2 * s + 1] = v;
        break;
      }
      if (old == k) meta[0] = 1;
      s = (s + 1) & mask;
    }
    if (probes > mask) latch(st, PQ_ERR_CAPACITY, i);
  }
}

// Hash-join probe: a warp probes 64 rows at a time, two per lane, whose
// chains of loads (key, then slot after slot of linear probing, every
// matching build row when the build keys repeat) run side by side.  The
// warp stages its matches in shared memory and writes them out kPrbBuf at a
// time, reserving each run with one atomic on the output counter: one
// reservation per pair-producing round would make that counter the bound
// (millions of atomics on one address).  Blocks of 8 warps, one resident
// wave.
constexpr int kPrbBuf = 256;
template <typename TK>
__global__ void __launch_bounds__(256) k_ht_probe(const TK* __restrict__ pkey, i64 n,
                                                  const longlong2* __restrict__ slots, int log2cap,
                                                  const i64* meta, i64* __restrict__ out_row,
                                                  i64* __restrict__ out_val, i64 cap,
                                                  u64* d_count) {
  __shared__ i64 s_row[8][kPrbBuf], s_val[8][kPrbBuf];
  const u64 mask = (1ULL << log2cap) - 1;
  const bool dup = meta[0] != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  i64* br = s_row[warp];
  i64* bv = s_val[warp];
  u32 nb = 0;  // staged pairs (warp-uniform)
  auto flush = [&]() {
    __syncwarp();
    u64 base = 0;
    if (lane == 0) base = atomicAdd(d_count, (u64)nb);
    base = __shfl_sync(kFull, base, 0);
    for (u32 e = lane; e < nb; e += 32) {
      const u64 pos = base + e;
      if (pos < (u64)cap) out_row[pos] = br[e], out_val[pos] = bv[e];
    }
    __syncwarp();
    nb = 0;
  };
  const i64 gw = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nwarps = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 wb = gw * 64; wb < n; wb += nwarps * 64) {
    i64 i[2], k[2];
    bool active[2];
    u64 s[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      i[h] = wb + h * 32 + lane;
      active[h] = i[h] < n;
      k[h] = active[h] ? (i64)__ldg(pkey + i[h]) : 0;
      if (k[h] == kEmpty) active[h] = false;
      s[h] = slot_hash(k[h]) & mask;
    }
    while (__any_sync(kFull, active[0] || active[1])) {
      longlong2 kv[2];  // {key, value} of each row's current slot
#pragma unroll
      for (int h = 0; h < 2; ++h) kv[h] = active[h] ? __ldg(slots + s[h]) : make_longlong2(kEmpty, 0);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        bool emit = false;
        i64 v = 0;
        if (active[h]) {
          if (kv[h].x == kEmpty) {
            active[h] = false;
          } else {
            if (kv[h].x == k[h]) {
              emit = true;
              v = kv[h].y;
              if (!dup) active[h] = false;
            }
            s[h] = (s[h] + 1) & mask;
          }
        }
        const u32 m = __ballot_sync(kFull, emit);
        if (emit) {
          const u32 at = nb + __popc(m & lanemask_lt());
          br[at] = i[h], bv[at] = v;
        }
        nb += __popc(m);
      }
      if (nb > kPrbBuf - 64) flush();  // room for a full round stays
    }
  }
  if (nb) flush();
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

// Dense keys (a key range of at most 4 rows per key): the group of key k is
// slot k - min, its sum in a zeroed array and its existence in a bitmap, so
// a group costs one reduction and one bit, at addresses that follow the key
// order.  The key range is measured first (k_gb_range).
__device__ __forceinline__ u64 gb_ukey(i64 k) { return (u64)k ^ 0x8000000000000000ULL; }

template <typename TK>
__global__ void __launch_bounds__(256) k_gb_range(const TK* __restrict__ key, i64 n, u64* rng) {
  u64 lo = ~0ULL, hi = 0;
  const i64 stride = (i64)gridDim.x * blockDim.x * 4;
  for (i64 i0 = ((i64)blockIdx.x * blockDim.x + threadIdx.x) * 4; i0 < n; i0 += stride) {
    i64 k[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? (i64)__ldg(key + i0 + j) : (i64)__ldg(key + i0);
#pragma unroll
    for (int j = 0; j < 4; ++j) lo = min(lo, gb_ukey(k[j])), hi = max(hi, gb_ukey(k[j]));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, (u64)__shfl_xor_sync(kFull, lo, o));
    hi = max(hi, (u64)__shfl_xor_sync(kFull, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(reinterpret_cast<unsigned long long*>(rng), (unsigned long long)lo);
    atomicMax(reinterpret_cast<unsigned long long*>(rng + 1), (unsigned long long)hi);
  }
}

// Each lane takes 4 consecutive rows of a 128-row warp step; runs of equal
// keys are summed by a segmented scan over the lanes and each run adds its
// total to its slot once (sorted or clustered keys: one reduction per group
// and step).  The reserved key is reported as for the hash table.
template <typename TK, typename TV>
__global__ void __launch_bounds__(256) k_gb_dense(const TK* __restrict__ key,
                                                  const TV* __restrict__ val, i64 n, u64 umin,
                                                  i64* __restrict__ sums, u32* __restrict__ bm,
                                                  DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const i64 gw = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const i64 nw = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 wb = gw * 128; wb < n; wb += nw * 128) {
    const i64 r0 = wb + 4 * lane;
    u64 idx[4];
    i64 v[4];
    u32 ok = 0;  // bit j: row j exists and its key is not the reserved one
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool in = r0 + j < n;
      const i64 k = in ? (i64)__ldg(key + r0 + j) : kEmpty;
      v[j] = in ? (i64)__ldg(val + r0 + j) : 0;
      if (in && k == kEmpty) latch(st, PQ_ERR_RESERVED_KEY, r0 + j);
      ok |= (in && k != kEmpty ? 1u : 0u) << j;
      idx[j] = gb_ukey(k) - umin;
    }
    // Runs: a row starts one when its key differs from the row before it
    // (or it is not a group row); lane 0's first row always does.
    const u64 prev = __shfl_up_sync(kFull, idx[3], 1);
    const u32 okp = __shfl_up_sync(kFull, ok, 1);
    u32 head = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool pj = j ? ((ok >> (j - 1)) & 1u) : (lane ? (okp >> 3) & 1u : 0u);
      const u64 pk = j ? idx[j - 1] : prev;
      const bool oj = (ok >> j) & 1u;
      head |= (!oj || !pj || idx[j] != pk || (j == 0 && lane == 0) ? 1u : 0u) << j;
    }
    // The lane's last run, summed back to the lane where it starts.
    i64 ls = 0;
    u32 fl = 0;  // bit 0: the run starts in this lane
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if ((head >> j) & 1u) ls = 0, fl = 1;
      ls += v[j];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (__all_sync(kFull, fl & 1u)) break;
      const i64 us = __shfl_up_sync(kFull, ls, o);
      const u32 uf = __shfl_up_sync(kFull, fl, o);
      if (lane >= o) {
        if (!(fl & 1u)) ls += us;
        fl |= uf & 1u;
      }
    }
    const i64 in_s = __shfl_up_sync(kFull, ls, 1);
    const bool next_head = __shfl_down_sync(kFull, head & 1u, 1);
    i64 acc = (head & 1u) ? 0 : in_s;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j > 0 && ((head >> j) & 1u)) acc = 0;
      acc += v[j];
      const bool end = j < 3 ? (head >> (j + 1)) & 1u : (lane == 31 || next_head);
      if (end && ((ok >> j) & 1u)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(sums + idx[j]), (unsigned long long)acc);
        atomicOr(bm + (idx[j] >> 5), 1u << (idx[j] & 31));
      }
    }
  }
}

// Positions for a block's outputs, cnt per thread: one atomic on the
// output counter per block step (a block-wide scan of the counts), so that
// the counter is not a point of contention.  Every thread of the block
// calls it; returns this thread's first position.
__device__ __forceinline__ u64 block_reserve(u64* counter, u32 cnt) {
  __shared__ u64 s_base;
  const u32 before = block_exclusive_sum(cnt);
  if (threadIdx.x == blockDim.x - 1) s_base = atomicAdd(counter, (u64)(before + cnt));
  __syncthreads();
  const u64 pos = s_base + before;
  __syncthreads();  // s_base is read before the next call writes it
  return pos;
}

// The groups of the dense slot array, from its existence bitmap, in key
// order within each block step: a thread reserves the positions of one
// bitmap word's groups (one atomic per block step), then the warp writes
// its 32 words one after another, lane l taking bit l, so that the sums are
// read and the groups written in contiguous runs.
__global__ void __launch_bounds__(256) k_gb_dense_emit(const u32* __restrict__ bm,
                                                       const i64* __restrict__ sums, u64 span,
                                                       u64 umin, i64* __restrict__ out_keys,
                                                       i64* __restrict__ out_sums, i64 cap,
                                                       u64* d_ngroups) {
  const i64 words = (i64)((span + 31) / 32);
  const i64 stride = (i64)gridDim.x * blockDim.x;
  for (i64 w0 = (i64)blockIdx.x * blockDim.x; w0 < words; w0 += stride) {  // block-uniform
    const i64 w = w0 + threadIdx.x;
    const u32 bits = w < words ? __ldg(bm + w) : 0u;
    const u64 pos = block_reserve(d_ngroups, (u32)__popc(bits));
    const int lane = threadIdx.x & 31;
    const i64 wfirst = w - lane;
    for (int c = 0; c < 32; ++c) {
      const u32 wc = __shfl_sync(kFull, bits, c);
      const u64 pc = __shfl_sync(kFull, pos, c);
      if (!((wc >> lane) & 1u)) continue;
      const u64 p = pc + __popc(wc & lanemask_lt());
      const u64 idx = (u64)(wfirst + c) * 32 + (u64)lane;
      if (p < (u64)cap) {
        out_keys[p] = (i64)((umin + idx) ^ 0x8000000000000000ULL);
        out_sums[p] = __ldg(sums + idx);
      }
    }
  }
}

// The groups of the hash table: a thread takes kGbEmitPer consecutive slots
// and writes their groups at consecutive positions reserved per block step.
constexpr int kGbEmitPer = 8;
__global__ void __launch_bounds__(256) k_gb_emit(const i64* __restrict__ keys,
                                                 const i64* __restrict__ sums, i64 slots,
                                                 i64* __restrict__ out_keys,
                                                 i64* __restrict__ out_sums, i64 cap,
                                                 u64* d_ngroups) {
  const i64 step = (i64)gridDim.x * blockDim.x * kGbEmitPer;
  for (i64 b0 = (i64)blockIdx.x * blockDim.x * kGbEmitPer; b0 < slots; b0 += step) {  // block-uniform
    const i64 b = b0 + (i64)threadIdx.x * kGbEmitPer;
    i64 k[kGbEmitPer];
    u32 m = 0;
#pragma unroll
    for (int j = 0; j < kGbEmitPer; ++j) {
      k[j] = b + j < slots ? keys[b + j] : kEmpty;
      m |= (u32)(k[j] != kEmpty) << j;
    }
    u64 pos = block_reserve(d_ngroups, (u32)__popc(m));
#pragma unroll
    for (int j = 0; j < kGbEmitPer; ++j)
      if ((m >> j) & 1u) {
        if (pos < (u64)cap) out_keys[pos] = k[j], out_sums[pos] = sums[b + j];
        ++pos;
      }
  }
}

// ================================================================ top-k ====
__global__ void __launch_bounds__(256, 2) k_topk(const i64* __restrict__ keys,
                                              const i64* __restrict__ sums, i64 n_cap,
                                              const i64* d_n, int K, i64* part_k, i64* part_s,
                                              int* part_c, u32* ticket, i64* out_keys,
                                              i64* out_sums, i64* d_nout, const u64* rec_ctr,
                                              pq_result* rec) {
  __shared__ i64 sk[8 * kMaxK], ss[8 * kMaxK];
  __shared__ int sc[8];
  __shared__ bool s_last;
  __shared__ i64 s_scr[8][kTopScr];
  __shared__ LaneRankSmem<256> s_lr;
  chain_begin();
  const i64 n = d_n ? min(*d_n, n_cap) : n_cap;
  // Only the first nb blocks take pairs (at least 256 each: one per thread),
  // so that a small count read on the device leaves few lists to merge.
  const int nb = (int)max((i64)1, min((i64)gridDim.x, (n + 255) / 256));
  if ((int)blockIdx.x >= nb) return;  // no pairs: the nb blocks take the ticket
  const i64 per = (n + nb - 1) / nb;
  const i64 lo = min(n, per * blockIdx.x), hi = min(n, lo + per);
  const int lane = threadIdx.x & 31;
  // A single block writes the result itself; otherwise its list.
  i64* bk = nb == 1 ? out_keys : part_k + (i64)blockIdx.x * K;
  i64* bs = nb == 1 ? out_sums : part_s + (i64)blockIdx.x * K;
  // K <= 32: each thread keeps its best kLL pairs in registers and the
  // block ranks the few that can be in its top K (tk_lane_rank); when that
  // cannot vouch for its result, and for K > 32, the warps' register lists
  // are merged in shared memory (TopList).
  int cnt = -1;
  if (K <= 32) {
    // A first threshold: each thread's best of 4 of its pairs spread over
    // its share (a sorted input then gives a threshold near its end), and
    // thr = the K-th best of those.  At least K pairs are not after thr, so
    // a pair after it cannot be among the block's K best: only the others
    // enter the lists, which keeps the lanes of a warp on the same path.
    // Blocks with fewer than 8 pairs per thread skip it (block-uniform).
    bool filt = false;
    i64 thk = 0, ths = 0;
    if (hi - lo >= 8 * 256) {
      const i64 mine = hi - lo > (i64)threadIdx.x ? (hi - lo - threadIdx.x + 255) / 256 : 0;
      i64 hk = 0, hs = 0;
      bool hv = false;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const i64 j = mine * q / 4;
        if (j < mine) {
          const i64 xk = keys[lo + threadIdx.x + j * 256], xs = sums[lo + threadIdx.x + j * 256];
          if (!hv || ks_bef(xk, xs, hk, hs)) hk = xk, hs = xs, hv = true;
        }
      }
      if (threadIdx.x == 0) s_lr.nh = 0, s_lr.found = 0;
      __syncthreads();
      int h = -1;
      if (hv) {
        h = atomicAdd(&s_lr.nh, 1);
        s_lr.hk[h] = hk, s_lr.hs[h] = hs;
      }
      __syncthreads();
      if (hv && rank_among(s_lr.hk, s_lr.hs, s_lr.nh, hk, hs, h) == K - 1)
        s_lr.thk = hk, s_lr.ths = hs, s_lr.found = 1;
      __syncthreads();
      filt = s_lr.found != 0;
      thk = s_lr.thk, ths = s_lr.ths;
      __syncthreads();  // tk_lane_rank reuses s_lr
    }
    LaneTop T;
    T.clear();
    i64 i = lo + threadIdx.x;
    for (; i + 3 * 256 < hi; i += 4 * 256) {  // four pairs' loads in flight
      i64 k[4], s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k[u] = __ldcs(keys + i + u * 256), s[u] = __ldcs(sums + i + u * 256);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (!filt || !ks_bef(thk, ths, k[u], s[u])) T.insert(k[u], s[u]);
    }
    for (; i < hi; i += blockDim.x) {
      const i64 xk = keys[i], xs = sums[i];
      if (!filt || !ks_bef(thk, ths, xk, xs)) T.insert(xk, xs);
    }
    cnt = tk_lane_rank(T, K, s_lr, bk, bs);
  }
  TopList L;
  L.bind(s_scr[threadIdx.x >> 5]);
  if (cnt < 0) {
    L.clear();
    for (i64 b = lo; b < hi; b += blockDim.x) {
      const i64 i = b + threadIdx.x;
      const bool v = i < hi;
      L.offer(K, v, v ? keys[i] : 0, v ? sums[i] : 0);
    }
    tk_block_merge(L, K, sk, ss, sc);
    if (threadIdx.x < 32) {
      L.store(bk, bs);
      cnt = L.cnt;
    }
  }
  // Thread 0 holds the count on either path.
  if (nb == 1) {
    if (threadIdx.x == 0) *d_nout = cnt;
  } else {
    if (threadIdx.x == 0) part_c[blockIdx.x] = cnt;
    __threadfence();  // every thread's list writes, before the ticket
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == (u32)nb - 1;
    __syncthreads();
    if (!s_last) return;
    // The last block merges the blocks' lists, read from L2 (other blocks
    // wrote them): entry e of the nb * K list slots is valid when its slot
    // is below its list's count.
    __threadfence();
    const int total = nb * K;
    cnt = -1;
    if (K <= 32) {
      LaneTop T;
      T.clear();
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int b = e / K;
        const int c = __ldcg(part_c + b);
        const i64 k = __ldcg(part_k + e), s = __ldcg(part_s + e);
        if (e - b * K < c) T.insert(k, s);
      }
      cnt = tk_lane_rank(T, K, s_lr, out_keys, out_sums);
    }
    if (cnt < 0) {
      // Each warp offers 32 of the list slots per round.
      L.clear();
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
        cnt = L.cnt;
      }
    }
    if (threadIdx.x == 0) *d_nout = cnt;
  }
  // A plan's result record (out_keys, out_sums, d_nout point into it): the
  // rest of it from the plan's counters (groups, status, F rows).
  if (threadIdx.x == 0 && rec) {
    rec->ngroups = (i64)rec_ctr[0];
    rec->status = (int)rec_ctr[3];
    rec->reserved = 0;
    rec->hits = (i64)rec_ctr[2];
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

// Blocks of 256 threads (static shared memory only) resident per SM.
int resident_blocks256(const void* k) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    occ = 1;
  }
  return occ;
}

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
                        cudaStream_t s, const uint64_t* rec_ctr, pq_result* rec) {
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
                            (i64*)out_sums, (i64*)d_nout, (const u64*)rec_ctr, rec);
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
  const bool vec2 = sel ? aligned16(sel_in) : aligned16(col.data);
  if (ntiles >= (i64)ctx->num_sms * 8) {
    // Large input: count, scan the tile counts, write (no chain between tiles).
    const i64 stiles = (ntiles + 4095) / 4096;
    const size_t cnt_b = (size_t)((ntiles * 4 + 255) / 256 * 256), off_b = (size_t)((ntiles * 8 + 255) / 256 * 256);
    char* w2 = (char*)scr.get(cnt_b + off_b + stiles * 8 + 256);
    if (!w2) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_filter: no scratch");
    u32* counts = (u32*)w2;
    i64* offs = (i64*)(w2 + cnt_b);
    u32* sctr = (u32*)(w2 + cnt_b + off_b);
    PQ_CUDA(ctx, cudaMemsetAsync(counts, 0, cnt_b, s));
    PQ_CUDA(ctx, cudaMemsetAsync(sctr, 0, stiles * 8 + 256, s));
    const int g2 = (int)std::max<i64>(1, std::min<i64>(ntiles, (i64)ctx->num_sms * 8));
    PQ_DISPATCH_T(col.type, T, {
      if (sel) {
        if (vec2) k_filter_count<T, true, true><<<g2, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in, n_cap, (const i64*)d_n_in, p, counts);
        else k_filter_count<T, true, false><<<g2, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in, n_cap, (const i64*)d_n_in, p, counts);
      } else {
        if (vec2) k_filter_count<T, false, true><<<g2, 256, 0, s>>>((const T*)col.data, nullptr, n_cap, nullptr, p, counts);
        else k_filter_count<T, false, false><<<g2, 256, 0, s>>>((const T*)col.data, nullptr, n_cap, nullptr, p, counts);
      }
    });
    PQ_LAUNCHED(ctx);
    k_scan_u32<<<(unsigned)std::min<i64>(stiles, (i64)ctx->num_sms * 4), 256, 0, s>>>(
        counts, ntiles, offs, (u64*)(sctr + 64), sctr, ctx->opt.spin_limit, ctx->d_status);
    PQ_LAUNCHED(ctx);
    PQ_DISPATCH_T(col.type, T, {
      if (sel) {
        if (vec2) k_filter_write<T, true, true><<<g2, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in, n_cap, (const i64*)d_n_in, p, offs, counts, (i64*)sel_out, (i64*)d_count);
        else k_filter_write<T, true, false><<<g2, 256, 0, s>>>((const T*)col.data, (const i64*)sel_in, n_cap, (const i64*)d_n_in, p, offs, counts, (i64*)sel_out, (i64*)d_count);
      } else {
        if (vec2) k_filter_write<T, false, true><<<g2, 256, 0, s>>>((const T*)col.data, nullptr, n_cap, nullptr, p, offs, counts, (i64*)sel_out, (i64*)d_count);
        else k_filter_write<T, false, false><<<g2, 256, 0, s>>>((const T*)col.data, nullptr, n_cap, nullptr, p, offs, counts, (i64*)sel_out, (i64*)d_count);
      }
    });
    PQ_LAUNCHED(ctx);
    return PQ_OK;
  }
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
  if (log2P <= kStagedMaxLog2) {
    // Staged scatter: G persistent blocks, one chunk of rows each; with bulk
    // copies into double-buffered sub-tiles when every column is 16-byte
    // aligned and the buffers fit.
    TmaCols tc{};
    tc.n = 1 + npay;
    tc.src[0] = key.data;
    tc.dst[0] = out_key;
    tc.es[0] = (int)pqh::dtype_size(key.type);
    bool aligned = ((uintptr_t)key.data & 15) == 0 && ((uintptr_t)out_key & 15) == 0;
    for (int j = 0; j < npay; ++j) {
      tc.src[1 + j] = payload[j].data;
      tc.dst[1 + j] = out_payload[j];
      tc.es[1 + j] = (int)pqh::dtype_size(payload[j].type);
      aligned = aligned && ((uintptr_t)payload[j].data & 15) == 0;
    }
    // Sub-tiles of 4096 rows from 512 buckets on (when they fit), so that a
    // bucket's run in a sub-tile fills its sectors; 2048 otherwise.
    auto layout = [&](int sub) {
      int off = 0;
      for (int c = 0; c < tc.n; ++c) tc.off[c] = off, off += sub * tc.es[c];
      tc.buf_bytes = off;
      return tma_smem(P, tc.buf_bytes, sub);
    };
    int sub = log2P >= 9 ? 4096 : kSub;
    size_t smem_tma = layout(sub);
    if (smem_tma > 200 * 1024 && sub != kSub) smem_tma = layout(sub = kSub);
    const bool use_tma = aligned && smem_tma <= 200 * 1024;
    const size_t smem = use_tma ? smem_tma : staged_smem(P);
    const i64 rows_sub = use_tma ? sub : kSub;
    int occ = 1;
    PQ_DISPATCH_T(key.type, T, {
      const void* fn = !use_tma      ? (const void*)k_part_scatter_blk<T>
                       : sub == 4096 ? (const void*)k_part_scatter_tma<T, 4096>
                                     : (const void*)k_part_scatter_tma<T, kSub>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem) != cudaSuccess)
        occ = 1;
    });
    cudaGetLastError();
    const i64 g = std::max<i64>(1, std::min<i64>((n + rows_sub - 1) / rows_sub,
                                                 (i64)ctx->num_sms * std::max(occ, 1)));
    const i64 m = g * P;
    const i64 stiles = (m + 4095) / 4096;
    pqh::Scratch scr(ctx, s);
    u32* hist = (u32*)scr.get(m * 4);
    i64* gofs = (i64*)scr.get(m * 8);
    char* w = (char*)scr.get(stiles * 8 + 256);
    if (!hist || !gofs || !w) return pqh::fail(ctx, PQ_ERR_BUDGET, "pq_partition: no scratch");
    PQ_CUDA(ctx, cudaMemsetAsync(w, 0, stiles * 8 + 256, s));
    PQ_CUDA(ctx, cudaMemsetAsync(hist, 0, m * 4, s));
    // Histogram blocks: at most one wave of eight per SM (hsplit blocks per
    // chunk), each with at least 4096 rows.
    const int hsplit = (int)std::max<i64>(
        1, std::min<i64>(((i64)ctx->num_sms * 8) / g, (n / g) / 4096));
    PQ_DISPATCH_T(key.type, T, {
      k_part_hist_blk<T><<<(unsigned)(g * hsplit), 256, (size_t)P * 4, s>>>(
          (const T*)key.data, n, log2P, hist, g, hsplit);
      PQ_LAUNCHED(ctx);
      k_scan_u32<<<(unsigned)std::min<i64>(stiles, (i64)ctx->num_sms * 4), 256, 0, s>>>(
          hist, m, gofs, (u64*)(w + 256), (u32*)w, ctx->opt.spin_limit, ctx->d_status);
      PQ_LAUNCHED(ctx);
      if (use_tma && sub == 4096)
        k_part_scatter_tma<T, 4096><<<(unsigned)g, 256, smem, s>>>(
            n, log2P, gofs, tc, (i64*)d_offsets, ctx->opt.spin_limit, ctx->d_status);
      else if (use_tma)
        k_part_scatter_tma<T, kSub><<<(unsigned)g, 256, smem, s>>>(
            n, log2P, gofs, tc, (i64*)d_offsets, ctx->opt.spin_limit, ctx->d_status);
      else
        k_part_scatter_blk<T><<<(unsigned)g, 256, smem, s>>>((const T*)key.data, n, log2P, gofs,
                                                             pa, (T*)out_key, (i64*)d_offsets);
    });
    PQ_LAUNCHED(ctx);
    return PQ_OK;
  }
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
  ht->keys = (i64*)((char*)ht->block + 256);  // {key, value} per slot
  ht->vals = ht->keys + 1;
  ht->log2cap = log2cap;
  ht->n = key.n;
  pq_status st = pqh::fill_i64(ctx, ht->keys, 2 * cap, kEmpty, s);
  if (st == PQ_OK && cudaMemsetAsync(ht->meta, 0, 256, s) != cudaSuccess)
    st = pqh::fail(ctx, PQ_ERR_CUDA, "memset");
  if (st == PQ_OK && key.n > 0) {
    const int grid = (int)std::min<i64>((key.n + 255) / 256, (i64)ctx->num_sms * 8);
    PQ_DISPATCH_T(key.type, TK, {
      if (!val.data) {
        k_ht_build<TK, long long><<<grid, 256, 0, s>>>((const TK*)key.data, nullptr, key.n,
                                                       ht->keys, log2cap, ht->meta,
                                                       ctx->d_status);
      } else {
        PQ_DISPATCH_T(val.type, TV, {
          k_ht_build<TK, TV><<<grid, 256, 0, s>>>((const TK*)key.data, (const TV*)val.data,
                                                  key.n, ht->keys, log2cap, ht->meta,
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
  PQ_DISPATCH_T(probe_key.type, TK, {
    static const int occ = std::max(1, resident_blocks256((const void*)k_ht_probe<TK>));
    const int grid = (int)std::min<i64>((probe_key.n + 511) / 512, (i64)ctx->num_sms * occ);
    k_ht_probe<TK><<<grid, 256, 0, s>>>((const TK*)probe_key.data, probe_key.n,
                                        (const longlong2*)ht->keys, ht->log2cap, ht->meta,
                                        (i64*)out_probe_row,
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
  // Large inputs outside stream capture: measure the key range (one read of
  // the keys and one small read-back); dense keys take the slot array.
  cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &capst);
  if (capst == cudaStreamCaptureStatusNone && key.n >= (1 << 20)) {
    pqh::Scratch rs(ctx, s);
    u64* rng = (u64*)rs.get(256);
    if (rng) {
      PQ_CUDA(ctx, cudaMemsetAsync(rng, 0xFF, 8, s));
      PQ_CUDA(ctx, cudaMemsetAsync(rng + 1, 0, 8, s));
      const int gr = (int)std::min<i64>((key.n + 1023) / 1024, (i64)ctx->num_sms * 8);
      PQ_DISPATCH_T(key.type, TK, {
        k_gb_range<TK><<<gr, 256, 0, s>>>((const TK*)key.data, key.n, rng);
      });
      PQ_LAUNCHED(ctx);
      pqh::SmallPinned hp(ctx);
      PQ_CUDA(ctx, cudaMemcpyAsync(hp.p, rng, 16, cudaMemcpyDeviceToHost, s));
      PQ_CUDA(ctx, cudaStreamSynchronize(s));
      const u64 lo = (u64)hp.p[0], hi = (u64)hp.p[1];
      const u64 span = hi >= lo ? hi - lo + 1 : 0;
      if (span && span <= 4 * (u64)key.n && span <= (1ULL << 34)) {
        pqh::Scratch scr(ctx, s);
        const size_t sb = (size_t)((span * 8 + 255) / 256 * 256);
        const size_t bb = (size_t)(((span + 31) / 32 * 4 + 255) / 256 * 256);
        char* blk = (char*)scr.get(sb + bb);
        if (blk) {
          i64* sums = (i64*)blk;
          u32* bm = (u32*)(blk + sb);
          PQ_CUDA(ctx, cudaMemsetAsync(blk, 0, sb + bb, s));
          const int gd = (int)std::min<i64>((key.n + 1023) / 1024, (i64)ctx->num_sms * 8);
          PQ_DISPATCH_T(key.type, TK, {
            PQ_DISPATCH_T(val.type, TV, {
              k_gb_dense<TK, TV><<<gd, 256, 0, s>>>((const TK*)key.data, (const TV*)val.data,
                                                    key.n, lo, sums, bm, ctx->d_status);
            });
          });
          PQ_LAUNCHED(ctx);
          const i64 words = (i64)((span + 31) / 32);
          const int ge = (int)std::max<i64>(1, std::min<i64>((words + 255) / 256, (i64)ctx->num_sms * 8));
          k_gb_dense_emit<<<ge, 256, 0, s>>>(bm, sums, span, lo, (i64*)out_keys, (i64*)out_sums,
                                             cap, (u64*)d_ngroups);
          PQ_LAUNCHED(ctx);
          k_check_cap<<<1, 1, 0, s>>>((const i64*)d_ngroups, cap, ctx->d_status);
          PQ_LAUNCHED(ctx);
          return PQ_OK;
        }
      }
    }
  }
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
