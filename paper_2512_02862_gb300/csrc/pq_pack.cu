// pq_pack.cu -- packed columns: frame of reference + bit packing per block of
// PQ_PACK_BLOCK rows, packed on the host (storage format) and decoded on the
// device after each chunk's copy, so that the host link carries the packed
// bytes (Sec. 4.1: the scan loads compressed row groups and GPU kernels decode
// them; Sec. 5.4: data crosses the link compressed and is decoded only on the
// GPU).  The layout is documented with pq_pack_column in pq.h.
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "pq_internal.h"

namespace pqh {

namespace {

constexpr uint32_t kMagic = 0x4B505150u;  // "PQPK"
constexpr int64_t kB = PQ_PACK_BLOCK;
constexpr int kPadWords = 4;

struct PackHeader {
  uint32_t magic, version;
  int32_t type;
  uint32_t block_rows;
  int64_t nrows, nblocks;
};
static_assert(sizeof(PackHeader) == 32, "packed header");

size_t table_bytes(int64_t nblocks) { return (size_t)(nblocks + 1) * sizeof(PackBlock); }
size_t payload_offset(int64_t nblocks) {
  return (sizeof(PackHeader) + table_bytes(nblocks) + 15) / 16 * 16;
}

int64_t value_at(const void* src, int type, int64_t i) {
  switch (type) {
    case PQ_INT8: return ((const int8_t*)src)[i];
    case PQ_INT32: return ((const int32_t*)src)[i];
    default: return ((const int64_t*)src)[i];
  }
}

int bits_for(uint64_t x) {
  int w = 0;
  while (w < 64 && (x >> w) != 0) ++w;
  return w;
}

// Run f(lo, hi) over [0, n) split across the machine's threads.
template <typename F>
void parallel_for(int64_t n, F f) {
  const int64_t nt = std::max<int64_t>(
      1, std::min<int64_t>(std::thread::hardware_concurrency(), (n + 63) / 64));
  if (nt == 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t)
    th.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

}  // namespace

bool packed_info(const void* p, int type, int64_t nrows, PackedView* v) {
  PackHeader h;
  memcpy(&h, p, sizeof h);
  if (h.magic != kMagic || h.version != 1 || h.type != type || h.block_rows != (uint32_t)kB ||
      h.nrows != nrows || h.nblocks != (nrows + kB - 1) / kB)
    return false;
  v->blocks = reinterpret_cast<const PackBlock*>((const char*)p + sizeof(PackHeader));
  v->words = reinterpret_cast<const uint32_t*>((const char*)p + payload_offset(h.nblocks));
  v->nblocks = h.nblocks;
  v->total_words = v->blocks[h.nblocks].word;
  return true;
}

// One value of a packed column: base + bits [i*width, (i+1)*width) of its
// block's stream (`words` starts at payload word w0), read from the two or
// three words that hold them.
__device__ __forceinline__ int64_t unpack_one(const PackBlock& b, const uint32_t* words, int64_t w0,
                                              int64_t i) {
  if (!b.width) return b.base;
  const uint64_t bit = (uint64_t)i * b.width;
  const uint32_t* w = words + (b.word - w0) + (bit >> 5);
  const uint32_t sh = (uint32_t)(bit & 31);
  const uint64_t lo = (uint64_t)__ldg(w) | ((uint64_t)__ldg(w + 1) << 32);
  uint64_t d = lo >> sh;
  if (sh + b.width > 64) d |= (uint64_t)__ldg(w + 2) << (64 - sh);
  if (b.width < 64) d &= (1ULL << b.width) - 1;
  return (int64_t)((uint64_t)b.base + d);
}

// Decode rows [row0, row0 + n) of a packed column into `out` (element size of
// `type`, 16-byte aligned).  `blk` and `words` are the chunk's copies of the
// block table (starting at the block holding row0) and of the payload
// (starting at that block's first word, w0).  Each thread decodes four
// consecutive output rows and stores them with one vector store; it reloads
// the block entry only when its rows cross into the next block.
template <typename T>
__global__ void __launch_bounds__(256) k_unpack(const PackBlock* blk, const uint32_t* words,
                                                int64_t w0, int64_t row0, int64_t n, T* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = row0 % PQ_PACK_BLOCK;  // position of output row 0 in block 0
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * g < n; g += stride) {
    const int64_t r = 4 * g;
    int64_t pos = first + r;
    int64_t bi = pos / PQ_PACK_BLOCK;
    PackBlock b = blk[bi];
    T v[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 4; ++k, ++pos) {
      if (r + k < n) {
        if (pos / PQ_PACK_BLOCK != bi) b = blk[++bi];
        v[k] = (T)unpack_one(b, words, w0, pos % PQ_PACK_BLOCK);
      }
    }
    if (r + 4 <= n) {
      if (sizeof(T) == 8) {
        reinterpret_cast<longlong2*>(out + r)[0] = make_longlong2((int64_t)v[0], (int64_t)v[1]);
        reinterpret_cast<longlong2*>(out + r)[1] = make_longlong2((int64_t)v[2], (int64_t)v[3]);
      } else if (sizeof(T) == 4) {
        *reinterpret_cast<int4*>(out + r) = make_int4((int)v[0], (int)v[1], (int)v[2], (int)v[3]);
      } else {
        const uint32_t x = (uint32_t)(uint8_t)v[0] | (uint32_t)(uint8_t)v[1] << 8 |
                           (uint32_t)(uint8_t)v[2] << 16 | (uint32_t)(uint8_t)v[3] << 24;
        *reinterpret_cast<uint32_t*>(out + r) = x;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (r + k < n) out[r + k] = v[k];
    }
  }
}

PackedRange packed_range(const PackedView& v, int64_t row0, int64_t n) {
  PackedRange r;
  r.b0 = row0 / kB;
  r.b1 = (row0 + n + kB - 1) / kB;
  r.w0 = v.blocks[r.b0].word;
  r.w1 = v.blocks[r.b1].word + kPadWords;  // the decoder may read past a block's end
  return r;
}

cudaError_t unpack_launch(const PackBlock* dblk, const uint32_t* dwords, int64_t w0, int64_t row0,
                          int64_t n, int type, void* out, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 1023) / 1024, (int64_t)num_sms * 8);
  switch (type) {
    case PQ_INT8:
      k_unpack<<<(int)blocks, 256, 0, s>>>(dblk, dwords, w0, row0, n, static_cast<int8_t*>(out));
      break;
    case PQ_INT32:
      k_unpack<<<(int)blocks, 256, 0, s>>>(dblk, dwords, w0, row0, n, static_cast<int32_t*>(out));
      break;
    default:
      k_unpack<<<(int)blocks, 256, 0, s>>>(dblk, dwords, w0, row0, n, static_cast<int64_t*>(out));
      break;
  }
  return cudaGetLastError();
}

}  // namespace pqh

extern "C" {

int64_t pq_pack_bound(int64_t nrows, int32_t type) {
  if (nrows < 0 || !pqh::valid_dtype(type)) return -1;
  const int64_t nb = (nrows + pqh::kB - 1) / pqh::kB;
  const int64_t words = (nrows * 64 + 31) / 32 + nb + pqh::kPadWords;  // width <= 64
  return (int64_t)pqh::payload_offset(nb) + 4 * words;
}

pq_status pq_pack_column(const void* src, int32_t type, int64_t nrows, void* out, int64_t cap,
                         int64_t* out_bytes) {
  using namespace pqh;
  if ((!src && nrows) || !out || !out_bytes || nrows < 0 || !valid_dtype(type))
    return PQ_ERR_INVALID_ARG;
  const int64_t nb = (nrows + kB - 1) / kB;
  std::vector<PackBlock> blk(nb + 1);
  // Pass 1: each block's base and width.
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b) {
      const int64_t r0 = b * kB, r1 = std::min(nrows, r0 + kB);
      int64_t mn = value_at(src, type, r0), mx = mn;
      for (int64_t i = r0 + 1; i < r1; ++i) {
        const int64_t x = value_at(src, type, i);
        mn = std::min(mn, x);
        mx = std::max(mx, x);
      }
      PackBlock p{};
      p.base = mn;
      p.width = (uint8_t)bits_for((uint64_t)mx - (uint64_t)mn);
      blk[b] = p;
    }
  });
  // Word offsets: each block's stream starts on a word boundary.
  int64_t words = 0;
  for (int64_t b = 0; b < nb; ++b) {
    blk[b].word = (uint32_t)words;
    const int64_t rows = std::min(kB, nrows - b * kB);
    words += (rows * blk[b].width + 31) / 32;
    if (words > 0xFFFFFFF0LL) return PQ_ERR_CAPACITY;  // 32-bit word offsets
  }
  blk[nb] = PackBlock{};
  blk[nb].word = (uint32_t)words;
  const size_t off = payload_offset(nb);
  const int64_t need = (int64_t)off + 4 * (words + kPadWords);
  *out_bytes = need;
  if (cap < need) return PQ_ERR_CAPACITY;
  char* o = static_cast<char*>(out);
  PackHeader h{kMagic, 1, type, (uint32_t)kB, nrows, nb};
  memcpy(o, &h, sizeof h);
  memcpy(o + sizeof h, blk.data(), table_bytes(nb));
  memset(o + sizeof h + table_bytes(nb), 0, off - sizeof h - table_bytes(nb));
  uint32_t* w = reinterpret_cast<uint32_t*>(o + off);
  memset(w, 0, 4 * (size_t)(words + kPadWords));
  // Pass 2: the bit streams (blocks own disjoint words).
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; ++b) {
      const int width = blk[b].width;
      if (!width) continue;
      const int64_t r0 = b * kB, r1 = std::min(nrows, r0 + kB);
      uint32_t* bw = w + blk[b].word;
      for (int64_t i = r0; i < r1; ++i) {
        const uint64_t d = (uint64_t)value_at(src, type, i) - (uint64_t)blk[b].base;
        const uint64_t bit = (uint64_t)(i - r0) * width;
        uint32_t* p = bw + (bit >> 5);
        const int sh = (int)(bit & 31);
        p[0] |= (uint32_t)(d << sh);
        if (sh + width > 32) p[1] |= (uint32_t)(d >> (32 - sh));
        if (sh + width > 64) p[2] |= (uint32_t)(d >> (64 - sh));
      }
    }
  });
  return PQ_OK;
}

}  // extern "C"
