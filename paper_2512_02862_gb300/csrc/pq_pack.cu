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

// Decode rows [row0, row0 + n) of a packed column into `out` (element size of
// `type`).  `blk` and `words` are the chunk's copies of the block table
// (starting at the block holding row0, whose index in the column is b0) and
// of the payload (starting at that block's first word, w0).  One thread per
// output row: value = base + bits [i*width, (i+1)*width) of its block's
// stream, read from the two or three words that hold them.
__global__ void __launch_bounds__(256) k_unpack(const PackBlock* blk, const uint32_t* words,
                                                int64_t w0, int64_t row0, int64_t n, int type,
                                                void* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int64_t pos = row0 % PQ_PACK_BLOCK + r;  // row within the chunk's first block onward
    const PackBlock b = blk[pos / PQ_PACK_BLOCK];
    const uint64_t bit = (uint64_t)(pos % PQ_PACK_BLOCK) * b.width;
    int64_t v = b.base;
    if (b.width) {
      const uint32_t* w = words + (b.word - w0) + (bit >> 5);
      const uint32_t sh = (uint32_t)(bit & 31);
      const uint64_t lo = (uint64_t)__ldg(w) | ((uint64_t)__ldg(w + 1) << 32);
      uint64_t d = lo >> sh;
      if (sh + b.width > 64) d |= (uint64_t)__ldg(w + 2) << (64 - sh);
      if (b.width < 64) d &= (1ULL << b.width) - 1;
      v = (int64_t)((uint64_t)b.base + d);
    }
    switch (type) {
      case PQ_INT8: static_cast<int8_t*>(out)[r] = (int8_t)v; break;
      case PQ_INT32: static_cast<int32_t*>(out)[r] = (int32_t)v; break;
      default: static_cast<int64_t*>(out)[r] = v; break;
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
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
  k_unpack<<<(int)blocks, 256, 0, s>>>(dblk, dwords, w0, row0, n, type, out);
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
