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
#include <type_traits>

#include "../../include/pq.h"
#include "pq_dev.cuh"
#include "pq_topk.cuh"

namespace pqk {

// Largest rows per warp tile of the D, M and F scans; a plan uses smaller
// tiles (down to 512, 128 and 128 rows) when its table would otherwise leave
// resident warps without a tile.
constexpr int kTD = 1024;
constexpr int kTM = 1024;
constexpr int kTF = 2048;
constexpr int kTB = 128;     // list entries inserted per warp tile (4 per lane)
constexpr int kQ = 256;      // entries of a warp's shared-memory ring

struct QCtr {
  u64 dcount, mcount, gcount;
  int dup;          // dense M dictionary: the M list repeats keys
  u32 tk_ticket;
  int status;
  int mlog2;
  // Order-preserving key ranges (ukey = key xor 2^63), zero-initialised:
  // n* holds ~min, u* holds max, both grown with atomicMax.
  u64 d_nmin, d_umax, m_nmin, m_umax;
  u64 m_umin;  // M bitmap: ukey of bit 0
  u64 m_bits;  // M bitmap: bit count (0 = no bitmap)
  u64 pad[2];
  // Regions the D and M fills clear: byte offset from the table's start and
  // 16-byte units (set by the scans' last blocks).
  u64 d_fill_off, d_fill_units, m_fill_off, m_fill_units;
  u64 m_distinct;  // dense M dictionary: distinct keys (the rank pass)
  u64 hcount;      // F rows in the hit list
  u64 hits_total;  // F rows that joined, over all chunks
  i64 hp_tile;     // hits per warp tile of the probe
};

// Key-range semi-join filter.  When the keys of a filtered build side span
// at most 32 bits per table slot, an exact bitmap over that range sits beside
// the table: a probe key outside the range, or whose bit is clear, cannot
// match, so only the few keys whose bit is set probe the table.
__device__ __forceinline__ u64 ukey(i64 k) { return (u64)k ^ 0x8000000000000000ULL; }

struct RangeBits {
  u64 umin, bits;
};
// Largest key-range bitmap, in bits (bitmap word indices fit in 32 bits).
constexpr u64 kMaxBmBits = 1ULL << 37;
// Choose a bitmap for `count` keys spanning [~nmin, umax] (ukeys) in a table
// of 2^e slots: used when the span is below 32 * 2^e bits (and kMaxBmBits).
__device__ __forceinline__ RangeBits range_bits(i64 count, u64 nmin, u64 umax, int e) {
  RangeBits r{0, 0};
  if (count <= 0) return r;
  const u64 umin = ~nmin;
  const u64 span = umax - umin;  // bits - 1
  if (umax >= umin && span < (32ULL << e) && span < kMaxBmBits) {
    r.umin = umin;
    r.bits = span + 1;
  }
  return r;
}
// Layout of a plan table of 2^e slots (byte offsets from its tag array; the
// host carves workspaces and the device clears tables with this one
// function).  tags: 2 B per slot (0 = free); bcnt: one u32 fill counter per
// 8-slot bucket; hit: first-hit bits (tables with sums only); keybm: the
// key-range bitmap (up to 32 bits per slot); rec: 8-byte keys, or 16-byte
// {key, sum} records.  Everything before `rec` starts at zero.
struct TableLayout {
  u64 bcnt, hit, keybm, rec, total;
};
__host__ __device__ __forceinline__ TableLayout table_layout(int e, bool with_sums) {
  const u64 n = 1ULL << e;
  auto a = [](u64 x) { return (x + 255) & ~255ULL; };
  TableLayout L;
  L.bcnt = a(2 * n);
  L.hit = L.bcnt + a(n / 2);
  L.keybm = L.hit + (with_sums ? a(n / 8) : 0);
  L.rec = L.keybm + a(4 * n);
  L.total = L.rec + (with_sums ? 16 : 8) * n;
  return L;
}

// Clearing a table: its tags, bucket counters, hit bits and the used part of
// its key bitmap, in 16-byte units, kTCU units per fill tile.
constexpr int kTCU = 2048;
__host__ __device__ __forceinline__ i64 clear_units(int e, bool with_sums, u64 bits) {
  return (i64)((table_layout(e, with_sums).keybm + ((bits + 31) / 32) * 4 + 15) / 16);
}
__host__ __device__ __forceinline__ i64 fill_tiles(int e, bool with_sums, u64 bits) {
  return (clear_units(e, with_sums, bits) + kTCU - 1) / kTCU;
}

// Top-k tiles of an M table of 2^e slots: ranges of its first-hit bitmap,
// at least 32 words each and at most kTKP tiles per table (so that the
// last tile's threshold is taken over at most kTKP tile maxima).
constexpr int kTKP = 256;  // most top-k tiles of a plan
__host__ __device__ __forceinline__ i64 topk_tile_words(int e) {
  const i64 words = ((1LL << e) + 31) >> 5;
  i64 tw = 32;
  while ((words + tw - 1) / tw > kTKP) tw <<= 1;
  return tw;
}
__host__ __device__ __forceinline__ i64 topk_parts(int e) {
  const i64 words = ((1LL << e) + 31) >> 5;
  const i64 tw = topk_tile_words(e);
  return (words + tw - 1) / tw;
}
// Entries of the tiles' top-K lists: at most kTKP (256) tiles of at least
// 1024 slots each, so K lists fit in K tiles' worth of slots (or the whole
// table).
__host__ __device__ __forceinline__ i64 topk_cand_cap(int e, int K) {
  const i64 slots = 1LL << e, tile_slots = topk_tile_words(e) * 32;
  return slots < (i64)K * tile_slots ? slots : (i64)K * tile_slots;
}

// Dense M dictionary.  When the M' keys have a key-range bitmap, the M side
// is not a hash table: a group's slot is the rank of its key among the
// distinct M' keys (the set bits before its bit), read from a two-level
// directory (set bits before each tile of kRankTile 512-bit blocks, and
// before each 32-bit word within its tile) plus the key's word: three loads
// and one popcount.  Slots follow key order.  Layout in the M table's
// region, for c entries in the M list (members of M') and `bits` bitmap bits
// (byte offsets; the bitmap comes first so that its place does not depend
// on c):
//   bm    the key-range bitmap                64 B per 512-bit block
//   tdir  u32 set bits before each tile, then the total
//   wdir  u16 set bits before each word within its tile (2 B per word)
//   hit   first-hit bit per slot              c/8 B
//   sums  i64 sum per slot                    8c B
//   cnt   u32 copies of the key per slot      4c B (written only when the
//         members repeat keys)
// The bitmap is cleared before the bits are set (by the host, or by the M
// fill); the rank pass writes the directories and clears hit, sums, cnt.
constexpr int kRankTile = 64;   // bitmap blocks per tile (at most 32768 bits)
struct DenseLayout {
  u64 bm, tdir, wdir, hit, sums, cnt, total;
};
__host__ __device__ __forceinline__ DenseLayout dense_layout(i64 c, u64 bits) {
  auto a = [](u64 x) { return (x + 255) & ~255ULL; };
  const u64 blocks = (bits + 511) / 512, tiles = (blocks + kRankTile - 1) / kRankTile;
  DenseLayout L;
  L.bm = 0;
  L.tdir = a(64 * blocks);
  L.wdir = L.tdir + a(4 * (tiles + 1));
  L.hit = L.wdir + a(32 * blocks);
  L.sums = L.hit + a(((u64)c + 7) / 8);
  L.cnt = L.sums + a(8 * (u64)c);
  L.total = L.cnt + a(4 * (u64)c);
  return L;
}

// Top-k tiling over a first-hit bitmap of `words` words (the hash table's
// slots, or the dense dictionary's slots).
__host__ __device__ __forceinline__ i64 topk_tile_words_w(i64 words) {
  i64 tw = 32;
  while ((words + tw - 1) / tw > kTKP) tw <<= 1;  // at most kTKP tiles
  return tw;
}

__device__ __forceinline__ bool bit_test(const u32* bm, u64 idx, u64 keep) {
  u32 w;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(w) : "l"(bm + (idx >> 5)), "l"(keep));
  return (w >> (idx & 31)) & 1u;
}
__device__ __forceinline__ void bit_set(u32* bm, u64 idx) {
  atomicOr(bm + (idx >> 5), 1u << (idx & 31));
}

// Key-range bitmap test of a lane's 4 keys, split in two so that the word
// loads issued in one scan iteration are consumed in the next.  Keys outside
// `valid` never pass; with no bitmap (bits == 0) every valid key passes, and
// the caller resolves it against the table.
struct BmStage {
  u32 w[4];  // loaded words (0: key invalid or out of range)
  u32 sh;    // bit positions within the words, 5 bits per key
};
template <typename K>
__device__ __forceinline__ void bm_issue(BmStage& st, const u32* bm, u64 umin, u64 bits, u32 valid,
                                         const K k[4], u64 keep) {
  st.sh = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const u64 idx = ukey((i64)k[s]) - umin;
    const bool in = ((valid >> s) & 1u) && (bits == 0 || idx < bits);
    u32 w = 0;
    if (in) {
      if (bits == 0) {
        w = ~0u;
      } else {
        asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;"
            : "=r"(w) : "l"(bm + (idx >> 5)), "l"(keep));
      }
    }
    st.w[s] = w;
    st.sh |= (u32)(idx & 31) << (5 * s);
  }
}
// bm_issue for a bitmap that exists (bits > 0), with fewer instructions:
// ubase = umin xor 2^63, so that key - ubase (mod 2^64) is the key's bit
// index, and the word index is the low 32 bits of idx >> 5 (in range,
// idx < bits <= kMaxBmBits).
template <typename K>
__device__ __forceinline__ void bm_issue_fast(BmStage& st, const u32* bm, u64 ubase, u64 bits,
                                              u32 valid, const K k[4], u64 keep) {
  st.sh = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const u64 idx = (u64)(i64)k[s] - ubase;
    u32 w = 0;
    if (((valid >> s) & 1u) && idx < bits) {
      const u32 wi = (u32)(idx >> 5);
      asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(w) : "l"(bm + wi), "l"(keep));
    }
    st.w[s] = w;
    st.sh |= ((u32)idx & 31u) << (5 * s);
  }
}
__device__ __forceinline__ u32 bm_hits(const BmStage& st) {
  u32 h = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) h |= ((st.w[s] >> ((st.sh >> (5 * s)) & 31)) & 1u) << s;
  return h;
}

// Warp-wide fold of per-lane key ranges into the (zero-initialised) counters.
__device__ __forceinline__ void range_commit(u64 lane_nmin, u64 lane_umax, u64* nmin, u64* umax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 a = __shfl_xor_sync(kFull, lane_nmin, o), c = __shfl_xor_sync(kFull, lane_umax, o);
    lane_nmin = a > lane_nmin ? a : lane_nmin;
    lane_umax = c > lane_umax ? c : lane_umax;
  }
  if ((threadIdx.x & 31) == 0 && (lane_nmin | lane_umax)) {
    atomicMax(nmin, lane_nmin);
    atomicMax(umax, lane_umax);
  }
}

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
  int d_tile, m_tile, f_tile;  // rows per warp tile of the D, M and F scans
  // Key bitmaps over the whole key range of a resident table, known before
  // the plan runs: the D (M) scan sets the bits of its passing (member) keys
  // directly, with no key list and no build phase.  The host clears them.
  int d_static, m_static;
  // The M (F) columns are host memory read in place (mapped tables): the
  // scans then give lane l rows 2l, 2l+1, 64+2l, 65+2l of each 128-row step,
  // so that every load instruction of a warp reads one contiguous run (the
  // host link moves whole lines; on HBM the 4l .. 4l+3 layout is cheaper).
  int m_pair, f_pair;
  int d_e, m_e;  // log2 slots of the D-set and the M table for the table's rows
  u64 d_su, d_sb, m_su, m_sb;  // base ukey and bit count of those bitmaps
  Pred pd, pm, pf;
  int k, lf1024;
  int build_dset;   // this plan fills its D-set in this batch
  int vec;          // every column pointer is 16-byte aligned
  i64* dlist;
  int* dset_log2;   // header of the D-set block: log2 slots, then (u64) bitmap
                    // base ukey at byte 8 and bit count at byte 16
  unsigned short* dset_tag;  // D-set table (keys only), laid out by table_layout
  i64* mlist;
  unsigned short* ht_tag;    // M table ({key, sum} records), laid out by table_layout
  int* tk_c;    // top-k: per tile, the length of its list
  i64* cand_k;  // top-k: per tile, its sorted list of K (key, sum) records
  i64* cand_s;  // (topk_cand_cap entries hold every tile's)
  u32* hlist;   // F rows that hit (n_f entries, rows of the plan)
  // Partitioned F phase (PQ_PLAN_PARTITIONED): the hits are radix-
  // partitioned by group slot into 2^part_log2 buckets (part_shift) before
  // they are aggregated, so that each bucket's slice of the group arrays is
  // small enough to stay in L2 while its hits are added.  0: not partitioned.
  // Dynamic buffering of a streamed plan's F hits (hb_cap > 0): the F scan
  // gathers every hit's key, price and discount into these arrays (so the
  // chunk's ring slot is free at once); the host launches the probe only
  // after every few chunks (as many as the buffer holds rows of) and after
  // the last one.
  i64* hb_key;
  i64* hb_price;
  signed char* hb_disc;
  u64 hb_cap;
  // Upper bound of |price * (100 - disc)| over the F table's rows (from the
  // measured range of its price column), or 0 when unknown.  When the hits
  // times this bound times the largest multiplicity stay below 2^63, no
  // group sum or partial sum can leave int64, and the probe commits with
  // fire-and-forget reductions and no overflow checks (fast_commit).
  u64 rev_max;
  int part_log2;
  u64* part;    // [2^part_log2 + 1]: matched hits per bucket, then the
                // buckets' write cursors (their offsets in pslot / pval)
  i64* pval0;   // revenue of each hit in hit order (n_f entries; the slot
                // replaces the row in hlist)
  u32* pslot;   // partitioned hits (n_f entries): group slot
  i64* pval;    //                                 revenue times multiplicity
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
  int tile;  // rows per warp tile
};

struct Batch {
  PlanDev* q;
  int nq;
  int clear_m;    // the D scan clears the plans' static M bitmaps
  const i64* tD;  // static tile prefixes [nq + 1]
  const i64* tM;
  const i64* tF;
  i64* dyn;       // dynamic prefixes [5][nq + 1]: dclear, dbuild, mclear, mbuild, topk
  u32* work;      // [8] work tickets, [8..16) done tickets
  DevStatus* st;
  i64 spin_limit;
  Ovr ov;
};

enum { kPhDscan = 0, kPhDfill, kPhDbuild, kPhMscan, kPhMfill, kPhMbuild, kPhFprobe, kPhTopk,
       kPhMrank, kPhMdup, kPhFscan, kPhFpart, kPhFagg, kPhFscatter };

// Largest fan-out of a partitioned plan (buckets 2^kMaxPartLog2), hits per
// block tile of its partition and scatter passes, records per warp tile of
// its aggregation pass.
constexpr int kMaxPartLog2 = 10;
constexpr int kPT = 2048;
constexpr int kAT = 1024;

// Bucket of a hit in a partitioned plan with 2^log2P buckets: the top bits
// of its group slot among the plan's n slots, bucket = slot >> part_shift(n,
// log2P).  Dense M dictionary: slots are ranks in key order, so a bucket is
// a key range; hash table: a slot's top bits are its key's home bucket, the
// top bits of the key's Fibonacci product (a radix hash partition).  Either
// way a bucket's groups occupy one contiguous range of the group arrays.
__host__ __device__ __forceinline__ int part_shift(u64 n, int log2P) {
  int len = 0;  // bits needed for the largest slot, n - 1
  for (u64 x = n > 0 ? n - 1 : 0; x; x >>= 1) ++len;
  return len > log2P ? len - log2P : 0;
}

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

// Tile claims of the persistent plan kernels.  A warp's (block's) first
// tile is its own index in the grid; later ones come from the phase's ticket
// counter, offset by the number of warps (blocks), so a phase with fewer
// tiles than warps takes no ticket at all.
struct WarpClaim {
  bool first = true;
  __device__ __forceinline__ i64 next(u32* work, int ph) {
    const i64 nw = (i64)gridDim.x * (blockDim.x >> 5);
    if (first) {
      first = false;
      return (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    }
    u32 t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(&work[ph], 1u);
    return (i64)__shfl_sync(kFull, t, 0) + nw;
  }
};
struct BlockClaim {
  bool first = true;
  __device__ __forceinline__ i64 next(u32* work, int ph, i64* s_t) {
    if (first) {
      first = false;
      return blockIdx.x;
    }
    __syncthreads();
    if (threadIdx.x == 0) *s_t = atomicAdd(&work[ph], 1u);
    __syncthreads();
    return *s_t + gridDim.x;
  }
};

// Returns true in the block that finishes last; that block also resets the
// phase's tickets so that the next launch starts from zero.
__device__ __forceinline__ bool finish(u32* work, int ph) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const u32 t = atomicAdd(&work[16 + ph], 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) {
      work[ph] = 0;
      work[16 + ph] = 0;
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

// Device view of a table laid out by table_layout.
struct TableView {
  unsigned short* tags;
  u32* bcnt;
  u32* hit;
  u32* keybm;
  i64* rec;
  Geo g;
};
__device__ __forceinline__ TableView table_view(unsigned short* tags, int e, bool with_sums) {
  const TableLayout L = table_layout(e, with_sums);
  char* base = reinterpret_cast<char*>(tags);
  TableView t;
  t.tags = tags;
  t.bcnt = reinterpret_cast<u32*>(base + L.bcnt);
  t.hit = reinterpret_cast<u32*>(base + L.hit);
  t.keybm = reinterpret_cast<u32*>(base + L.keybm);
  t.rec = reinterpret_cast<i64*>(base + L.rec);
  t.g = geo(e);
  return t;
}

// Membership of k in a bucketized key set (8-byte key records).
__device__ __forceinline__ bool set_contains(const TableView& t, i64 k, u64 keep) {
  const BucketTag bt = bucket_tag(k, t.g.shiftb);
  const unsigned v2 = bt.tag * 0x10001u;
  u64 b = bt.bucket;
  for (u64 p = 0; p <= t.g.bmask; ++p) {
    const uint4 w = ld_keep_v4u(t.tags + b * 8, keep);
    Mask8 m = match8(w, v2);
    while (any8(m)) {
      const int j = first8(m);
      if (ld_keep(t.rec + b * 8 + j, keep) == k) return true;
      drop8(m, j);
    }
    if (any8(match8(w, 0u))) return false;
    b = (b + 1) & t.g.bmask;
  }
  return false;
}

// Claim a slot for a key of home bucket bt.bucket (one slot per insert, so
// duplicate keys take one slot each): the bucket's fill counter hands out
// slots 0..7; a full bucket passes the key to the next one.  The tag is
// written here; the caller writes the record.  Returns the slot.
__device__ __forceinline__ u64 claim_from(const TableView& t, BucketTag bt, u32 first) {
  u64 b = bt.bucket;
  u32 c = first;
  for (u64 p = 0; p <= t.g.bmask; ++p) {
    if (c < 8) {
      t.tags[b * 8 + c] = (unsigned short)bt.tag;
      return b * 8 + c;
    }
    b = (b + 1) & t.g.bmask;
    c = atomicAdd(t.bcnt + b, 1u);
  }
  return ~0ULL;  // unreachable: a table is never filled beyond its load factor
}

// A warp inserts the entries [i0, i0 + 128) of `src` (those below n): four
// per lane, whose four slot claims (counter atomics) are in flight together.
// on(k, slot) writes the record after each claim.
template <typename OnSlot>
__device__ __forceinline__ void insert_x4(const TableView& t, const i64* src, i64 i0, i64 n,
                                          OnSlot on) {
  const int lane = threadIdx.x & 31;
  i64 k[4];
  BucketTag bt[4];
  u32 c[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const i64 idx = i0 + j * 32 + lane;
    k[j] = idx < n ? src[idx] : kEmpty;
    bt[j] = bucket_tag(k[j], t.g.shiftb);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (k[j] != kEmpty) c[j] = atomicAdd(t.bcnt + bt[j].bucket, 1u);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (k[j] != kEmpty) on(k[j], claim_from(t, bt[j], c[j]));
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
  chain_begin();
  const bool ov = b.ov.table == 1;
  const i64 total = ov ? b.ov.tiles : b.tD[b.nq];
  const int lane = threadIdx.x & 31;
  const u64 strm = policy_stream();
  if (b.clear_m) {  // the M scan sets these bits next
    const i64 nt = (i64)gridDim.x * blockDim.x, tid = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    for (int qi = 0; qi < b.nq; ++qi) {
      const PlanDev& q = b.q[qi];
      if (!q.m_static) continue;
      int4* z = reinterpret_cast<int4*>(q.ht_tag);  // dense layout: bitmap at 0
      const i64 units = (i64)(dense_layout(0, q.m_sb).tdir / 16);
      for (i64 u = tid; u < units; u += nt) z[u] = make_int4(0, 0, 0, 0);
    }
  }
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhDscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tD, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int* d_key = ov ? (const int*)b.ov.p[0] : q.d_key;
    const signed char* d_seg = ov ? (const signed char*)b.ov.p[1] : q.d_seg;
    const i64 n = ov ? b.ov.n : q.n_d;
    const int tile = ov ? b.ov.tile : q.d_tile;
    const i64 base = (t - (ov ? 0 : b.tD[qi])) * tile;
    // Static bitmap: set the passing keys' bits (no list, no build phase).
    const bool stat = !ov && q.d_static;
    u32* sbm = stat ? table_view(q.dset_tag, q.d_e, false).keybm : nullptr;
    u64 lnmin = 0, lumax = 0;  // this lane's range of appended keys
    for (int it = 0; it < tile / 512; ++it) {
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
      // The lane's 16 keys at once (four 128-bit loads), not one dependent
      // load per passing row.
      int kk[16];
      if (VEC && e0 + 16 <= n) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int4 x = bits ? ld_stream_v4(d_key + e0 + 4 * v, strm) : make_int4(0, 0, 0, 0);
          kk[4 * v] = x.x, kk[4 * v + 1] = x.y, kk[4 * v + 2] = x.z, kk[4 * v + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int s = 0; s < 16; ++s) kk[s] = (bits >> s) & 1u ? __ldg(d_key + e0 + s) : 0;
      }
      if (stat) {
#pragma unroll
        for (int s = 0; s < 16; ++s)
          if ((bits >> s) & 1u) bit_set(sbm, ukey((i64)kk[s]) - q.d_su);
        continue;
      }
      u64 at = warp_reserve(&q.ctr->dcount, (u32)__popc(bits));
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        if (!((bits >> s) & 1u)) continue;
        const i64 k = (i64)kk[s];
        q.dlist[at++] = k;
        lnmin = max(lnmin, ~ukey(k));
        lumax = max(lumax, ukey(k));
      }
    }
    range_commit(lnmin, lumax, &q.ctr->d_nmin, &q.ctr->d_umax);
  }
  if (finish(b.work, kPhDscan)) {
    block_prefix(b.dyn, b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      if (!q.build_dset) return 0;
      if (q.d_static) {  // bitmap over the table's key range, cleared by the host
        *q.dset_log2 = q.d_e;
        u64* hdr = reinterpret_cast<u64*>(q.dset_log2);
        hdr[1] = q.d_su;
        hdr[2] = q.d_sb;
        q.ctr->d_fill_units = 0;
        return 0;
      }
      const i64 cnt = ld_count(&q.ctr->dcount);
      const int e = cap_log2(cnt, q.lf1024);
      const RangeBits rb = range_bits(cnt, ld_volatile_u64(&q.ctr->d_nmin),
                                      ld_volatile_u64(&q.ctr->d_umax), e);
      *q.dset_log2 = e;
      u64* hdr = reinterpret_cast<u64*>(q.dset_log2);
      hdr[1] = rb.umin;
      hdr[2] = rb.bits;
      // With a bitmap the D-set is the bitmap alone (membership is all that
      // the M scan asks); otherwise tags and bucket counters.
      const TableLayout L = table_layout(e, false);
      q.ctr->d_fill_off = rb.bits ? L.keybm : 0;
      q.ctr->d_fill_units = rb.bits ? (rb.bits + 127) / 128 : L.keybm / 16;
      return ((i64)q.ctr->d_fill_units + kTCU - 1) / kTCU;
    });
    block_prefix(b.dyn + (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      return q.build_dset && !q.d_static ? (ld_count(&q.ctr->dcount) + kTB - 1) / kTB : 0;
    });
  }
}

// ------------------------------------------------------------------- fill ----
// Clear the region of the D-set (which = 0) or the M side (which = 1) that
// the scan's last block recorded: tags and counters of a hash table, or the
// bitmap (and for M the dense arrays); records are written by the builds.
__global__ void __launch_bounds__(256) k_plan_fill(Batch b, int which) {
  chain_begin();
  const i64* pre = b.dyn + (which == 0 ? 0 : 2) * (b.nq + 1);
  const int ph = which == 0 ? kPhDfill : kPhMfill;
  const i64 total = pre[b.nq];
  __shared__ i64 s_t;
  BlockClaim bc;
  while (true) {
    const i64 t = bc.next(b.work, ph, &s_t);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const u64 off = which == 0 ? q.ctr->d_fill_off : q.ctr->m_fill_off;
    const i64 units = (i64)(which == 0 ? q.ctr->d_fill_units : q.ctr->m_fill_units);
    int4* base = reinterpret_cast<int4*>(
        reinterpret_cast<char*>(which == 0 ? (void*)q.dset_tag : (void*)q.ht_tag) + off);
    const i64 u0 = (t - pre[qi]) * kTCU;
    for (i64 u = u0 + threadIdx.x; u < u0 + kTCU && u < units; u += blockDim.x)
      base[u] = make_int4(0, 0, 0, 0);
  }
  finish(b.work, ph);
}

// ----------------------------------------------------------------- dbuild ----
// Warp tiles of 128 D-list entries, claimed per warp: bitmap bits when the
// D-set is a bitmap, else table inserts (insert_x4).
__global__ void __launch_bounds__(256) k_plan_dbuild(Batch b) {
  chain_begin();
  const i64* pre = b.dyn + (b.nq + 1);
  const i64 total = pre[b.nq];
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhDbuild);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const TableView tv = table_view(q.dset_tag, *q.dset_log2, false);
    const u64* hdr = reinterpret_cast<const u64*>(q.dset_log2);
    const u64 umin = hdr[1], bits = hdr[2];
    const i64 i0 = (t - pre[qi]) * kTB, n = (i64)q.ctr->dcount;
    if (bits) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const i64 idx = i0 + j * 32 + (threadIdx.x & 31);
        if (idx < n) bit_set(tv.keybm, ukey(q.dlist[idx]) - umin);
      }
    } else {
      insert_x4(tv, q.dlist, i0, n, [&](i64 k, u64 s) { tv.rec[s] = k; });
    }
  }
  finish(b.work, kPhDbuild);
}

// ------------------------------------------------------------------ mscan ----
// The M scan's last block: the M side's layout per plan (static bitmap, or
// sized from the members' count and key range) and the tile counts of the
// phases that follow.
__device__ void mscan_finish(const Batch& b) {
  block_prefix(b.dyn + 2 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
    const PlanDev& q = b.q[qi];
    if (q.m_static) {  // bitmap over the table's key range, set by this scan
      q.ctr->mlog2 = q.m_e;
      q.ctr->m_umin = q.m_su;
      q.ctr->m_bits = q.m_sb;
      q.ctr->m_fill_units = 0;
      return 0;
    }
    const i64 cnt = ld_count(&q.ctr->mcount);
    const int e = cap_log2(cnt, q.lf1024);
    const RangeBits rb = range_bits(cnt, ld_volatile_u64(&q.ctr->m_nmin),
                                    ld_volatile_u64(&q.ctr->m_umax), e);
    q.ctr->mlog2 = e;
    q.ctr->m_umin = rb.umin;
    q.ctr->m_bits = rb.bits;
    // With a bitmap the M side is a dense dictionary, else a hash table.
    q.ctr->m_fill_off = 0;
    q.ctr->m_fill_units = rb.bits ? dense_layout(cnt, rb.bits).tdir / 16
                                  : table_layout(e, true).keybm / 16;
    return ((i64)q.ctr->m_fill_units + kTCU - 1) / kTCU;
  });
  block_prefix(b.dyn + 3 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
    const PlanDev& q = b.q[qi];
    return q.m_static ? 0 : (ld_count(&q.ctr->mcount) + kTB - 1) / kTB;
  });
  block_prefix(b.dyn + 5 * (b.nq + 1), b.nq, [&](int qi) -> i64 {  // rank tiles
    const QCtr* c = b.q[qi].ctr;
    const u64 blocks = (c->m_bits + 511) / 512;
    return c->m_bits ? (i64)((blocks + kRankTile - 1) / kRankTile) : 0;
  });
}

// Warp tiles of up to 1024 M rows (sized per plan), 128 per iteration
// (lane l: rows 4l .. 4l+3).
// Pipeline per lane: date is read two iterations ahead, dref one ahead (only
// for 4-row groups with a date hit), the D-set bitmap words of the passing
// drefs are loaded in the iteration the drefs arrive and tested in the next.
// Member rows enter candidate ring C; rounds of 32 read their keys (only
// theirs) into ring B, which leaves for the M list in runs of 128 (one
// atomic reservation per run).  With no bitmap, every date-passing row is a
// candidate and the D-set table decides.
// LIST = false: every plan of the batch has a static M bitmap (no key list,
// ring B or key range), which keeps the kernel small.
template <bool VEC, bool LIST>
__global__ void __launch_bounds__(256, 3) k_plan_mscan(Batch b) {
  chain_begin();
  __shared__ u32 s_c[8][kQ];
  __shared__ i64 s_rb[8][LIST ? kQ : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32* cr = s_c[warp];
  i64* rb = s_rb[warp];
  const u64 keep = policy_keep(), strm = policy_stream();
  const bool ov = b.ov.table == 2;
  const i64 total = ov ? b.ov.tiles : b.tM[b.nq];
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhMscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tM, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* m_key = ov ? (const i64*)b.ov.p[0] : q.m_key;
    const int* m_dref = ov ? (const int*)b.ov.p[1] : q.m_dref;
    const int* m_date = ov ? (const int*)b.ov.p[2] : q.m_date;
    const TableView dt = table_view(q.dset_tag, *q.dset_log2, false);
    const u64* dhdr = reinterpret_cast<const u64*>(q.dset_log2);
    const u64 d_umin = dhdr[1], d_bits = dhdr[2];
    u64 lnmin = 0, lumax = 0;  // this lane's range of member keys
    const Pred32 pm = to32(q.pm);
    const i64 n = ov ? b.ov.n : q.n_m;
    const int tile = ov ? b.ov.tile : q.m_tile;
    const i64 base = (t - (ov ? 0 : b.tM[qi])) * tile;
    const i64 lim = min(n - base, (i64)tile);
    const int iters = (int)((lim + 127) / 128);
    const i64 r0 = lane * 4;
    // Static bitmap: members set their key's bit and are counted; no list.
    const bool stat = !LIST || (!ov && q.m_static);
    u32* sbm = stat ? reinterpret_cast<u32*>(q.ht_tag) : nullptr;  // dense layout: bm at 0
    u64 members = 0;
    u32 ch = 0, ct = 0, bh = 0, bt = 0;
    auto flush_b = [&](u32 cnt) {
      if (!LIST) return;
      u64 o = 0;
      if (lane == 0) o = atomicAdd(&q.ctr->mcount, (u64)cnt);
      o = __shfl_sync(kFull, o, 0);
      for (u32 j = lane; j < cnt; j += 32) q.mlist[o + j] = rb[(bh + j) & (kQ - 1)];
      bh += cnt;
    };
    auto resolve = [&](u32 cnt) {  // cnt <= 32 entries of C from ch
      bool mem = false;
      i64 key = 0;
      if ((u32)lane < cnt) {
        const u32 r = cr[(ch + lane) & (kQ - 1)];
        mem = d_bits || set_contains(dt, (i64)__ldg(m_dref + base + r), keep);
        if (mem) {
          key = __ldg(m_key + base + r);
          if (!stat) {
            lnmin = max(lnmin, ~ukey(key));
            lumax = max(lumax, ukey(key));
          }
        }
      }
      // A static bitmap covers the plan's M key window (the whole key range,
      // or one pass of an out-of-core plan): keys outside it are no members.
      if (stat && mem && ukey(key) - q.m_su >= q.m_sb) mem = false;
      const u32 m = __ballot_sync(kFull, mem);
      if (!LIST || stat) {
        if (mem) bit_set(sbm, ukey(key) - q.m_su);
        members += __popc(m);  // added to the plan's count once per tile
        ch += cnt;
        __syncwarp();
        return;
      }
      if (mem) rb[(bt + __popc(m & lanemask_lt())) & (kQ - 1)] = key;
      bt += __popc(m);
      ch += cnt;
      __syncwarp();
      if (bt - bh >= 128) flush_b(128);
    };
    auto append_c = [&](u32 hits, int it) {
      if (__any_sync(kFull, hits)) {
        __syncwarp();
        ct += ring_append(hits, ct, [&](int s, u32 pos) {
          cr[pos & (kQ - 1)] = (u32)(it * 128 + r0 + s);
        });
        __syncwarp();
      }
    };
    int4 dB = load_i32x4<VEC>(m_date, base + r0, lim - r0, strm);
    int4 dC = iters > 1 ? load_i32x4<VEC>(m_date, base + 128 + r0, lim - 128 - r0, strm)
                        : make_int4(0, 0, 0, 0);
    u32 hA = pass4(pm, dB, lim - r0);
    int4 rA = hA ? load_i32x4<VEC>(m_dref, base + r0, lim - r0, strm) : make_int4(0, 0, 0, 0);
    dB = dC;
    if (iters > 2) dC = load_i32x4<VEC>(m_date, base + 256 + r0, lim - 256 - r0, strm);
    BmStage wP;
    wP.w[0] = wP.w[1] = wP.w[2] = wP.w[3] = 0;
    wP.sh = 0;
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
      BmStage wN;
      bm_issue(wN, dt.keybm, d_umin, d_bits, hA, dr, keep);
      if (it > 0) {
        append_c(bm_hits(wP), it - 1);
        while (ct - ch >= 32) resolve(32);
      }
      wP = wN;
      hA = hB;
      rA = rB;
    }
    append_c(bm_hits(wP), iters - 1);
    while (ct - ch >= 32) resolve(32);
    if (ct - ch) resolve(ct - ch);
    if (bt - bh) flush_b(bt - bh);
    __syncwarp();
    if (!LIST || stat) {
      if (lane == 0 && members) atomicAdd(&q.ctr->mcount, members);
    } else {
      range_commit(lnmin, lumax, &q.ctr->m_nmin, &q.ctr->m_umax);
    }
  }
  if (finish(b.work, kPhMscan)) mscan_finish(b);
}

// Every plan of the batch has a static M bitmap and a D-set bitmap: each
// lane keeps its own 4 rows per step in registers, no ring.  date and dref
// are read two steps ahead, the D bitmap words are loaded when they arrive
// and tested one step later; then the members' keys are loaded, and two
// steps after that their bits are set (reductions nobody waits for).
// WIN: some plan of the batch is one pass of an out-of-core plan, whose M
// bitmap covers a key window: members outside it are dropped (compiled
// separately, so that the whole-range scan keeps its registers).
template <bool VEC, bool WIN>
__global__ void __launch_bounds__(256, 3) k_plan_mscan_bm(Batch b) {
  chain_begin();
  const int lane = threadIdx.x & 31;
  const u64 keep = policy_keep(), strm = policy_stream();
  const i64 total = b.tM[b.nq];
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhMscan);
    if (t >= total) break;
    const int qi = find_q(b.tM, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64* m_key = q.m_key;
    const int* m_dref = q.m_dref;
    const int* m_date = q.m_date;
    const u64* dhdr = reinterpret_cast<const u64*>(q.dset_log2);
    const u64 d_umin = dhdr[1], d_bits = dhdr[2];
    const TableView dt = table_view(q.dset_tag, *q.dset_log2, false);
    const u32* dt_keybm = dt.keybm;
    u32* sbm = reinterpret_cast<u32*>(q.ht_tag);  // dense layout: bm at 0
    const u64 m_su = q.m_su, m_sb = WIN ? q.m_sb : 0;  // the plan's M key window
    const Pred32 pm = to32(q.pm);
    const i64 base = (t - b.tM[qi]) * q.m_tile;
    const int lim = (int)min(q.n_m - base, (i64)q.m_tile);
    // The tile's rows, addressed with 32-bit offsets.
    const int* pdate = m_date + base;
    const int* pdref = m_dref + base;
    const i64* pkey = m_key + base;
    u32 members = 0;  // this lane's
    auto set_bits = [&](u32 m, const i64 k[4]) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const u64 idx = ukey(k[s]) - m_su;
        if (((m >> s) & 1u) && (!WIN || idx < m_sb)) bit_set(sbm, idx), ++members;
      }
    };
    if (d_bits == 0) {
      // A D-set that is a hash table (the host does not choose this kernel
      // then): row by row.
      for (int r = lane; r < lim; r += 32) {
        if (!pass32(pm, ld_stream(pdate + r))) continue;
        if (!set_contains(dt, (i64)__ldg(pdref + r), keep)) continue;
        const u64 idx = ukey(__ldg(pkey + r)) - m_su;
        if (!WIN || idx < m_sb) bit_set(sbm, idx), ++members;
      }
    } else {
      // Slot p = it % 2 holds date and dref of step it (read two steps
      // ahead, for every row); the key slots hold the member keys of two
      // earlier steps, read one step after their bitmap test and used two
      // steps later.  The loop is unrolled by two so that slots keep their
      // registers.
      const int iters = (lim + 127) / 128;
      // Compiled for full tiles of aligned columns (no row limits) and in
      // general.
      auto run = [&](auto full_c, auto pair_c) {
        constexpr bool FULL = decltype(full_c)::value, PAIR = decltype(pair_c)::value;
        // e0: the step's first row + the lane's first row (4l, or 2l).
        const int r0 = PAIR ? 2 * lane : 4 * lane;
        auto ld4 = [&](const int* p, int e0) -> int4 {
          if (PAIR) {
            const int2 a = ld_stream_v2i(p + e0, strm), c = ld_stream_v2i(p + e0 + 64, strm);
            return make_int4(a.x, a.y, c.x, c.y);
          }
          return FULL ? ld_stream_v4(p + e0, strm) : load_i32x4<VEC>(p, e0, lim - e0, strm);
        };
        auto ldk = [&](int e0, u32 bits, i64 v[4]) {
          if (PAIR) {
            if (bits & 3u) {
              const longlong2 x = ld_stream_v2(pkey + e0, strm);
              v[0] = x.x, v[1] = x.y;
            }
            if (bits & 12u) {
              const longlong2 y = ld_stream_v2(pkey + e0 + 64, strm);
              v[2] = y.x, v[3] = y.y;
            }
          } else if (FULL) {
            const longlong2 x = ld_stream_v2(pkey + e0, strm), y = ld_stream_v2(pkey + e0 + 2, strm);
            v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
          } else {
            load_i64x4<VEC>(pkey, e0, lim - e0, bits, strm, v);
          }
        };
        int4 dt0 = ld4(pdate, r0);
        int4 dr0 = ld4(pdref, r0);
        int4 dt1 = make_int4(0, 0, 0, 0), dr1 = make_int4(0, 0, 0, 0);
        if (iters > 1) {
          dt1 = ld4(pdate, 128 + r0);
          dr1 = ld4(pdref, 128 + r0);
        }
        BmStage W;  // D-bitmap words of the previous step's drefs
        W.w[0] = W.w[1] = W.w[2] = W.w[3] = 0;
        W.sh = 0;
        u32 km0 = 0, km1 = 0;  // member masks of the key slots
        i64 k0[4] = {0, 0, 0, 0}, k1[4] = {0, 0, 0, 0};
        auto step = [&](int it, int4& dt, int4& dr, u32& km, i64 (&kk)[4]) {
          set_bits(km, kk);  // members of step it - 3
          km = bm_hits(W);   // members of step it - 1: read their keys
          if (km) ldk((it - 1) * 128 + r0, km, kk);
          const int rel0 = it * 128 + r0;
          const u32 h = pass4(pm, dt, FULL ? 4 : lim - rel0);
          const int drv[4] = {dr.x, dr.y, dr.z, dr.w};
          bm_issue_fast(W, dt_keybm, d_umin ^ 0x8000000000000000ULL, d_bits, h, drv, keep);
          if (it + 2 < iters) {
            dt = ld4(pdate, rel0 + 256);
            dr = ld4(pdref, rel0 + 256);
          }
        };
        for (int it = 0; it < iters; it += 2) {
          step(it, dt0, dr0, km1, k1);
          if (it + 1 < iters) step(it + 1, dt1, dr1, km0, k0);
        }
        set_bits(km0, k0);
        set_bits(km1, k1);
        const u32 mL = bm_hits(W);
        i64 kL[4] = {0, 0, 0, 0};
        if (mL) ldk((iters - 1) * 128 + r0, mL, kL);
        set_bits(mL, kL);
      };
      if (VEC && lim == iters * 128) {
        if (q.m_pair) run(std::true_type{}, std::true_type{});
        else run(std::true_type{}, std::false_type{});
      } else {
        run(std::false_type{}, std::false_type{});
      }
    }
    const u32 wm = __reduce_add_sync(kFull, members);
    if (lane == 0 && wm) atomicAdd(&q.ctr->mcount, (u64)wm);
  }
  if (finish(b.work, kPhMscan)) mscan_finish(b);
}

// ----------------------------------------------------------------- mbuild ----
// Warp tiles of 128 M-list entries, claimed per warp.  Dense dictionary: set
// the keys' bitmap bits (reductions nobody waits for).  Hash table: insert
// {key, 0} records (insert_x4); a key equal to the reserved INT64_MIN is
// reported and skipped.
__global__ void __launch_bounds__(256) k_plan_mbuild(Batch b) {
  chain_begin();
  const i64* pre = b.dyn + 3 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31;
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhMbuild);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const u64 m_umin = q.ctr->m_umin, m_bits = q.ctr->m_bits;
    const i64 n = (i64)q.ctr->mcount;
    const i64 i0 = (t - pre[qi]) * kTB;
    if (m_bits) {
      u32* bm = reinterpret_cast<u32*>(reinterpret_cast<char*>(q.ht_tag) +
                                       dense_layout(n, m_bits).bm);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const i64 idx = i0 + j * 32 + lane;
        if (idx < n) bit_set(bm, ukey(q.mlist[idx]) - m_umin);
      }
      continue;
    }
    const TableView tv = table_view(q.ht_tag, q.ctr->mlog2, true);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const i64 idx = i0 + j * 32 + lane;
      if (idx < n && q.mlist[idx] == kEmpty) q_latch(q.ctr, b.st, PQ_ERR_RESERVED_KEY, idx);
    }
    insert_x4(tv, q.mlist, i0, n, [&](i64 k, u64 s) {
      *reinterpret_cast<longlong2*>(tv.rec + 2 * s) = make_longlong2(k, 0);  // {key, sum}
    });
  }
  finish(b.work, kPhMbuild);
}

// ------------------------------------------------------ dense dictionary ----
// Pointers of a plan's dense dictionary.
struct DenseView {
  const u32* bm;
  const u32* tdir;
  const unsigned short* wdir;
  u64 blocks;
};
__device__ __forceinline__ DenseView dense_view(const void* region, i64 c, u64 bits) {
  const DenseLayout L = dense_layout(c, bits);
  const char* base = reinterpret_cast<const char*>(region);
  DenseView v;
  v.bm = reinterpret_cast<const u32*>(base + L.bm);
  v.tdir = reinterpret_cast<const u32*>(base + L.tdir);
  v.wdir = reinterpret_cast<const unsigned short*>(base + L.wdir);
  v.blocks = (bits + 511) / 512;
  return v;
}

// Rank of bitmap bit idx (which is set): set bits before it -- the tile's
// prefix, the word's prefix within the tile, the bits below it in its word.
__device__ __forceinline__ u64 dense_rank(const DenseView& d, u64 idx, u64 keep) {
  const u64 wi = idx >> 5;
  u32 t, w;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;"
      : "=r"(t) : "l"(d.tdir + (idx >> 15)), "l"(keep));
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(w) : "l"(d.bm + wi), "l"(keep));
  const u32 wp = ld_keep_u16(d.wdir + wi, keep);
  return (u64)t + wp + __popc(w & ((1u << (idx & 31)) - 1u));
}

// Last index i in [lo, hi) with a[i] <= x, for a non-decreasing a with
// a[lo] <= x: a 16-ary search (15 independent loads per round, so that a
// round costs one memory latency).
template <typename T>
__device__ __forceinline__ u64 last_le(const T* a, u64 lo, u64 hi, u64 x) {
  while (hi - lo > 1) {
    const u64 step = (hi - lo + 15) / 16;
    u32 c = 0;
#pragma unroll
    for (int j = 1; j < 16; ++j) {
      const u64 p = lo + j * step;
      c += p < hi && (u64)a[p] <= x;
    }
    hi = min(hi, lo + (c + 1) * step);
    lo += c * step;
  }
  return lo;
}

// last_le with a first guess g: a window of 16 entries around g is read at
// once (one memory latency when the answer lies in it, as it does for keys
// spread evenly); otherwise the search goes on on the side the window shows.
template <typename T>
__device__ __forceinline__ u64 last_le_near(const T* a, u64 lo, u64 hi, u64 x, u64 g) {
  if (hi - lo <= 16) return last_le(a, lo, hi, x);
  g = min(max(g, lo), hi - 1);
  const u64 w0 = min(g > lo + 7 ? g - 7 : lo, hi - 16);
  u32 le = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) le += (u64)a[w0 + j] <= x;  // a prefix of the window
  if (le == 0) return last_le(a, lo, w0, x);
  if (le == 16 && w0 + 16 < hi) return last_le(a, w0 + 15, hi, x);
  return w0 + le - 1;
}

// Key of dense slot `rank` (< total, the distinct keys): the rank-th set
// bit.  The tile and the word are first looked for where an even spread of
// the keys puts them.
__device__ __forceinline__ i64 dense_key(const DenseView& d, u64 umin, u64 rank, u64 total) {
  const u64 tiles = (d.blocks + kRankTile - 1) / kRankTile;
  // First guesses in single precision (only where to look first: the
  // searches are exact from any guess).
  const u64 tg = total ? (u64)((float)rank / (float)total * (float)tiles) : 0;
  const u64 t = last_le_near(d.tdir, 0, tiles, rank, tg);  // tdir[tiles] = total > rank
  const u32 r = (u32)(rank - d.tdir[t]);
  const u64 words = d.blocks * 16, w_lo = t * kRankTile * 16,
            w_hi = min(words, (t + 1) * kRankTile * 16);
  const u32 tbits = (u32)(d.tdir[t + 1] - d.tdir[t]);
  const u64 wg = w_lo + (tbits ? (u64)((float)r / (float)tbits * (float)(w_hi - w_lo)) : 0);
  const u64 w0 = last_le_near(d.wdir, w_lo, w_hi, r, wg);
  u32 rr = r - d.wdir[w0];
  u32 x = d.bm[w0];
  for (; rr; --rr) x &= x - 1;
  const u64 u = umin + w0 * 32 + (u64)(__ffs(x) - 1);
  return (i64)(u ^ (1ULL << 63));
}

// Rank pass: one warp per tile of kRankTile blocks writes each block's set
// bits before it within the tile and the tile's total, and clears its share
// of the slot arrays (hit bits, sums, copy counts); the block that finishes
// last turns the tile totals into prefixes, writes the number of distinct
// keys and notes whether the members repeat keys.
__global__ void __launch_bounds__(256) k_plan_mrank(Batch b) {
  chain_begin();
  const i64* pre = b.dyn + 5 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31;
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhMrank);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const u64 bits = q.ctr->m_bits;
    const DenseLayout L = dense_layout((i64)q.ctr->mcount, bits);
    char* base = reinterpret_cast<char*>(q.ht_tag);
    const uint4* bm = reinterpret_cast<const uint4*>(base + L.bm);
    u32* tdir = reinterpret_cast<u32*>(base + L.tdir);
    unsigned short* wdir = reinterpret_cast<unsigned short*>(base + L.wdir);
    const u64 blocks = (bits + 511) / 512;
    const i64 lt = t - pre[qi];
    const u64 b0 = (u64)lt * kRankTile, b1 = min(blocks, b0 + kRankTile);
    {  // this tile's share of [hit, total), in 16-byte units
      const i64 units = (i64)(L.total - L.hit) / 16, tiles = pre[qi + 1] - pre[qi];
      const i64 u0 = units * lt / tiles, u1 = units * (lt + 1) / tiles;
      int4* z = reinterpret_cast<int4*>(base + L.hit);
      for (i64 u = u0 + lane; u < u1; u += 32) z[u] = make_int4(0, 0, 0, 0);
    }
    u32 run = 0;
    for (u64 j0 = b0; j0 < b1; j0 += 32) {
      const u64 j = j0 + lane;  // the lane's block: 16 words
      u32 c[16];
      u32 p = 0;
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        const uint4 v = j < b1 ? __ldcg(bm + j * 4 + qd) : make_uint4(0, 0, 0, 0);
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
      if (j < b1) {  // the block's 16 word prefixes, two 16-byte stores
        u32 pre = run + incl - p;
        u32 h[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const u32 lo = pre;
          pre += c[2 * x];
          h[x] = lo | (pre << 16);
          pre += c[2 * x + 1];
        }
        uint4* dst = reinterpret_cast<uint4*>(wdir + j * 16);
        dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
        dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
      }
      run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) tdir[lt] = run;  // the tile's total, a prefix after the scan
  }
  if (finish(b.work, kPhMrank)) {
    for (int qi = 0; qi < b.nq; ++qi) {  // exclusive scan of each dense plan's tile totals
      const PlanDev& q = b.q[qi];
      const u64 bits = q.ctr->m_bits;
      if (!bits) continue;
      u32* tdir = reinterpret_cast<u32*>(reinterpret_cast<char*>(q.ht_tag) +
                                         dense_layout((i64)q.ctr->mcount, bits).tdir);
      const i64 tiles = (i64)(((bits + 511) / 512 + kRankTile - 1) / kRankTile);
      __shared__ u32 s_carry;
      if (threadIdx.x == 0) s_carry = 0;
      __syncthreads();
      // Each thread takes 16 consecutive totals per pass (loaded together),
      // so a pass costs one round trip to memory.
      for (i64 t0 = 0; t0 < tiles; t0 += (i64)blockDim.x * 16) {
        const i64 tb = t0 + (i64)threadIdx.x * 16;
        u32 v[16], sum = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] = tb + j < tiles ? __ldcg(tdir + tb + j) : 0u;
          sum += v[j];
        }
        const u32 ex = block_exclusive_sum(sum);
        u32 run = s_carry + ex;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (tb + j < tiles) tdir[tb + j] = run;
          run += v[j];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += ex + sum;
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        tdir[tiles] = s_carry;
        q.ctr->m_distinct = s_carry;
        q.ctr->dup = s_carry != (u32)q.ctr->mcount ? 1 : 0;
      }
      __syncthreads();
    }
    block_prefix(b.dyn + 6 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      const QCtr* c = q.ctr;
      if (!c->m_bits || !c->dup) return 0;
      return q.m_static ? (q.n_m + q.m_tile - 1) / q.m_tile  // rescan M
                        : (i64)((c->mcount + kTB - 1) / kTB);
    });
  }
}

// Copies per key when the members repeat keys: count the members of each
// dense slot (the F probe multiplies a row's revenue by it).  With a key list
// (tiles of 128 entries) the keys come from it; with a static bitmap (tiles
// of M rows) the M rows are tested again (date, D-set) for their members.
__global__ void __launch_bounds__(256) k_plan_mdup(Batch b) {
  chain_begin();
  const i64* pre = b.dyn + 6 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31;
  const u64 keep = policy_keep();
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhMdup);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64 n = (i64)q.ctr->mcount;
    const DenseView dv = dense_view(q.ht_tag, n, q.ctr->m_bits);
    u32* cnt = reinterpret_cast<u32*>(reinterpret_cast<char*>(q.ht_tag) +
                                      dense_layout(n, q.ctr->m_bits).cnt);
    const u64 umin = q.ctr->m_umin;
    if (q.m_static) {
      const TableView dt = table_view(q.dset_tag, *q.dset_log2, false);
      const u64* dhdr = reinterpret_cast<const u64*>(q.dset_log2);
      const u64 d_umin = dhdr[1], d_bits = dhdr[2];
      const i64 r0 = (t - pre[qi]) * q.m_tile, r1 = min(q.n_m, r0 + q.m_tile);
      for (i64 r = r0 + lane; r < r1; r += 32) {
        if (!pass(q.pm, __ldg(q.m_date + r))) continue;
        const i64 dr = __ldg(q.m_dref + r);
        const u64 di = ukey(dr) - d_umin;
        const bool mem = d_bits ? di < d_bits && bit_test(dt.keybm, di, keep)
                                : set_contains(dt, dr, keep);
        const u64 idx = mem ? ukey(__ldg(q.m_key + r)) - umin : ~0ULL;
        if (idx < q.m_sb) atomicAdd(cnt + dense_rank(dv, idx, keep), 1u);
      }
      continue;
    }
    const i64 i0 = (t - pre[qi]) * kTB;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const i64 idx = i0 + j * 32 + lane;
      if (idx < n) atomicAdd(cnt + dense_rank(dv, ukey(q.mlist[idx]) - umin, keep), 1u);
    }
  }
  finish(b.work, kPhMdup);
}

// ----------------------------------------------------------------- fprobe ----
constexpr int kAggLog2 = 8;
constexpr int kAgg = 1 << kAggLog2;  // entries of a block's shared-memory aggregation table
constexpr int kH = 256;              // entries of a warp's hit ring
constexpr int kHF = 1024;            // entries of a warp's ring in the F scan

// What a probe needs besides the plan (kept small: it lives in registers
// across the scan loop; the table details are derived in the probe).
struct ProbeCtx {
  const i64* mkey;
  const i64* price;
  const signed char* disc;
  i64 base;
  u64 keep;
  int qi;  // plan index in the batch
};

// The fast commit of a plan (see PlanDev::rev_max), for `hits` hits.
__device__ __forceinline__ bool fast_commit(const PlanDev& q, u64 hits) {
  if (!q.rev_max) return false;
  // Largest multiplicity: 1 for a dense dictionary of distinct keys, else
  // the plan's M rows (a hash table may hold a key in many slots).
  const unsigned __int128 mult = q.ctr->m_bits && !q.ctr->dup ? 1 : (u64)max(q.n_m, (i64)1);
  return (unsigned __int128)hits * q.rev_max * mult < ((unsigned __int128)1 << 63);
}
__device__ __forceinline__ void red_add(i64* p, i64 v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_or(u32* p, u32 v) {
  asm volatile("red.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool add_overflows(i64 old, i64 v) {
  return (v > 0 && old > INT64_MAX - v) || (v < 0 && old < INT64_MIN - v);
}

// One probed F row: the M-table slot of its group and the revenue to add.
struct Hit {
  bool act;
  u64 slot;
  i64 v;
};

// Probe the M side with the key of F row base + r.  Dense dictionary: the
// slot is the rank of the key's bit (set: the caller tested it) and the
// multiplicity its copy count.  Hash table: count the slots holding the key
// (its multiplicity in M', found in the home bucket and, while buckets are
// full, the next ones) and take the first.  The row adds its exact revenue
// times the multiplicity to the group of that slot.
__device__ __forceinline__ Hit probe_row(const Batch& bt_, const ProbeCtx& c, u32 r) {
  const PlanDev& q = bt_.q[c.qi];
  Hit h = {false, 0, 0};
  const i64 row = c.base + r;
  const i64 k = __ldg(c.mkey + row);
  const i64 price = __ldg(c.price + row);  // loaded with the key: one round trip
  const i64 disc = __ldg(c.disc + row);
  i64 first = -1, mult = 0;
  if (q.ctr->m_bits) {
    const DenseView dv = dense_view(q.ht_tag, (i64)q.ctr->mcount, q.ctr->m_bits);
    first = (i64)dense_rank(dv, ukey(k) - q.ctr->m_umin, c.keep);
    mult = q.ctr->dup ? (i64)__ldg(reinterpret_cast<const u32*>(
                                       reinterpret_cast<const char*>(q.ht_tag) +
                                       dense_layout((i64)q.ctr->mcount, q.ctr->m_bits).cnt) +
                                   first)
                      : 1;
  } else {
    const TableView t = table_view(q.ht_tag, q.ctr->mlog2, true);
    const BucketTag bt = bucket_tag(k, t.g.shiftb);
    const unsigned v2 = bt.tag * 0x10001u;
    u64 b = bt.bucket;
    for (u64 p = 0; p <= t.g.bmask; ++p) {
      const uint4 w = ld_keep_v4u(t.tags + b * 8, c.keep);
      Mask8 m = match8(w, v2);
      while (any8(m)) {
        const int j = first8(m);
        const u64 slot = b * 8 + j;
        if (ld_keep(t.rec + 2 * slot, c.keep) == k) {
          if (first < 0) first = (i64)slot;
          ++mult;
        }
        drop8(m, j);
      }
      if (any8(match8(w, 0u))) break;
      b = (b + 1) & t.g.bmask;
    }
  }
  if (first < 0) return h;
  // Exact revenue: the product is formed in 128 bits so that a value outside
  // int64 is reported instead of wrapping.
  const __int128 v128 = (__int128)mult * ((__int128)price * (100 - disc));
  h.v = (i64)v128;
  if (v128 != (__int128)h.v) q_latch(q.ctr, bt_.st, PQ_ERR_OVERFLOW, k);
  h.act = true;
  h.slot = (u64)first;
  return h;
}

// Add v into the block's direct-mapped shared-memory table under key ak (plan
// and slot): the first key to reach an entry keeps it for the rest of the
// kernel, so the repeated hits of hot groups (skewed data) stay on chip.
// False when the entry belongs to another key.  (Measured on Zipf data: a
// 2048-entry table with 4-way probing was slower than this one.)
__device__ __forceinline__ bool agg_try(u64* akey, i64* asum, u64 ak, i64 v, bool& ovf,
                                        bool exact) {
  const u32 h = (u32)((ak * 0x9E3779B97F4A7C15ULL) >> (64 - kAggLog2));
  u64 cur = *(volatile u64*)&akey[h];
  if (cur == 0) {
    cur = atomicCAS((unsigned long long*)&akey[h], 0ULL, ak);
    if (cur == 0) cur = ak;
  }
  if (cur != ak) return false;
  if (exact) {
    const i64 old = (i64)atomicAdd((unsigned long long*)&asum[h], (unsigned long long)v);
    ovf = ovf || add_overflows(old, v);
  } else {
    atomicAdd((unsigned long long*)&asum[h], (unsigned long long)v);
  }
  return true;
}

// Where a plan's groups keep their sums and first-hit bits: the dense
// dictionary's arrays, or the hash table's records (sum in the second word).
struct GroupStore {
  u32* hit;
  i64* sums;
  int stride;
};
__device__ __forceinline__ GroupStore group_store(const PlanDev& q) {
  GroupStore g;
  if (q.ctr->m_bits) {
    const DenseLayout L = dense_layout((i64)q.ctr->mcount, q.ctr->m_bits);
    char* base = reinterpret_cast<char*>(q.ht_tag);
    g.hit = reinterpret_cast<u32*>(base + L.hit);
    g.sums = reinterpret_cast<i64*>(base + L.sums);
    g.stride = 1;
  } else {
    const TableView t = table_view(q.ht_tag, q.ctr->mlog2, true);
    g.hit = t.hit;
    g.sums = t.rec + 1;
    g.stride = 2;
  }
  return g;
}

// Warp-wide commit of per-lane sums (every lane calls; lanes with `act` add
// v to slot s of plan qi).  Lanes with the same plan and slot combine first
// (their lowest lane carries the exact total); that lane adds it to the
// block's shared table when `akey` is given and the entry is free or its own,
// else to the M table and sets the slot's first-hit bit (a reduction nobody
// waits for).  The groups are read from the first-hit bits by the top-k
// phase.  sc: the warp's 32-entry scratch.
__device__ __forceinline__ void commit_hits_g(const Batch& b, i64* sc, u64* akey, i64* asum,
                                              bool act, int qi, u64 s, i64 v,
                                              const GroupStore* gs, bool exact);
__device__ __forceinline__ void commit_hits(const Batch& b, i64* sc, u64* akey, i64* asum,
                                            bool act, int qi, u64 s, i64 v) {
  commit_hits_g(b, sc, akey, asum, act, qi, s, v, nullptr, true);
}
// As commit_hits, with the plan's group store already resolved (gs, for
// callers whose batch of 32 belongs to one plan; nullptr: look it up).
// exact = false (fast_commit holds): reductions with no overflow checks.
__device__ __forceinline__ void commit_hits_g(const Batch& b, i64* sc, u64* akey, i64* asum,
                                              bool act, int qi, u64 s, i64 v,
                                              const GroupStore* gs, bool exact) {
  const int lane = threadIdx.x & 31;
  const u64 ak = act ? ((u64)qi << 40) + s + 1 : 0;
  const u32 peers = __match_any_sync(kFull, ak);
  const bool lead = act && __ffs(peers) - 1 == lane;
  sc[lane] = v;
  __syncwarp();
  i64 tot = v;
  bool ovf = false;
  if (lead && peers != (1u << lane)) {
    __int128 acc = 0;
    for (u32 m = peers; m; m &= m - 1) acc += sc[__ffs(m) - 1];
    tot = (i64)acc;
    ovf = exact && acc != (__int128)tot;
  }
  __syncwarp();
  if (lead) {
    const PlanDev& q = b.q[qi];
    if (!(akey && agg_try(akey, asum, ak, tot, ovf, exact))) {
      const GroupStore g = gs ? *gs : group_store(q);
      red_or(g.hit + (s >> 5), 1u << (s & 31));
      if (exact) {
        const i64 old = (i64)atomicAdd((u64*)(g.sums + s * g.stride), (u64)tot);
        ovf = ovf || add_overflows(old, tot);
      } else {
        red_add(g.sums + s * g.stride, tot);
      }
    }
    if (ovf) q_latch(q.ctr, b.st, PQ_ERR_OVERFLOW, (i64)s);
  }
}

// Words of a plan's first-hit bitmap: dense slots, or hash-table slots.
__device__ __forceinline__ i64 topk_words(const PlanDev& q) {
  const i64 slots = q.ctr->m_bits ? (i64)q.ctr->mcount : (1LL << q.ctr->mlog2);
  return (slots + 31) >> 5;
}

// End of an F-probe kernel: flush the block's aggregated sums to the plans'
// tables; the block that finishes last sizes the top-k phase.
// Flush a block's shared aggregation table into the plans' groups; with
// `reset` the table is emptied for further use.
__device__ __forceinline__ void agg_flush(const Batch& b, u64* s_akey, i64* s_asum, i64* sc,
                                          bool reset = false) {
  __syncthreads();
  int used = 0;
  for (int i = threadIdx.x; i < kAgg; i += blockDim.x) used |= s_akey[i] != 0;
  for (int i0 = 0; __syncthreads_or(used) && i0 < kAgg; i0 += blockDim.x) {  // uniform
    const int i = i0 + threadIdx.x;
    const u64 ak = i < kAgg ? s_akey[i] : 0;
    commit_hits(b, sc, nullptr, nullptr, ak != 0, ak ? (int)((ak - 1) >> 40) : 0,
                (ak - 1) & ((1ULL << 40) - 1), ak ? s_asum[i] : 0);
    if (reset && ak) s_akey[i] = 0, s_asum[i] = 0;
  }
  __syncthreads();
}

__device__ __forceinline__ void fprobe_epilogue(const Batch& b, u64* s_akey, i64* s_asum,
                                                i64* sc) {
  agg_flush(b, s_akey, s_asum, sc);
  if (finish(b.work, kPhFprobe)) {
    block_prefix(b.dyn + 4 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      q.out->status = q.ctr->status;
      q.out->reserved = 0;
      // A streamed F table probes chunk by chunk (or buffer by buffer).
      q.ctr->hits_total += (u64)ld_count(&q.ctr->hcount);
      q.ctr->hcount = 0;
      q.out->hits = (i64)q.ctr->hits_total;
      const i64 w = topk_words(q);
      return max((i64)1, (w + topk_tile_words_w(w) - 1) / topk_tile_words_w(w));
    });
  }
}

// Partitioned plans, in the last block of the partition pass: each bucket's
// count becomes its write cursor (exclusive scan, part[P] = total matched
// hits), and the tile counts of the scatter pass (kPT hits per block tile)
// and of the aggregation pass (kAT records per warp tile) go to their
// prefixes.
__device__ __forceinline__ void part_sizes(const Batch& b) {
  __shared__ u64 s_carry;
  for (int qi = 0; qi < b.nq; ++qi) {
    const PlanDev& q = b.q[qi];
    if (!q.part_log2) continue;
    const int P = 1 << q.part_log2;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int p0 = 0; p0 < P; p0 += (int)blockDim.x) {
      const int p = p0 + (int)threadIdx.x;
      const u64 v = p < P ? __ldcg(q.part + p) : 0;
      const u32 ex = block_exclusive_sum((u32)v);  // a plan holds < 2^32 hits
      const u64 base = s_carry;
      if (p < P) q.part[p] = base + ex;
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) s_carry = base + ex + v;
      __syncthreads();
    }
    if (threadIdx.x == 0) q.part[P] = s_carry;
    __syncthreads();
  }
  block_prefix(b.dyn + 9 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
    const PlanDev& q = b.q[qi];
    return q.part_log2 ? (ld_count(&q.ctr->hcount) + kPT - 1) / kPT : 0;
  });
  block_prefix(b.dyn + 10 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
    const PlanDev& q = b.q[qi];
    return q.part_log2 ? (i64)(__ldcg(q.part + (1 << q.part_log2)) + 8 * kAT - 1) / (8 * kAT)
                       : 0;
  });
}

// F scan: warp tiles of F rows (up to 2048), 128 per step (lane l: rows
// 4l .. 4l+3).  Pipeline per lane: date2 is read two steps ahead, mkey one
// ahead (only for 4-row groups with a passing row), the key-range bitmap
// words of the passing keys are loaded in the step the keys arrive and
// tested in the next.  Rows whose bit is set (the join hits) enter the
// warp's ring as rows of the plan; runs of 512 leave for the plan's hit list
// with one atomic reservation each.  With no bitmap every passing row is a
// hit candidate and the probe decides.  The ring carries over from tile to
// tile of the same plan.  The kernel does nothing else, so that it stays
// small enough for four blocks per SM.
// BUF: some plan of the batch buffers its hits (dynamic buffering of a
// streamed F table): compiled separately, so that the resident scan keeps
// its registers.
template <bool VEC, bool BUF>
__global__ void __launch_bounds__(256, 4) k_plan_fscan(Batch b) {
  chain_begin();
  __shared__ u32 s_hr[8][kHF];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u32* hr = s_hr[warp];
  const u64 keep = policy_keep(), strm = policy_stream();
  const bool ov = b.ov.table == 3;
  const i64 total = ov ? b.ov.tiles : b.tF[b.nq];
  int cq = -1;  // plan of the rows in the ring
  u32 hh = 0, ht = 0;
  auto flush = [&](u32 cnt) {  // cnt entries from hh to plan cq's hit list
    const PlanDev& q = b.q[cq];
    u64 at = 0;
    if (lane == 0) at = atomicAdd(&q.ctr->hcount, (u64)cnt);
    at = __shfl_sync(kFull, at, 0);
    if (BUF && q.hb_cap) {  // buffered: the hit's columns, not its row
      const i64* mk = ov ? (const i64*)b.ov.p[0] : q.f_mkey;
      const i64* pr = ov ? (const i64*)b.ov.p[1] : q.f_price;
      const signed char* ds = ov ? (const signed char*)b.ov.p[2] : q.f_disc;
      for (u32 j = lane; j < cnt; j += 32) {
        const u32 row = hr[(hh + j) & (kHF - 1)];
        if (at + j < q.hb_cap) {  // the host sizes the buffer for a whole chunk
          q.hb_key[at + j] = __ldg(mk + row);
          q.hb_price[at + j] = __ldg(pr + row);
          q.hb_disc[at + j] = __ldg(ds + row);
        }
      }
    } else {
      for (u32 j = lane; j < cnt; j += 32) q.hlist[at + j] = hr[(hh + j) & (kHF - 1)];
    }
    hh += cnt;
    __syncwarp();
  };
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhFscan);
    if (t >= total) break;
    const int qi = ov ? 0 : find_q(b.tF, b.nq, t);
    const PlanDev& q = b.q[qi];
    if (qi != cq) {
      if (cq >= 0 && ht != hh) flush(ht - hh);
      cq = qi;
      hh = ht = 0;
    }
    const i64 n = ov ? b.ov.n : q.n_f;
    const int tile = ov ? b.ov.tile : q.f_tile;
    const i64 base = (t - (ov ? 0 : b.tF[qi])) * tile;
    // The tile's rows, addressed with 32-bit offsets.
    const i64* f_mkey = (ov ? (const i64*)b.ov.p[0] : q.f_mkey) + base;
    const int* f_date = (ov ? (const int*)b.ov.p[3] : q.f_date) + base;
    const u64 bm_umin = q.ctr->m_umin, bm_bits = q.ctr->m_bits;
    const u32* bm = bm_bits ? reinterpret_cast<const u32*>(
                                  reinterpret_cast<const char*>(q.ht_tag) +
                                  dense_layout((i64)q.ctr->mcount, bm_bits).bm)
                            : nullptr;
    const Pred32 pf = to32(q.pf);
    const int lim = (int)min(n - base, (i64)tile);
    const int iters = (lim + 127) / 128;
    auto append_hits = [&](u32 hits, int it, bool pair) {
      if (__any_sync(kFull, hits)) {
        __syncwarp();
        ht += ring_append(hits, ht, [&](int s, u32 pos) {
          const int off = pair ? 2 * lane + (s & 1) + (s >> 1) * 64 : 4 * lane + s;
          hr[pos & (kHF - 1)] = (u32)(base + it * 128 + off);
        });
        __syncwarp();
        if (ht - hh >= 512) flush(512);
      }
    };
    // The step loop, compiled for full tiles of aligned columns (no row
    // limits) and for a bitmap that exists, and in general.
    auto run = [&](auto full_c, auto fast_c, auto pair_c) {
      constexpr bool FULL = decltype(full_c)::value, FAST = decltype(fast_c)::value;
      constexpr bool PAIR = decltype(pair_c)::value;
      // e0: the step's first row + the lane's first row (4l, or 2l).
      const int r0 = PAIR ? 2 * lane : 4 * lane;
      auto ld_d = [&](int e0) -> int4 {
        if (PAIR) {
          const int2 a = ld_stream_v2i(f_date + e0, strm), c = ld_stream_v2i(f_date + e0 + 64, strm);
          return make_int4(a.x, a.y, c.x, c.y);
        }
        return FULL ? ld_stream_v4(f_date + e0, strm) : load_i32x4<VEC>(f_date, e0, lim - e0, strm);
      };
      auto ld_k = [&](int e0, u32 bits, i64 v[4]) {
        if (PAIR) {
          if (bits & 3u) {
            const longlong2 x = ld_stream_v2(f_mkey + e0, strm);
            v[0] = x.x, v[1] = x.y;
          }
          if (bits & 12u) {
            const longlong2 y = ld_stream_v2(f_mkey + e0 + 64, strm);
            v[2] = y.x, v[3] = y.y;
          }
        } else if (FULL) {
          const longlong2 x = ld_stream_v2(f_mkey + e0, strm), y = ld_stream_v2(f_mkey + e0 + 2, strm);
          v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
        } else {
          load_i64x4<VEC>(f_mkey, e0, lim - e0, bits, strm, v);
        }
      };
      auto p4 = [&](int4 d, int e0) { return pass4(pf, d, FULL ? 4 : lim - e0); };
      int4 dB = ld_d(r0);
      int4 dC = iters > 1 ? ld_d(128 + r0) : make_int4(0, 0, 0, 0);
      u32 bA = p4(dB, r0);
      i64 mA[4] = {0, 0, 0, 0};
      if (bA) ld_k(r0, bA, mA);
      dB = dC;
      if (iters > 2) dC = ld_d(256 + r0);
      BmStage wP;
      wP.w[0] = wP.w[1] = wP.w[2] = wP.w[3] = 0;
      wP.sh = 0;
      for (int it = 0; it < iters; ++it) {
        const int rel1 = (it + 1) * 128 + r0;
        u32 bB = 0;
        i64 mB[4] = {0, 0, 0, 0};
        if (it + 1 < iters) {
          bB = p4(dB, rel1);
          if (bB) ld_k(rel1, bB, mB);
        }
        dB = dC;
        if (it + 3 < iters) dC = ld_d((it + 3) * 128 + r0);
        BmStage wN;
        if (FAST) bm_issue_fast(wN, bm, bm_umin ^ 0x8000000000000000ULL, bm_bits, bA, mA, keep);
        else bm_issue(wN, bm, bm_umin, bm_bits, bA, mA, keep);
        if (it > 0) append_hits(bm_hits(wP), it - 1, PAIR);
        wP = wN;
        bA = bB;
#pragma unroll
        for (int s = 0; s < 4; ++s) mA[s] = mB[s];
      }
      append_hits(bm_hits(wP), iters - 1, PAIR);
    };
    using T = std::true_type;
    using F = std::false_type;
    if (VEC && lim == iters * 128) {
      if (bm_bits && q.f_pair && !ov) run(T{}, T{}, T{});
      else if (bm_bits) run(T{}, T{}, F{});
      else run(T{}, F{}, F{});
    } else {
      if (bm_bits) run(F{}, T{}, F{});
      else run(F{}, F{}, F{});
    }
  }
  if (cq >= 0 && ht != hh) flush(ht - hh);
  if (finish(b.work, kPhFscan)) {
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    block_prefix(b.dyn + 7 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      QCtr* c = q.ctr;
      const i64 h = ld_count(&c->hcount);
      if (q.hb_cap && h > (i64)q.hb_cap) q_latch(c, b.st, PQ_ERR_CAPACITY, h);
      // Hits per probe tile: about two tiles per warp of this grid, in
      // multiples of 32, between 64 and 4096.
      i64 tl = (h / (2 * warps) + 31) / 32 * 32;
      tl = tl < 64 ? 64 : tl > 4096 ? 4096 : tl;
      c->hp_tile = tl;
      return q.part_log2 ? 0 : (h + tl - 1) / tl;  // partitioned: fpart .. fagg
    });
    block_prefix(b.dyn + 8 * (b.nq + 1), b.nq, [&](int qi) -> i64 {
      const PlanDev& q = b.q[qi];
      return q.part_log2 ? (ld_count(&q.ctr->hcount) + kPT - 1) / kPT : 0;
    });
  }
}

// F probe: warp tiles of the hit list (hp_tile rows), 32 per batch: each
// lane re-reads its row's key, price and discount, finds the group (dense:
// rank of the key's bit; hash: probe), and the batch commits (lanes of the
// same group combined, then the group's sum and first-hit bit in global
// memory).  A plan with at least 2048 hits per block of the grid (skewed or
// pass-all data, where groups repeat within a block) first tries the
// block's shared aggregation table.
__global__ void __launch_bounds__(256) k_plan_fprobe(Batch b) {
  chain_begin();
  __shared__ u64 s_akey[kAgg];
  __shared__ i64 s_asum[kAgg];
  __shared__ i64 s_sc[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  i64* sc = s_sc[warp];
  for (int i = threadIdx.x; i < kAgg; i += blockDim.x) s_akey[i] = 0, s_asum[i] = 0;
  __syncthreads();
  const u64 agg_min = (u64)gridDim.x * 2048;
  const u64 keep = policy_keep();
  const bool ov = b.ov.table == 3;
  const i64* pre = b.dyn + 7 * (b.nq + 1);
  const i64 total = pre[b.nq];
  WarpClaim wc;
  while (true) {
    const i64 t = wc.next(b.work, kPhFprobe);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    ProbeCtx pc;
    const bool buffered = q.hb_cap != 0;  // hits are buffer entries, not rows
    pc.mkey = buffered ? q.hb_key : ov ? (const i64*)b.ov.p[0] : q.f_mkey;
    pc.price = buffered ? q.hb_price : ov ? (const i64*)b.ov.p[1] : q.f_price;
    pc.disc = buffered ? q.hb_disc : ov ? (const signed char*)b.ov.p[2] : q.f_disc;
    pc.base = 0;
    pc.keep = keep;
    pc.qi = qi;
    QCtr* const c = q.ctr;
    const i64 tl = c->hp_tile, h = (i64)c->hcount;
    const i64 i0 = (t - pre[qi]) * tl, i1 = min(h, i0 + tl);
    u64* const akey = (u64)h >= agg_min ? s_akey : nullptr;
    const u64 m_bits = c->m_bits;
    if (m_bits) {
      // Dense dictionary, with the plan's constants held in registers for
      // the whole tile: slot = rank of the key's bit (three loads), the
      // multiplicity only when the members repeat keys.
      const i64 mc = (i64)c->mcount;
      const DenseView dv = dense_view(q.ht_tag, mc, m_bits);
      const DenseLayout L = dense_layout(mc, m_bits);
      char* const gb = reinterpret_cast<char*>(q.ht_tag);
      const u32* const cnt = c->dup ? reinterpret_cast<const u32*>(gb + L.cnt) : nullptr;
      GroupStore g;
      g.hit = reinterpret_cast<u32*>(gb + L.hit);
      g.sums = reinterpret_cast<i64*>(gb + L.sums);
      g.stride = 1;
      const u64 umin = c->m_umin;
      const bool exact = !fast_commit(q, (u64)h);
      for (i64 i = i0; i < i1; i += 32) {
        const bool act = i + lane < i1;
        u64 slot = 0;
        i64 v = 0;
        if (act) {
          const i64 row = buffered ? i + lane : (i64)__ldg(q.hlist + i + lane);
          const i64 k = __ldg(pc.mkey + row);
          const i64 price = __ldg(pc.price + row);
          const i64 disc = __ldg(pc.disc + row);
          slot = dense_rank(dv, ukey(k) - umin, keep);
          const i64 mult = cnt ? (i64)__ldg(cnt + slot) : 1;
          if (exact) {
            const __int128 v128 = (__int128)mult * ((__int128)price * (100 - disc));
            v = (i64)v128;
            if (v128 != (__int128)v) q_latch(c, b.st, PQ_ERR_OVERFLOW, k);
          } else {
            v = mult * (price * (100 - disc));  // fits: fast_commit's bound
          }
        }
        commit_hits_g(b, sc, akey, s_asum, act, qi, slot, v, &g, exact);
      }
      continue;
    }
    const bool exact = !fast_commit(q, (u64)h);
    for (i64 i = i0; i < i1; i += 32) {
      const bool act = i + lane < i1;
      Hit x = {false, 0, 0};
      if (act) x = probe_row(b, pc, buffered ? (u32)(i + lane) : __ldg(q.hlist + i + lane));
      commit_hits_g(b, sc, akey, s_asum, x.act, qi, x.slot, x.v, nullptr, exact);
    }
  }
  fprobe_epilogue(b, s_akey, s_asum, sc);
}

// Probe of one hit against a dense dictionary, with the plan's constants in
// registers: slot = rank of the key's bit, revenue times the key's copies in
// M' (cnt: copy counts, or null when the members do not repeat keys), formed
// in 128 bits (an int64 overflow is latched).
struct DenseProbe {
  DenseView dv;
  const u32* cnt;
  u64 umin;
};
__device__ __forceinline__ DenseProbe dense_probe(const PlanDev& q) {
  const QCtr* c = q.ctr;
  const i64 mc = (i64)c->mcount;
  DenseProbe p;
  p.dv = dense_view(q.ht_tag, mc, c->m_bits);
  p.cnt = c->dup ? reinterpret_cast<const u32*>(reinterpret_cast<const char*>(q.ht_tag) +
                                                dense_layout(mc, c->m_bits).cnt)
                 : nullptr;
  p.umin = c->m_umin;
  return p;
}
__device__ __forceinline__ i64 dense_hit(const DenseProbe& p, const ProbeCtx& pc, const Batch& b,
                                         QCtr* ctr, i64 row, u64* slot) {
  const i64 k = __ldg(pc.mkey + row);
  const i64 price = __ldg(pc.price + row);
  const i64 disc = __ldg(pc.disc + row);
  *slot = dense_rank(p.dv, ukey(k) - p.umin, pc.keep);
  const i64 mult = p.cnt ? (i64)__ldg(p.cnt + *slot) : 1;
  const __int128 v128 = (__int128)mult * ((__int128)price * (100 - disc));
  const i64 v = (i64)v128;
  if (v128 != (__int128)v) q_latch(ctr, b.st, PQ_ERR_OVERFLOW, k);
  return v;
}

// Group slots of a plan: dense dictionary members, or hash-table slots.
__device__ __forceinline__ u64 plan_slots(const QCtr* c) {
  return c->m_bits ? c->mcount : (1ULL << c->mlog2);
}

// Partition pass of a partitioned plan (the radix partition ahead of the
// exchange, Sec. 3.1, kept on one GPU), 1 of 2: block tiles of kPT hits.
// Every hit is probed once (group slot and revenue, as in the F probe); the
// slot replaces the row in the hit list and the revenue goes to pval0, both
// in hit order (coalesced), a hit that misses the hash table gets slot ~0;
// each matched hit is counted into its bucket (slot >> shift) in a block
// histogram in shared memory, flushed to the plan's bucket counters when
// the block moves to another plan and at the end.  The last block turns the
// counts into bucket cursors (part_sizes).
__global__ void __launch_bounds__(256) k_plan_fpart(Batch b) {
  chain_begin();
  constexpr int kPmax = 1 << kMaxPartLog2;
  __shared__ u32 s_hist[kPmax];
  __shared__ i64 s_t;
  const u64 keep = policy_keep();
  const bool ov = b.ov.table == 3;
  const i64* pre = b.dyn + 8 * (b.nq + 1);
  const i64 total = pre[b.nq];
  for (int p = threadIdx.x; p < kPmax; p += blockDim.x) s_hist[p] = 0;
  __syncthreads();
  int cq = -1;  // plan whose counts s_hist holds
  auto flush = [&]() {
    __syncthreads();
    if (cq >= 0) {
      const PlanDev& q = b.q[cq];
      for (int p = threadIdx.x; p < (1 << q.part_log2); p += blockDim.x) {
        const u32 c = s_hist[p];
        if (c) {
          atomicAdd(reinterpret_cast<unsigned long long*>(q.part + p), (unsigned long long)c);
          s_hist[p] = 0;
        }
      }
    }
    __syncthreads();
  };
  BlockClaim bc;
  while (true) {
    const i64 t = bc.next(b.work, kPhFpart, &s_t);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    if (qi != cq) flush(), cq = qi;  // block-uniform
    const PlanDev& q = b.q[qi];
    QCtr* const c = q.ctr;
    const int shift = part_shift(plan_slots(c), q.part_log2);
    ProbeCtx pc;
    pc.mkey = ov ? (const i64*)b.ov.p[0] : q.f_mkey;
    pc.price = ov ? (const i64*)b.ov.p[1] : q.f_price;
    pc.disc = ov ? (const signed char*)b.ov.p[2] : q.f_disc;
    pc.base = 0;
    pc.keep = keep;
    pc.qi = qi;
    const i64 i0 = (t - pre[qi]) * kPT, i1 = min((i64)c->hcount, i0 + kPT);
    if (c->m_bits) {
      const DenseProbe dp = dense_probe(q);
      for (i64 i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        u64 slot;
        const i64 v = dense_hit(dp, pc, b, c, __ldcg(q.hlist + i), &slot);
        q.hlist[i] = (u32)slot;
        q.pval0[i] = v;
        atomicAdd(&s_hist[slot >> shift], 1u);
      }
    } else {
      for (i64 i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const Hit x = probe_row(b, pc, __ldcg(q.hlist + i));
        q.hlist[i] = x.act ? (u32)x.slot : ~0u;
        q.pval0[i] = x.v;
        if (x.act) atomicAdd(&s_hist[x.slot >> shift], 1u);
      }
    }
  }
  flush();
  if (finish(b.work, kPhFpart)) part_sizes(b);
}

// Partition pass, 2 of 2: block tiles of kPT hits in hit order.  The block
// counts its matched hits per bucket in shared memory, claims one run per
// bucket from the bucket's cursor, orders the tile's records by bucket in
// shared memory and writes every run with consecutive threads on
// consecutive records.  Record order inside a bucket is unspecified (the
// sums are exact in any order).
__global__ void __launch_bounds__(256) k_plan_fscatter(Batch b) {
  chain_begin();
  constexpr int kPmax = 1 << kMaxPartLog2;
  constexpr int kPer = kPT / 256;
  __shared__ u32 s_cnt[kPmax];  // the tile's records per bucket, then their offsets
  __shared__ u64 s_go[kPmax];   // global position of the tile's run of each bucket
  __shared__ u32 s_slot[kPT];
  __shared__ i64 s_val[kPT];
  __shared__ unsigned short s_bk[kPT];
  __shared__ i64 s_t;
  const i64* pre = b.dyn + 9 * (b.nq + 1);
  const i64 total = pre[b.nq];
  BlockClaim bc;
  while (true) {
    const i64 t = bc.next(b.work, kPhFscatter, &s_t);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    QCtr* const c = q.ctr;
    const int P = 1 << q.part_log2;
    const int shift = part_shift(plan_slots(c), q.part_log2);
    const i64 i0 = (t - pre[qi]) * kPT;
    const int n = (int)min((i64)kPT, (i64)c->hcount - i0);
    for (int p = threadIdx.x; p < P; p += blockDim.x) s_cnt[p] = 0;
    __syncthreads();
    u32 slot[kPer], bl[kPer];  // bl: bucket << 16 | rank within the bucket's run
    i64 val[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int idx = j * 256 + (int)threadIdx.x;
      slot[j] = idx < n ? __ldcs(q.hlist + i0 + idx) : ~0u;
      val[j] = idx < n ? __ldcs(q.pval0 + i0 + idx) : 0;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const u32 bk = slot[j] != ~0u ? slot[j] >> shift : 0u;
      bl[j] = slot[j] != ~0u ? bk << 16 | atomicAdd(&s_cnt[bk], 1u) : ~0u;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
      const u32 cn = s_cnt[p];
      s_go[p] = cn ? atomicAdd(reinterpret_cast<unsigned long long*>(q.part + p),
                               (unsigned long long)cn)
                   : 0;
    }
    u32 m = 0;  // matched records of the tile
    {           // exclusive scan of the tile's bucket counts (P <= 4 * 256)
      u32 v[4], sum = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = (int)threadIdx.x * 4 + j;
        v[j] = p < P ? s_cnt[p] : 0u;
        sum += v[j];
      }
      u32 run = block_exclusive_sum(sum);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = (int)threadIdx.x * 4 + j;
        if (p < P) s_cnt[p] = run;
        run += v[j];
      }
      __shared__ u32 s_m;
      if (threadIdx.x == blockDim.x - 1) s_m = run;
      __syncthreads();
      m = s_m;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (bl[j] != ~0u) {
        const u32 bk = bl[j] >> 16, at = s_cnt[bk] + (bl[j] & 0xFFFFu);
        s_slot[at] = slot[j];
        s_val[at] = val[j];
        s_bk[at] = (unsigned short)bk;
      }
    }
    __syncthreads();
    const u64 end = q.part[P];  // matched hits of the plan: the records' end
    for (int i = threadIdx.x; i < (int)m; i += blockDim.x) {
      const u32 bk = s_bk[i];
      const u64 g = s_go[bk] + (u64)(i - (int)s_cnt[bk]);
      if (g < end) {
        q.pslot[g] = s_slot[i];
        q.pval[g] = s_val[i];
      } else {  // bucket sizes disagree with the counts: never written out of bounds
        q_latch(c, b.st, PQ_ERR_CAPACITY, (i64)g);
      }
    }
    __syncthreads();
  }
  finish(b.work, kPhFscatter);
}

// Aggregation pass of a partitioned plan: block tiles of 8 * kAT
// partitioned records (each warp takes kAT of them), claimed in order, so
// that the GPU sweeps the buckets one after another and the group sums of
// the buckets in work stay in L2 (a bucket's groups are one range of the
// group arrays).  Records of the same group in a batch of 32 combine first;
// for hit-heavy plans the block's shared aggregation table takes the
// repeated groups of the tile (skewed data: the hot keys of the bucket in
// work), and is flushed and emptied at the end of every tile, so that each
// region of the sweep has the table to itself.
__global__ void __launch_bounds__(256) k_plan_fagg(Batch b) {
  chain_begin();
  __shared__ u64 s_akey[kAgg];
  __shared__ i64 s_asum[kAgg];
  __shared__ i64 s_sc[8][32];
  __shared__ i64 s_t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  i64* sc = s_sc[warp];
  for (int i = threadIdx.x; i < kAgg; i += blockDim.x) s_akey[i] = 0, s_asum[i] = 0;
  __syncthreads();
  const u64 agg_min = (u64)gridDim.x * 2048;
  const i64* pre = b.dyn + 10 * (b.nq + 1);
  const i64 total = pre[b.nq];
  BlockClaim bc;
  while (true) {
    const i64 t = bc.next(b.work, kPhFagg, &s_t);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const i64 h = (i64)q.part[1 << q.part_log2];  // matched hits (part_sizes)
    const i64 i0 = (t - pre[qi]) * (8 * kAT) + warp * kAT, i1 = min(h, i0 + kAT);
    const bool agg = (u64)h >= agg_min;
    // Slots of the plan's group arrays: a record outside them (which the
    // partition pass never writes) is reported, not added.
    const u64 nslots = plan_slots(q.ctr);
    const GroupStore g = group_store(q);
    const bool exact = !fast_commit(q, (u64)q.ctr->hcount);
    for (i64 i = i0; i < i1; i += 32) {
      const i64 idx = i + lane;
      const u32 sl = idx < i1 ? __ldcs(q.pslot + idx) : ~0u;
      const i64 v = idx < i1 ? __ldcs(q.pval + idx) : 0;
      const bool ok = sl != ~0u && (u64)sl < nslots;
      if (sl != ~0u && !ok) q_latch(q.ctr, b.st, PQ_ERR_CAPACITY, (i64)sl);
      commit_hits_g(b, sc, agg ? s_akey : nullptr, s_asum, ok, qi, sl, v, &g, exact);
    }
    if (agg) agg_flush(b, s_akey, s_asum, sc, true);  // block-uniform: one plan per tile
  }
  agg_flush(b, s_akey, s_asum, sc);
  finish(b.work, kPhFagg);
}

// ------------------------------------------------------------------- topk ----
// One pass over the M table's first-hit bitmap, tiled in block tiles
// (topk_tile_words; each of a block's 4 warps takes a quarter).  A warp reads
// 8 steps of 32 words (one per lane and step) at a time, writes the slots of
// their set bits into its shared-memory ring, and reads the ring's records
// 256 at a time (8 in flight per lane) into its top-K list.  A block merges
// its warps' lists in shared memory and stores the tile's sorted list; the
// block that finishes a plan's last tile merges the tiles' lists and writes
// the result with the group count.
constexpr int kTKR = 2048;  // entries of a top-k warp's slot ring
constexpr int kTKW = 4;     // warps per top-k block

struct KS {
  i64 k, s;
  bool v;
};
// Output order on (key, sum) records: valid first, then sum desc, key asc.
__device__ __forceinline__ bool ks_before(const KS& a, const KS& b) {
  return a.v && (!b.v || tk_before(a.k, a.s, b.k, b.s));
}

// Scan warp w's quarter of block tile lt of a table: calls on(KS) for 256
// ring records at a time (each lane gets 8: invalid ones have v = false);
// returns the number of set bits.
// A plan's groups for top-k: the first-hit bitmap and, per slot, the record
// {key, sum} of the hash table or the dense sum (the slot standing for the
// key: slots follow key order).
struct TopkSrc {
  const u32* hit;
  const longlong2* rec;
  const i64* sums;
  i64 words;
  bool dense;
};
__device__ __forceinline__ TopkSrc topk_src(const PlanDev& q) {
  TopkSrc t;
  t.dense = q.ctr->m_bits != 0;
  if (t.dense) {
    const DenseLayout L = dense_layout((i64)q.ctr->mcount, q.ctr->m_bits);
    const char* base = reinterpret_cast<const char*>(q.ht_tag);
    t.hit = reinterpret_cast<const u32*>(base + L.hit);
    t.rec = nullptr;
    t.sums = reinterpret_cast<const i64*>(base + L.sums);
  } else {
    const TableView tv = table_view(q.ht_tag, q.ctr->mlog2, true);
    t.hit = tv.hit;
    t.rec = reinterpret_cast<const longlong2*>(tv.rec);
    t.sums = nullptr;
  }
  t.words = topk_words(q);
  return t;
}
// The key of an output entry: dense entries carry their slot.
__device__ __forceinline__ i64 topk_out_key(const PlanDev& q, bool dense, i64 k) {
  if (!dense) return k;
  return dense_key(dense_view(q.ht_tag, (i64)q.ctr->mcount, q.ctr->m_bits), q.ctr->m_umin,
                   (u64)k, q.ctr->m_distinct);
}

template <typename On>
__device__ __forceinline__ u64 tk_scan(const TopkSrc& src, i64 tw, i64 lt, u32* ring, On on) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const i64 words = src.words;
  const i64 ww = tw / kTKW;
  const i64 w0 = lt * tw + warp * ww, w1 = min(words, w0 + ww);
  u32 head = 0, tail = 0;
  u64 groups = 0;
  auto drain = [&](u32 cnt) {  // cnt <= 256 entries from head
    KS r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const u32 j = u * 32 + lane;
      const u32 slot = j < cnt ? ring[(head + j) & (kTKR - 1)] : 0u;
      const longlong2 x = j >= cnt    ? make_longlong2(0, 0)
                          : src.rec   ? src.rec[slot]
                                      : make_longlong2((i64)slot, src.sums[slot]);
      r[u].k = x.x, r[u].s = x.y, r[u].v = j < cnt;
    }
    on(r);
    head += cnt;
    __syncwarp();
  };
  for (i64 w = w0; w < w1; w += 256) {
    u32 wb[8];  // 8 steps of bitmap words in flight
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const i64 wi = w + u * 32 + lane;
      wb[u] = wi < w1 ? __ldcg(src.hit + wi) : 0u;
    }
#pragma unroll 1
    for (int u = 0; u < 8; ++u) {
      u32 bits = wb[0];
#pragma unroll
      for (int x = 0; x < 7; ++x) wb[x] = wb[x + 1];  // static indices only
      const u32 c = __popc(bits);
      groups += c;
      u32 incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const u32 sb = (u32)(w + u * 32 + lane) * 32;
      u32 pos = tail + incl - c;
      while (bits) {
        const int j = __ffs(bits) - 1;
        bits &= bits - 1;
        ring[pos++ & (kTKR - 1)] = sb + j;
      }
      tail += __shfl_sync(kFull, incl, 31);
      __syncwarp();
      while (tail - head >= 256) drain(256);
    }
  }
  if (tail - head) drain(tail - head);
  return groups;
}

// K rounds of the last tile's merge (one warp): lane l owns tiles l + 32 j
// (j < kTKP / 32) and keeps their heads in registers; a round takes the best
// head of the warp (warp max reductions over the record's order value, 32
// bits at a time, until one lane is left), records it, and the winner moves
// that tile's head on.  lk / ls: the lists (K entries per tile, shared or
// global memory), lc: their lengths.  Entry n goes to f_k / f_s[n], and
// f_n (shared) then counts the entries out, by a release store that the
// converting warp's acquire loads pair with.  Returns the number of entries.
template <typename LoadK, typename LoadS>
__device__ __forceinline__ int topk_merge_rounds(int K, int parts, const int* lc, LoadK lk,
                                                 LoadS ls, i64* f_k, i64* f_s, int* f_n) {
  constexpr int J = kTKP / 32;
  const int lane = threadIdx.x & 31;
  i64 hk[J], hs[J];
  int pos[J], len[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int i = lane + 32 * j;
    len[j] = i < parts ? lc[i] : 0;
    pos[j] = 0;
    hk[j] = len[j] ? lk((i64)i * K) : 0;
    hs[j] = len[j] ? ls((i64)i * K) : 0;
  }
  auto best = [&](int& jb) {
    jb = -1;
    i64 ck = 0, cs = 0;
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (pos[j] < len[j] && (jb < 0 || ks_bef(hk[j], hs[j], ck, cs))) jb = j, ck = hk[j], cs = hs[j];
  };
  int jb;
  best(jb);
  int n = 0;
  for (; n < K; ++n) {
    u32 act = __ballot_sync(kFull, jb >= 0);
    if (!act) break;
    i64 bk = 0, bs = 0;
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (j == jb) bk = hk[j], bs = hs[j];
    // Order value: sum (signed order) then key (smaller first), as 4 words.
    const u64 hi = (u64)bs ^ (1ULL << 63), lo = ~((u64)bk ^ (1ULL << 63));
    const u32 w[4] = {(u32)(hi >> 32), (u32)hi, (u32)(lo >> 32), (u32)lo};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (__popc(act) == 1) break;
      const bool in = (act >> lane) & 1u;
      const u32 m = __reduce_max_sync(kFull, in ? w[j] : 0u);
      act &= __ballot_sync(kFull, in && w[j] == m);
    }
    if (lane == __ffs(act) - 1) {
      f_k[n] = bk, f_s[n] = bs;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (j == jb) {
          ++pos[j];
          if (pos[j] < len[j]) {
            const i64 e = (i64)(lane + 32 * j) * K + pos[j];
            hk[j] = lk(e), hs[j] = ls(e);
          }
        }
      best(jb);
    }
    __syncwarp();
    if (lane == 0) st_release_cta_s32(f_n, n + 1);  // entry n is out
  }
  return n;
}

// The plan's last tile: the top K of the tiles' sorted lists, merged by one
// warp in K rounds (dense slots follow key order; the K results become keys
// at the end).  The lists are first copied to shared memory when they fit.
// With dense slots, warp 1 turns each merged entry into its key as soon as
// the merge puts it out (lane i takes entries i and 32 + i), so that those
// dictionary searches overlap the remaining rounds; its waits are bounded
// (kTopkSpin polls, then PQ_ERR_TIMEOUT).
constexpr i64 kTopkSpin = 1 << 24;
__device__ __forceinline__ void topk_final(const PlanDev& q, int K, int parts, bool dense,
                                           u32* scratch, DevStatus* st) {
  __shared__ i64 f_k[kMaxK], f_s[kMaxK];  // the merged entries (slots when dense)
  __shared__ int f_n, f_end;               // entries out; 1 once the merge is done
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The dense dictionary's counters, loaded while the lists are copied.
  u64 m_n = 0, m_bits = 0, m_umin = 0, m_tot = 0;
  if (dense && warp == 1)
    m_n = q.ctr->mcount, m_bits = q.ctr->m_bits, m_umin = q.ctr->m_umin, m_tot = q.ctr->m_distinct;
  if (threadIdx.x == 0) f_n = 0, f_end = 0;
  int* lc = reinterpret_cast<int*>(scratch);  // list lengths
  i64* sk = reinterpret_cast<i64*>(lc + kTKP);
  const int all = parts * K;
  const bool fit = (size_t)all * 16 + kTKP * 4 <= (size_t)kTKW * kTKR * 4;
  i64* ss = sk + all;
  // The list lengths and (when they fit) the lists: every load issued
  // before any is used, so that the copy costs about one memory latency.
  constexpr int kLcPer = kTKP / (kTKW * 32);
  int lcv[kLcPer];
#pragma unroll
  for (int u = 0; u < kLcPer; ++u) {
    const int i = (int)threadIdx.x + u * kTKW * 32;
    lcv[u] = i < parts ? __ldcg(q.tk_c + i) : 0;
  }
  if (fit) {  // 16 entries per thread in flight
    for (int e0 = threadIdx.x; e0 < all; e0 += 16 * blockDim.x) {
      i64 xk[16], xs[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + u * blockDim.x;
        xk[u] = e < all ? __ldcg(q.cand_k + e) : 0;
        xs[u] = e < all ? __ldcg(q.cand_s + e) : 0;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < all) sk[e] = xk[u], ss[e] = xs[u];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kLcPer; ++u) {
    const int i = (int)threadIdx.x + u * kTKW * 32;
    if (i < parts) lc[i] = lcv[u];
  }
  __syncthreads();
  if (dense && warp == 1) {
    const DenseView dv = dense_view(q.ht_tag, (i64)m_n, m_bits);
    for (int i = lane; i < K; i += 32) {
      i64 spins = 0;
      int out = ld_acquire_cta_s32(&f_n);
      while (out <= i && !ld_acquire_cta_s32(&f_end) && ++spins < kTopkSpin) {
        __nanosleep(32);
        out = ld_acquire_cta_s32(&f_n);
      }
      out = ld_acquire_cta_s32(&f_n);
      if (out <= i) {  // fewer entries, or the wait ran out (reported)
        if (!ld_acquire_cta_s32(&f_end)) q_latch(q.ctr, st, PQ_ERR_TIMEOUT, i);
        break;
      }
      q.out->keys[i] = dense_key(dv, m_umin, (u64)f_k[i], m_tot), q.out->sums[i] = f_s[i];
    }
    return;
  }
  if (warp != 0) return;
  const int n =
      fit ? topk_merge_rounds(K, parts, lc, [&](i64 e) { return sk[e]; },
                              [&](i64 e) { return ss[e]; }, f_k, f_s, &f_n)
          : topk_merge_rounds(K, parts, lc, [&](i64 e) { return __ldcg(q.cand_k + e); },
                              [&](i64 e) { return __ldcg(q.cand_s + e); }, f_k, f_s, &f_n);
  __syncwarp();
  if (lane == 0) st_release_cta_s32(&f_end, 1);
  if (!dense)
    for (int i = lane; i < n; i += 32) q.out->keys[i] = f_k[i], q.out->sums[i] = f_s[i];
  if (lane == 0) {
    q.out->n = n;
    q.out->ngroups = (i64)ld_volatile_u64(&q.ctr->gcount);
  }
}

__global__ void __launch_bounds__(kTKW * 32) k_plan_topk(Batch b) {
  chain_begin();
  __shared__ __align__(16) u32 s_ring[kTKW][kTKR];
  __shared__ i64 s_scr[kTKW][kTopScr];
  __shared__ i64 s_mk[kTKW * kMaxK], s_ms[kTKW * kMaxK];
  __shared__ int s_mc[kTKW];
  __shared__ LaneRankSmem<kTKW * 32> s_lr;
  __shared__ i64 s_t;
  __shared__ int s_cnt;
  __shared__ bool s_last;
  const i64* pre = b.dyn + 4 * (b.nq + 1);
  const i64 total = pre[b.nq];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TopList L;
  L.bind(s_scr[warp]);
  BlockClaim bc;
  while (true) {
    const i64 t = bc.next(b.work, kPhTopk, &s_t);
    if (t >= total) break;
    const int qi = find_q(pre, b.nq, t);
    const PlanDev& q = b.q[qi];
    const int K = q.k;
    const TopkSrc src = topk_src(q);
    const i64 tw = topk_tile_words_w(src.words);
    const i64 lt = t - pre[qi];
    const int parts = (int)(pre[qi + 1] - pre[qi]);
    i64* tk = q.cand_k + lt * K;
    i64* ts = q.cand_s + lt * K;
    // The tile's top K.  K <= 32: each lane keeps its best kLL records;
    // thr = the K-th best of the lanes' best; the entries not after thr (at
    // most kLL from each of K lanes) are ranked.  Exact unless a lane dropped
    // a record that is not after the K-th result; then (and for K > 32) the
    // tile is scanned again into per-warp lists merged in shared memory.
    bool done = false;
    u64 groups = 0;
    if (K <= 32) {
      LaneTop T;
      T.clear();
      groups = tk_scan(src, tw, lt, s_ring[warp], [&](const KS* r) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (r[u].v) T.insert(r[u].k, r[u].s);
      });
      const int nres = tk_lane_rank(T, K, s_lr, tk, ts);
      done = nres >= 0;
      if (done && threadIdx.x == 0) s_cnt = nres;
    }
    if (!done) {
      L.clear();
      const u64 g = tk_scan(src, tw, lt, s_ring[warp], [&](const KS* r) {
#pragma unroll
        for (int u = 0; u < 8; ++u) L.offer(K, r[u].v, r[u].k, r[u].s);
      });
      if (K > 32) groups = g;
      tk_block_merge_all(L, K, s_mk, s_ms, s_mc);
      if (warp == 0) {
        L.store(tk, ts);
        if (lane == 0) s_cnt = L.cnt;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) groups += __shfl_xor_sync(kFull, groups, o);
    if (lane == 0 && groups) atomicAdd(&q.ctr->gcount, groups);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      q.tk_c[lt] = s_cnt;
      __threadfence();
      s_last = (int)atomicAdd(&q.ctr->tk_ticket, 1u) == parts - 1;
      if (s_last) fence_acq_rel_gpu();
    }
    __syncthreads();
    if (!s_last) {
      if (gridDim.x >= total) break;
      continue;
    }
    fence_acq_rel_gpu();  // the other tiles' lists, published before their tickets
    topk_final(q, K, parts, src.dense, &s_ring[0][0], b.st);
    if (gridDim.x >= total) break;  // one tile per block: no ticket needed to stop
  }
  finish(b.work, kPhTopk);
}


#endif  // PQ_DEFINE_PLAN_KERNELS

}  // namespace pqk
