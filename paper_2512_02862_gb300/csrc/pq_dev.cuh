// pq_dev.cuh -- device helpers shared by the kernels of libpq.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pqk {

typedef long long i64;
typedef unsigned long long u64;
typedef unsigned int u32;

constexpr i64 kEmpty = (i64)0x8000000000000000ULL;  // INT64_MIN marks a free slot
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 64;

// Device status word: first error wins; `detail` carries a count or index.
struct DevStatus {
  int code;
  int pad;
  i64 detail;
};

__device__ __forceinline__ void latch(DevStatus* st, int code, i64 detail) {
  if (atomicCAS(&st->code, 0, code) == 0) atomicExch((u64*)&st->detail, (u64)detail);
}

// Predicate "v op c" lowered on the host to a closed range with a negation:
// pass = (lo <= v <= hi) xor neg.  '<' c -> [MIN, c-1], '==' c -> [c, c],
// '!=' c -> [c, c] negated, always-true -> [MIN, MAX].
struct Pred {
  i64 lo, hi;
  int neg, pad;
};
__device__ __forceinline__ bool pass(const Pred& p, i64 v) {
  return ((v >= p.lo) & (v <= p.hi)) ^ (p.neg != 0);
}

// Hash-table slot hash: the MurmurHash3 64-bit finaliser (Appleby), so that
// dense or strided keys spread over a power-of-two table.
__device__ __forceinline__ u64 slot_hash(i64 k) {
  u64 x = (u64)k;
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

// Radix bucket: Fibonacci hashing (Knuth), top log2P bits of k * 2^64/phi.
__device__ __forceinline__ u32 fib_bucket(i64 k, int log2P) {
  return log2P == 0 ? 0u : (u32)(((u64)k * 0x9E3779B97F4A7C15ULL) >> (64 - log2P));
}

// Slot of key k in a plan hash table of 2^(64 - shift) slots: the top bits of
// the Fibonacci product (one 64-bit multiply).  Multiplicative hashing spreads
// arithmetic key sequences (dense ids, strided keys) evenly, which keeps
// linear-probing runs short.
__device__ __forceinline__ u64 fib_slot(i64 k, int shift) {
  return ((u64)k * 0x9E3779B97F4A7C15ULL) >> shift;
}

// A predicate on an int32 column as one unsigned range test:
// pass = ((u32)(v - lo) <= span) xor neg.
struct Pred32 {
  int lo;
  unsigned span;
  unsigned neg;
};
__host__ __device__ __forceinline__ Pred32 to32(const Pred& p) {
  const i64 lo = p.lo < (i64)INT32_MIN ? (i64)INT32_MIN : p.lo;
  const i64 hi = p.hi > (i64)INT32_MAX ? (i64)INT32_MAX : p.hi;
  Pred32 r;
  if (lo > hi) {  // no int32 value is in range: all-range test, inverted
    r.lo = INT32_MIN;
    r.span = 0xFFFFFFFFu;
    r.neg = p.neg ? 0u : 1u;
  } else {
    r.lo = (int)lo;
    r.span = (unsigned)(hi - lo);
    r.neg = p.neg ? 1u : 0u;
  }
  return r;
}
__device__ __forceinline__ unsigned pass32(const Pred32& p, int v) {
  return (unsigned)((unsigned)(v - p.lo) <= p.span) ^ p.neg;
}

// L2 cache policies: hash tables are probed many times and should stay in L2
// (evict_last); scanned columns are read once (evict_first, no L1 allocation).
__device__ __forceinline__ u64 policy_keep() {
  u64 p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ u64 policy_stream() {
  u64 p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ i64 ld_keep(const i64* ptr, u64 pol) {
  i64 v;
  asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ unsigned short ld_keep_u16(const unsigned short* ptr, u64 pol) {
  unsigned short v;
  asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(ptr), "l"(pol));
  return v;
}

// Bucketized, tagged open addressing for the plan's tables.  A table of 2^e
// slots is 2^(e-3) buckets of 8 slots; a bucket's eight 16-bit tags fill one
// 16-byte word.  Key k goes to bucket = top bits of the Fibonacci product
// h = k * 2^64/phi and carries tag = the 16 bits below them (forced odd, so
// 0 marks an empty slot).  A lookup reads one 16-byte tag word, compares all
// eight tags at once (SIMD halfword compares), reads an 8-byte key only on a
// tag match, and moves to the next bucket only while buckets are full; an
// insert claims the first free tag of the first non-full bucket with a 16-bit
// CAS, so a bucket with a free slot ends every lookup.
struct BucketTag {
  u64 bucket;
  unsigned tag;
};
__device__ __forceinline__ BucketTag bucket_tag(i64 k, int shiftb) {
  const u64 h = (u64)k * 0x9E3779B97F4A7C15ULL;
  BucketTag r;
  r.bucket = h >> shiftb;
  r.tag = (unsigned)((h >> (shiftb - 16)) & 0xFFFFu) | 1u;
  return r;
}

// Byte masks of the slots of a bucket whose tag equals v (v replicated in both
// halves of v2): byte j of lo (slots 0..3) / hi (slots 4..7) is 0xFF on a match.
struct Mask8 {
  u32 lo, hi;
};
__device__ __forceinline__ Mask8 match8(uint4 w, unsigned v2) {
  Mask8 m;
  m.lo = __byte_perm(__vcmpeq2(w.x, v2), __vcmpeq2(w.y, v2), 0x7531);
  m.hi = __byte_perm(__vcmpeq2(w.z, v2), __vcmpeq2(w.w, v2), 0x7531);
  return m;
}
__device__ __forceinline__ bool any8(Mask8 m) { return (m.lo | m.hi) != 0; }
// Index of the first set slot (mask must be non-empty) and its removal.
__device__ __forceinline__ int first8(Mask8 m) {
  return m.lo ? (__ffs(m.lo) - 1) >> 3 : 4 + ((__ffs(m.hi) - 1) >> 3);
}
__device__ __forceinline__ void drop8(Mask8& m, int j) {
  if (j < 4) m.lo &= ~(0xFFu << (8 * j));
  else m.hi &= ~(0xFFu << (8 * (j - 4)));
}

__device__ __forceinline__ uint4 ld_keep_v4u(const void* ptr, u64 pol) {
  uint4 v;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ int4 ld_stream_v4(const void* ptr, u64 pol) {
  int4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ int2 ld_stream_v2i(const void* ptr, u64 pol) {
  int2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(ptr), "l"(pol));
  return v;
}
// Four 64-bit values in one 256-bit load (32-byte aligned).
__device__ __forceinline__ void ld_stream_v4l(const void* ptr, u64 pol, i64 v[4]) {
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s64 {%0, %1, %2, %3}, [%4], %5;"
      : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3])
      : "l"(ptr), "l"(pol));
}
__device__ __forceinline__ longlong2 ld_stream_v2(const void* ptr, u64 pol) {
  longlong2 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y)
               : "l"(ptr), "l"(pol));
  return v;
}

// Smallest power-of-two exponent with 2^e > count / lf (and e >= 6).  The
// host sizes every table region with this same function from an upper bound
// of the count, so the device's choice always fits the region.
__host__ __device__ __forceinline__ int cap_log2(i64 count, int lf1024) {
  i64 need = (count * 1024 + lf1024 - 1) / lf1024 + 1;
  int e = 6;
  while (((i64)1 << e) < need) ++e;
  return e;
}

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}

// Programmatic dependent launch: every plan kernel is launched so that it may
// start while the previous kernel of the chain finishes.  It first waits
// until that kernel has completed and its writes are visible, then lets the
// next kernel of the chain launch early in turn.  Launched without the
// attribute, the wait returns at once.
__device__ __forceinline__ void chain_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Block-wide exclusive sum of one value per thread (every thread calls; the
// caller synchronises before calling it again).
__device__ __forceinline__ u32 block_exclusive_sum(u32 v) {
  __shared__ u32 s_w[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u32 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const u32 c = lane < nw ? s_w[lane] : 0u;
    u32 y = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 z = __shfl_up_sync(kFull, y, o);
      if (lane >= o) y += z;
    }
    if (lane < nw) s_w[lane] = y - c;
  }
  __syncthreads();
  return s_w[warp] + x - v;
}

__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Reserve `cnt` consecutive output positions per lane from a global counter
// with one atomic per warp.  Every lane of the warp must call it.
__device__ __forceinline__ u64 warp_reserve(u64* counter, u32 cnt) {
  const int lane = threadIdx.x & 31;
  u32 incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  u32 total = __shfl_sync(kFull, incl, 31);
  u64 base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, (u64)total);
  base = __shfl_sync(kFull, base, 31);
  return base + (incl - cnt);
}

// Bounded spin: returns false once `limit` polls have been spent.
struct Spin {
  i64 left;
  __device__ explicit Spin(i64 limit) : left(limit) {}
  __device__ __forceinline__ bool again() {
    if (--left <= 0) return false;
    __nanosleep(64);
    return true;
  }
};

// ---- 1D bulk copies (TMA) into shared memory, completing on an mbarrier ----
__device__ __forceinline__ u32 smem_u32(const void* p) {
  return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Makes initialised mbarriers visible to the async proxy (the copy engine).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Acquire-release fence at GPU scope: after a ticket shows that other blocks
// published their results (each behind a fence), their writes are visible to
// this thread's later reads.  Lighter than __threadfence (sequentially
// consistent).
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
// Release store / acquire load of a shared-memory int at CTA scope: a warp
// that sees the stored value also sees the writes ordered before the store.
__device__ __forceinline__ void st_release_cta_s32(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
// Orders this thread's earlier shared-memory accesses before later async-
// proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arrive on `bar` and add `bytes` to the bytes its current phase waits for.
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Wait until the phase of `bar` with parity `par` completes; false after
// `limit` polls (each poll itself waits up to a hardware time limit).
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 par, i64 limit) {
  for (i64 it = 0;; ++it) {
    u32 done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(par)
        : "memory");
    if (done) return true;
    if (it >= limit) return false;
  }
}

__device__ __forceinline__ u64 ld_volatile_u64(const u64* p) {
  return *(const volatile u64*)p;
}
__device__ __forceinline__ void st_volatile_u64(u64* p, u64 v) { *(volatile u64*)p = v; }

// A counter that other blocks of this kernel updated with atomics (read by
// the block that finishes last, after its fence).
__device__ __forceinline__ i64 ld_count(const u64* p) { return (i64)ld_volatile_u64(p); }

// Single-pass tile prefix by decoupled look-back (Merrill & Garland, "Single-
// pass Parallel Prefix Scan with Decoupled Look-back", NVIDIA TR 2016).  Each
// status word packs a 2-bit flag (0 not ready, 1 aggregate, 2 inclusive
// prefix) and a 62-bit non-negative value.  Called by one full warp of the
// block that owns `tile`; returns the exclusive prefix of `tile` in every
// lane and publishes tile's inclusive prefix.  Tiles must be claimed in
// increasing order by running blocks (an atomic ticket), so every awaited
// predecessor belongs to a resident block and the wait ends; it is still
// bounded by `limit`, after which the status latches PQ_ERR_TIMEOUT (6) and
// the missing part counts as zero.
__device__ __forceinline__ i64 lookback_prefix(u64* state, i64 tile, i64 aggregate,
                                               i64 limit, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  constexpr u64 kA = 1ULL << 62, kP = 2ULL << 62, kMask = (1ULL << 62) - 1;
  if (tile == 0) {
    if (lane == 0) st_volatile_u64(&state[0], kP | (u64)aggregate);
    return 0;
  }
  if (lane == 0) st_volatile_u64(&state[tile], kA | (u64)aggregate);
  i64 prefix = 0;
  i64 idx = tile - 1 - lane;
  Spin spin(limit);
  bool timed_out = false;
  while (true) {
    u64 s = idx >= 0 ? ld_volatile_u64(&state[idx]) : kP;
    while (__any_sync(kFull, (s >> 62) == 0)) {
      if (!spin.again()) {
        timed_out = true;
        if ((s >> 62) == 0) s = kP;  // give up: count the missing tile as 0
        break;
      }
      if ((s >> 62) == 0) s = ld_volatile_u64(&state[idx]);
    }
    const u32 pmask = __ballot_sync(kFull, (s >> 62) == 2);
    i64 v = (i64)(s & kMask);
    if (pmask) {
      const int first = __ffs(pmask) - 1;  // nearest predecessor with a prefix
      if (lane > first) v = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    prefix += v;
    if (pmask) break;
    idx -= 32;
  }
  if (timed_out && lane == 0) latch(st, 6, tile);
  if (lane == 0) st_volatile_u64(&state[tile], kP | (u64)(prefix + aggregate));
  return prefix;
}


}  // namespace pqk
