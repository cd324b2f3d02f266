// pq_internal.h -- host-side internals shared by the translation units of libpq.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pq.h"
#include "pq_dev.cuh"

namespace pqh {

using pqk::i64;

// ---------------------------------------------------------------------------
// Arena: first-fit pool allocator over the caller's device buffer (the pool
// allocator of Sec. 3.1).  Frees are stream-ordered: a block released on a
// stream becomes reusable once an event recorded on that stream completes.
class Arena {
 public:
  void init(char* base, size_t bytes);
  void shutdown();
  // nullptr when the request cannot be met even after waiting for pending frees.
  void* alloc(size_t bytes, size_t align = 256);
  void release(void* p, cudaStream_t s);  // reusable once `s` reaches this point
  void release_now(void* p);
  size_t in_use() const { return in_use_; }
  size_t high_water() const { return high_; }
  size_t capacity() const { return cap_; }
  size_t largest_free();

 private:
  void reclaim(bool wait_one);
  void insert_free(size_t off, size_t size);
  char* base_ = nullptr;
  size_t cap_ = 0, in_use_ = 0, high_ = 0;
  std::map<size_t, size_t> free_;             // offset -> size, coalesced
  std::unordered_map<size_t, size_t> live_;   // offset -> size
  struct Pending { size_t off, size; cudaEvent_t ev; };
  std::deque<Pending> pending_;
  std::vector<cudaEvent_t> events_;
  std::mutex mu_;
};

// Pinned host staging ring for small uploads (descriptors) and result
// read-back: no pageable copies ever reach a stream (Sec. 4.2, "mis-sync").
class PinnedRing {
 public:
  bool init(size_t slot_bytes, int slots);
  void shutdown();
  // Copies `bytes` (<= slot size) from `src` into a free pinned slot and
  // enqueues the upload to `dst` on `s`.
  cudaError_t upload(void* dst, const void* src, size_t bytes, cudaStream_t s);
  size_t slot_bytes() const { return slot_; }

 private:
  char* host_ = nullptr;
  size_t slot_ = 0;
  int n_ = 0, next_ = 0;
  std::vector<cudaEvent_t> ev_;
  std::mutex mu_;
};

// Packed columns (pq_pack.cu; layout in pq.h).
struct PackBlock {
  int64_t base;    // smallest value of the block
  uint32_t word;   // first payload word of the block's bit stream
  uint8_t width;   // bits per value (0..64)
  uint8_t pad[3];
};
static_assert(sizeof(PackBlock) == 16, "packed block entry");
struct PackedView {
  const PackBlock* blocks = nullptr;  // nblocks + 1 entries
  const uint32_t* words = nullptr;
  int64_t nblocks = 0, total_words = 0;
};
struct PackedRange {
  int64_t b0, b1;  // blocks holding the rows
  int64_t w0, w1;  // payload words to copy (with the decoder's padding)
};
// Check a packed column's header against its type and row count.
bool packed_info(const void* p, int type, int64_t nrows, PackedView* v);
PackedRange packed_range(const PackedView& v, int64_t row0, int64_t n);
// Decode rows [row0, row0 + n) (column rows) from device copies of the block
// table (from block row0 / PQ_PACK_BLOCK) and payload (from word w0).
cudaError_t unpack_launch(const PackBlock* dblk, const uint32_t* dwords, int64_t w0, int64_t row0,
                          int64_t n, int type, void* out, int num_sms, cudaStream_t s);

// Descent positions kept per key column (see KeyRange::desc).
constexpr int kMaxDescents = 8;

// Range of an integer key column (order-preserving ukey = key xor 2^63) and
// its key order: the rows that start a new non-decreasing run of keys
// (ascending), ndesc of them, or ndesc = -1 when there are more than
// kMaxDescents.  The fields are written once, before `ready` is set with
// release order; a reader that sees `ready` (acquire) reads them without a
// lock, since they never change afterwards.
struct KeyRange {
  std::atomic<bool> ready{false};
  uint64_t umin = 0, umax = 0;
  int ndesc = -1;
  int64_t desc[kMaxDescents] = {};
  KeyRange() = default;
  KeyRange(const KeyRange& o) { *this = o; }
  KeyRange& operator=(const KeyRange& o) {
    umin = o.umin, umax = o.umax, ndesc = o.ndesc;
    for (int j = 0; j < kMaxDescents; ++j) desc[j] = o.desc[j];
    ready.store(o.ready.load(std::memory_order_acquire), std::memory_order_release);
    return *this;
  }
  bool known() const { return ready.load(std::memory_order_acquire); }
};

// Rows per key-range bucket of an integer key column: kHistBuckets buckets
// of 2^shift keys from the column's smallest key (ukey order), measured on
// the first out-of-core plan over the table and kept.  Published like
// KeyRange: counts and shift are written before `ready` (release).
constexpr int kHistBuckets = 1024;
struct KeyHist {
  std::atomic<bool> ready{false};
  int shift = 0;
  std::vector<uint32_t> counts;
  KeyHist() = default;
  KeyHist(const KeyHist& o) { *this = o; }
  KeyHist& operator=(const KeyHist& o) {
    shift = o.shift;
    counts = o.counts;
    ready.store(o.ready.load(std::memory_order_acquire), std::memory_order_release);
    return *this;
  }
  bool known() const { return ready.load(std::memory_order_acquire); }
};

// Which keys of an integer key column's range occur in the column: a
// bitmap over [umin, umax] with a rank directory (the dense dictionary's
// layout: dense_layout(0, bits)), so that a key's rank among the column's
// distinct keys is three loads.  Measured on the first aggregate-first plan
// over the table, kept in an arena block the table owns.  Published like
// KeyRange.
struct KeyPresence {
  std::atomic<bool> ready{false};
  void* block = nullptr;
  uint64_t bits = 0, distinct = 0;
  // Bit j: the column's key-ordered segment j (rows from the j-th segment
  // start of its KeyRange) is gapless: its distinct keys are consecutive
  // among the column's distinct keys.
  uint32_t gapless = 0;
  KeyPresence() = default;
  KeyPresence(const KeyPresence& o) { *this = o; }
  KeyPresence& operator=(const KeyPresence& o) {
    block = o.block, bits = o.bits, distinct = o.distinct, gapless = o.gapless;
    ready.store(o.ready.load(std::memory_order_acquire), std::memory_order_release);
    return *this;
  }
  bool known() const { return ready.load(std::memory_order_acquire); }
};

struct Column {
  int type = 0;           // pq_dtype
  bool packed = false;    // source is a packed column (PQ_SRC_PACKED)
  PackedView pk;
  const void* dev = nullptr;   // device pointer (resident) or nullptr
  pq_source src{};        // original source (streaming)
  bool pinned = false;    // host source is page-locked
  void* owned = nullptr;  // arena block owned by the table
  std::string path;
  // Range and key order of an integer key column of a resident table,
  // measured on first use by a plan and kept (see KeyRange).
  mutable KeyRange range;
  mutable KeyHist hist;
  mutable KeyPresence pres;
};

}  // namespace pqh

struct pq_table {
  uint64_t id = 0;
  int64_t nrows = 0;
  int mode = 0;
  std::vector<pqh::Column> cols;
};

struct pq_ht {
  pqk::i64* keys = nullptr;
  pqk::i64* vals = nullptr;  // keys + 1: slots are {key, value} pairs
  pqk::i64* meta = nullptr;   // [0] duplicate-key flag, [1] inserted count
  int log2cap = 0;
  int64_t n = 0;
  void* block = nullptr;
};

namespace pqh {

struct Profile {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
  size_t used = 0;
  double total_ms = 0;
  int64_t launches = 0;
};

struct PlanCache;   // pq_plan.cu
struct Server;      // pq_serve.cu

struct DsetEntry {
  uint64_t table_id;
  int64_t row0, rows;
  pqk::Pred pred;
  int lf1024;
  void* block;        // arena block: header word (log2 of the slot count), slots
  pqk::i64* keys;
  int log2max;
  bool bm;            // built as a static key bitmap
  cudaEvent_t ready;  // recorded after the set is built
  uint64_t last_use;
  // Batches between their look-up of the entry and the record of their
  // completion event: an entry with pins is never released.
  int pins;
  bool dead;          // its table was freed while pinned: erased at unpin
  // Completion events of the batches that read the entry; a release of the
  // block is ordered after all of them.
  std::vector<cudaEvent_t> users;
};

}  // namespace pqh

struct pq_ctx {
  pq_options opt{};
  int device = 0;
  int num_sms = 0;
  pqh::Arena arena;
  pqh::PinnedRing ring;
  pqk::DevStatus* d_status = nullptr;
  pqk::DevStatus* h_status = nullptr;   // pinned mirror
  int64_t* h_small = nullptr;            // pinned read-back buffers (SmallPinned)
  std::vector<int64_t*> small_free;      // free buffers of h_small
  std::mutex small_mu;                   // guards small_free only
  std::mutex range_mu;                   // serialises writers of KeyRange
  std::mutex mu;                         // serialises API calls that touch state
  std::string last_error;
  std::atomic<int64_t> launches{0}, h2d{0}, d2h{0}, chunks{0}, plans{0}, replays{0}, passes{0};
  std::atomic<uint64_t> next_table_id{1};
  std::map<std::string, pqh::Profile> prof;
  std::vector<cudaStream_t> copy_streams;
  cudaStream_t util_stream = nullptr;    // key-range measurements
  std::list<pqh::DsetEntry> dsets;   // stable addresses
  uint64_t dset_tick = 0;
  pqh::PlanCache* plan_cache = nullptr;   // owned; freed by plan_cache_destroy
  pqh::Server* server = nullptr;          // owned; freed by server_stop
  double last_latency_us = 0;
  // tuning (kernel launch shapes chosen by pq_autotune or the options)
  int tune_threads = 256;
  int tune_bps = 2;
  // resident blocks per SM of each plan kernel (filled by plan_kernels_init)
  int plan_occ[28] = {0};
};

namespace pqh {

pq_status fail(pq_ctx* ctx, pq_status st, const char* fmt, ...);
// Per-device set-up of the plan kernels (shared-memory limits, occupancy).
pq_status plan_kernels_init(pq_ctx* ctx);
pq_status cuda_fail(pq_ctx* ctx, cudaError_t e, const char* what);

#define PQ_CUDA(ctx, call)                                      \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return pqh::cuda_fail(ctx, e_, #call); \
  } while (0)

// After a kernel launch: count it and turn a launch error into PQ_ERR_CUDA.
#define PQ_LAUNCHED(ctx)                                                  \
  do {                                                                    \
    (ctx)->launches.fetch_add(1, std::memory_order_relaxed);              \
    cudaError_t e_ = cudaGetLastError();                                  \
    if (e_ != cudaSuccess) return pqh::cuda_fail(ctx, e_, "kernel launch"); \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

pqk::Pred make_pred(int op, int64_t c, bool* ok);
size_t dtype_size(int type);
bool valid_dtype(int type);
int grid_persistent(pq_ctx* ctx, int threads);

// Profiling: start/stop events around a kernel when ctx->opt.profile is set.
void prof_begin(pq_ctx* ctx, const char* name, cudaStream_t s, cudaEvent_t* stop_out);
void prof_end(cudaEvent_t stop, cudaStream_t s);
void prof_collect(pq_ctx* ctx);

// A pinned read-back buffer of kSmallBytes from the context's pool, returned
// at scope exit.  The pool's lock is held only to take and return a buffer,
// never across a wait on the GPU.
constexpr size_t kSmallBytes = 512;
constexpr int kSmallBufs = 64;
struct SmallPinned {
  pq_ctx* ctx;
  int64_t* p = nullptr;
  bool own = false;  // allocated because the pool was empty
  explicit SmallPinned(pq_ctx* c);
  ~SmallPinned();
};

// Scoped arena scratch released on a stream at scope exit.
struct Scratch {
  pq_ctx* ctx;
  cudaStream_t s;
  std::vector<void*> blocks;
  Scratch(pq_ctx* c, cudaStream_t st) : ctx(c), s(st) {}
  void* get(size_t bytes) {
    void* p = ctx->arena.alloc(bytes ? bytes : 256);
    if (p) blocks.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void* p : blocks) ctx->arena.release(p, s);
  }
};

// Launchers implemented in pq_ops.cu, used by the plan paths.
pq_status fill_i64(pq_ctx* ctx, pqk::i64* p, int64_t n, pqk::i64 v, cudaStream_t s);
// The top-k operator's kernel on caller-provided scratch: `ticket` zeroed
// before the launch, `lists` topk_scratch_bytes(ctx, n, k) bytes; it always
// writes *d_nout (n >= 1).  `chained`: programmatic dependent launch.
size_t topk_scratch_bytes(pq_ctx* ctx, int64_t n, int k);
cudaError_t topk_launch(pq_ctx* ctx, const int64_t* keys, const int64_t* sums, int64_t n,
                        const int64_t* d_n, int k, int64_t* out_keys, int64_t* out_sums,
                        int64_t* d_nout, unsigned* ticket, void* lists, bool chained,
                        cudaStream_t s, const uint64_t* rec_ctr = nullptr,
                        pq_result* rec = nullptr);

// Plan internals (pq_plan.cu) used by pq_serve.cu and pq_tune.cu.
// The M key window of one pass of an out-of-core plan: M' restricted to the
// keys with ukey in [lo, lo + bits), at most `cap` members.
struct MWindow {
  uint64_t lo, bits;
  int64_t cap;
};
pq_status run_batch_internal(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                             cudaStream_t s, bool allow_graph, const MWindow* win = nullptr);
// Upper bound of the arena bytes a batch of these plans needs (0 if invalid).
size_t batch_workspace_bytes(pq_ctx* ctx, const pq_plan* plans, int n);
pq_status run_plan_streaming(pq_ctx* ctx, const pq_plan* plan, pq_result* result,
                             cudaStream_t s);
// A batch with streamed tables: one ingest pass over the tables shared by all
// plans (pq_stream.cu).
pq_status run_batch_streaming(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                              cudaStream_t s);
// Copy n results from the device (pinned destination: asynchronous).
pq_status read_back(pq_ctx* ctx, pq_result* results, const pq_result* dev, int n,
                    cudaStream_t s);
bool is_pinned(const void* p);
void plan_cache_destroy(pq_ctx* ctx);
// Drop cached graphs and D-sets that reference table `id`; their memory is
// released in the order of stream `s`.  Takes ctx->mu itself.
void forget_table(pq_ctx* ctx, uint64_t id, cudaStream_t s);
// Stop the serving loop; PQ_ERR_TIMEOUT if a batch did not complete in time.
pq_status server_stop(pq_ctx* ctx);

}  // namespace pqh
