/*
 * pq.h -- C ABI of the single-GPU relational hot path (libpq.so).
 *
 * The library runs a filter -> radix partition -> hash-join -> exact group-by
 * SUM -> top-k plan over integer columnar tables on one NVIDIA GB300
 * (sm_103a).  Every operator is a hand-written CUDA kernel; there is no CPU
 * fallback.  The operations are the data-parallel steps of the distributed
 * OLAP engine of arXiv 2512.02862 ("PystachIO"): columnar tensors split into
 * horizontal chunks (Sec. 2.1), filter pushdown in the scan (Sec. 4, 6.1),
 * partitioning by join key ahead of the exchange (Sec. 3.1), hash-table build
 * on the materialised left side and probe with right-side chunks (Sec. 3.1,
 * 3.2), aggregation (Sec. 3.2, 6.3), chunked ingest overlapped with compute
 * on several streams (Sec. 3.2, 4.2), deferred synchronisation (Sec. 3.3),
 * a multi-producer single-consumer chunk queue with a bounded size
 * (Sec. 5.4) and a pool allocator over one device buffer (Sec. 3.1).  Top-k
 * (ORDER BY ... LIMIT k) is not described in the paper.
 *
 * Conventions
 * -----------
 * - Every call returns a pq_status (0 = PQ_OK).  Nothing throws or aborts
 *   across the ABI.  pq_last_error(ctx) describes the last failure.
 * - Device-side operator calls are ASYNCHRONOUS on the CUDA stream passed as
 *   `void* stream` (a cudaStream_t; NULL = the legacy default stream).  Input
 *   arrays are BORROWED device pointers that must stay valid until the stream
 *   reaches the call.  Data-dependent counts are written to caller-owned
 *   DEVICE int64 words (`d_count`, ...), so no call waits for the GPU.
 * - Errors that only the device can see (output capacity exceeded, a
 *   reserved key, an int64 overflow, a bounded wait that ran out) are latched
 *   in a device status word and returned by the next pq_sync(ctx, stream).
 *   A latched PQ_ERR_CAPACITY leaves the needed count in the call's count
 *   word; the outputs hold the first `cap` results.
 * - Scratch memory and library-owned objects (tables, hash tables, plan
 *   workspaces) come from the arena passed to pq_create: one caller-allocated
 *   device buffer whose size is the device-memory budget.  Scratch is
 *   returned to the arena when the stream that used it passes an event, so
 *   concurrent calls on different streams never share scratch.  When the
 *   arena cannot satisfy a request the call returns PQ_ERR_BUDGET.
 * - Keys equal to INT64_MIN are reserved (the empty-slot marker of the hash
 *   tables); a build or group-by that meets one latches PQ_ERR_RESERVED_KEY.
 * - Column element types: int8, int32, int64 (pq_dtype).  Vectorised 128-bit
 *   loads are used when every column pointer is 16-byte aligned; other
 *   alignments take a scalar path with identical results.
 * - A ctx is safe to use from several host threads; its serving loop
 *   (pq_submit / pq_poll) runs on a library-owned thread.
 */
#ifndef PQ_H_
#define PQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PQ_ABI_VERSION 1
#define PQ_MAX_K 64          /* largest k accepted by pq_topk and plans      */
#define PQ_MAX_PAYLOAD 8     /* payload columns carried by pq_partition      */
#define PQ_MAX_LOG2P 12      /* largest fan-out exponent (4096 buckets)      */

typedef enum pq_status {
  PQ_OK = 0,
  PQ_ERR_INVALID_ARG = 1,  /* bad pointer, size, type or option             */
  PQ_ERR_BUDGET = 2,       /* the arena (device budget) is too small        */
  PQ_ERR_CAPACITY = 3,     /* an output buffer was too small                */
  PQ_ERR_CUDA = 4,         /* a CUDA runtime call failed                    */
  PQ_ERR_IO = 5,           /* a file read failed or came up short           */
  PQ_ERR_TIMEOUT = 6,      /* a bounded wait (device spin or host poll) ran out */
  PQ_ERR_OVERFLOW = 7,     /* an int64 aggregate overflowed                 */
  PQ_ERR_BUSY = 8,         /* the serving queue is full                     */
  PQ_ERR_RESERVED_KEY = 9  /* a key equal to INT64_MIN reached a hash table */
} pq_status;

typedef enum pq_dtype { PQ_INT8 = 1, PQ_INT32 = 2, PQ_INT64 = 3 } pq_dtype;

/* Predicate "value op constant" (the filter pushed into the scan, Sec. 4). */
typedef enum pq_cmp {
  PQ_LT = 0, PQ_LE = 1, PQ_GT = 2, PQ_GE = 3, PQ_EQ = 4, PQ_NE = 5,
  PQ_ALL = 6 /* always true */
} pq_cmp;

/* A borrowed column: `n` elements of type `type` at device address `data`. */
typedef struct pq_col {
  const void* data;
  int64_t n;
  int32_t type;      /* pq_dtype */
  int32_t reserved;  /* must be 0 */
} pq_col;

/* Context options.  Zero in any field selects its default. */
typedef struct pq_options {
  int32_t block_threads;   /* threads per block of the scan kernels (256)         */
  int32_t blocks_per_sm;   /* resident blocks per SM for persistent grids (2)     */
  float load_factor;       /* hash-table load factor, 0.05 .. 0.9 (0.5)           */
  int32_t log2P;           /* fan-out exponent of partitioned plans (6)           */
  int64_t chunk_bytes;     /* streaming chunk size in bytes (128 MiB)             */
  int32_t ingest_threads;  /* reader threads for file / pageable sources (4)      */
  int32_t copy_streams;    /* host-to-device copy streams (2)                     */
  int32_t ring_slots;      /* device chunk slots of the ingest ring (4)           */
  int32_t serve_slots;     /* plans in flight in the serving loop (4)            */
  int64_t spin_limit;      /* iteration limit of every device-side wait (1<<22)   */
  int32_t serve_queue;     /* pending requests before pq_submit says BUSY (4096)  */
  int32_t profile;         /* 1: record CUDA events around every plan kernel      */
  int32_t hit_buffer;      /* dynamic buffering of a streamed plan's F hits: the
                              device buffer holds the hits of this many chunks of
                              F rows (16); -1: probe every chunk (Sec. 5.3)       */
  int32_t reserved[5];
} pq_options;

typedef struct pq_ctx pq_ctx;
typedef struct pq_table pq_table;
typedef struct pq_ht pq_ht;

/* ---- context ------------------------------------------------------------ */

/* Fill `opt` with the defaults listed in pq_options. */
pq_status pq_default_options(pq_options* opt);

/* Create a context on the current CUDA device.  `arena` is a device buffer of
 * `arena_bytes` bytes that the caller owns and keeps alive until
 * pq_destroy; every library allocation on the device is carved from it (the
 * pool allocator of Sec. 3.1), so its size is the device-memory budget.
 * `opt` may be NULL (defaults).  On success *out receives the context. */
pq_status pq_create(const pq_options* opt, void* arena, size_t arena_bytes, pq_ctx** out);

/* Stop the serving loop, wait for the device, release everything the context
 * holds (the arena itself stays with the caller).  Requests still queued in
 * the serving loop complete with PQ_ERR_TIMEOUT without running; batches
 * already on the GPU get 30 s to finish.  If one does not, nothing is
 * released (its memory may still be in use), the context must not be used
 * again, and the call returns PQ_ERR_TIMEOUT instead of waiting without end. */
pq_status pq_destroy(pq_ctx* ctx);

/* Wait for `stream`, then return (and clear) the first device-latched error
 * since the previous pq_sync. */
pq_status pq_sync(pq_ctx* ctx, void* stream);

/* Message of the last failure on this context (valid until the next call). */
const char* pq_last_error(pq_ctx* ctx);

/* Static name of a status code. */
const char* pq_status_string(int status);

/* Counters kept by the context. */
typedef struct pq_stats {
  int64_t kernel_launches;   /* kernels launched by this context              */
  int64_t h2d_bytes;         /* bytes copied host -> device                   */
  int64_t d2h_bytes;         /* bytes copied device -> host                   */
  int64_t arena_bytes;       /* arena size                                    */
  int64_t arena_in_use;      /* bytes currently allocated                     */
  int64_t arena_high_water;  /* largest allocation total seen                 */
  int64_t chunks_ingested;   /* streaming chunks moved to the device          */
  int64_t plans_run;         /* plans completed (all paths)                   */
  int64_t graph_replays;     /* plan launches served by a captured CUDA graph */
  int64_t out_of_core_passes; /* passes of plans run out of core (pq_run_plan) */
  int64_t reserved[6];
} pq_stats;
pq_status pq_get_stats(pq_ctx* ctx, pq_stats* out);

/* Per-kernel timing (profile option): total milliseconds and launch count of
 * kernel `name` (e.g. "plan_fprobe") accumulated since the last reset.  The
 * caller synchronises the streams first.  Returns PQ_ERR_INVALID_ARG for an
 * unknown name. */
pq_status pq_profile_read(pq_ctx* ctx, const char* name, double* total_ms, int64_t* launches);
pq_status pq_profile_reset(pq_ctx* ctx);
/* Switch per-kernel timing on (1) or off (0) for the calls issued after it
 * (the profile option at creation sets the initial state).  While it is on,
 * plans run as separate launches with an event pair around each kernel;
 * while it is off, a repeated plan replays its CUDA graph.  The caller issues
 * no plan concurrently with the switch. */
pq_status pq_profile_enable(pq_ctx* ctx, int32_t on);

/* ---- tables --------------------------------------------------------------- */

typedef enum pq_src_kind {
  PQ_SRC_DEVICE = 0,  /* `ptr` is device memory (borrowed, never copied)       */
  PQ_SRC_HOST = 1,    /* `ptr` is host memory; pinned memory is copied
                         directly, pageable memory through pinned staging      */
  PQ_SRC_FILE = 2,    /* raw little-endian column file `path`, data starting at
                         byte `offset`, read with pread by the ingest threads  */
  PQ_SRC_PACKED = 3   /* `ptr` is a packed column (pq_pack_column) in page-
                         locked host memory; `type` is the column's type.  A
                         RESIDENT table decodes it into the arena once; a
                         STREAMING table copies each chunk's packed bytes and
                         decodes them on the device (Sec. 4.1: compressed
                         data decoded on the GPU); MAPPED refuses it.       */
} pq_src_kind;

typedef struct pq_source {
  int32_t kind;       /* pq_src_kind */
  int32_t type;       /* pq_dtype    */
  const void* ptr;
  const char* path;
  int64_t offset;
} pq_source;

typedef enum pq_load_mode {
  PQ_RESIDENT = 0,    /* copy into the arena now (device sources are borrowed) */
  PQ_STREAMING = 1,   /* keep on the host; plans stream it in chunks of
                         `chunk_bytes` through the ingest ring (Sec. 3.2, 4.2) */
  PQ_MAPPED = 2       /* keep in page-locked host memory (cudaHostAlloc'd or
                         cudaHostRegister'ed; device sources are borrowed) and
                         let the plan kernels read it in place over the host
                         link: a plan runs like one on resident tables and
                         moves only the bytes its kernels load (the
                         late-materialised columns only for the rows that
                         need them).  Pageable memory and files are refused
                         with PQ_ERR_INVALID_ARG. */
} pq_load_mode;

/* Describe (and for PQ_RESIDENT, copy in) a table of `ncols` columns of
 * `nrows` rows each.  Host memory and files must stay unchanged until the
 * table is freed.  *out receives a library-owned handle. */
pq_status pq_load_columns(pq_ctx* ctx, const pq_source* srcs, int ncols, int64_t nrows,
                          int mode, pq_table** out, void* stream);

/* Packed columns (frame of reference + bit packing): the rows are cut into
 * blocks of PQ_PACK_BLOCK rows; a block stores its smallest value and every
 * value's difference from it in the fewest bits that hold the block's largest
 * difference (0 to 64), one bit stream per block.  Layout of a packed column
 * (all little-endian):
 *   header (32 B): u32 magic "PQPK", u32 version 1, i32 type, u32 block rows,
 *                  i64 nrows, i64 nblocks;
 *   block table: nblocks + 1 entries of 16 B {i64 base, u32 first word,
 *                u8 width, 3 B zero}; the last entry holds the total words;
 *   payload: u32 words from the next 16-byte boundary; value i of a block is
 *   bits [i*width, (i+1)*width) of the block's stream (LSB first), followed
 *   by 4 zero words.
 * pq_pack_bound gives the largest packed size of `nrows` values of `type`;
 * pq_pack_column packs host memory into `out` (host memory, `cap` bytes) and
 * writes the size used to *out_bytes.  Host-only (no device work); returns
 * PQ_ERR_INVALID_ARG for a bad type or pointer and PQ_ERR_CAPACITY when `cap`
 * is too small. */
#define PQ_PACK_BLOCK 4096
int64_t pq_pack_bound(int64_t nrows, int32_t type);
pq_status pq_pack_column(const void* src, int32_t type, int64_t nrows, void* out, int64_t cap,
                         int64_t* out_bytes);

/* Number of rows of a table, and the device-accessible pointer of a resident
 * or mapped column (NULL for a streaming table). */
int64_t pq_table_rows(const pq_table* t);
const void* pq_table_column(const pq_table* t, int col);

/* Release a table or hash table once `stream` has passed all work queued so
 * far.  Cached hash tables built from the table are dropped too. */
pq_status pq_table_free(pq_ctx* ctx, pq_table* t, void* stream);
pq_status pq_ht_free(pq_ctx* ctx, pq_ht* ht, void* stream);

/* ---- operators ------------------------------------------------------------ */

/* Selection: write to `sel_out`, in ascending order, the row ids i with
 * `col[i] op c` (filter pushdown, Sec. 4), and their number to *d_count.
 * With `sel_in` (ascending row ids of a previous selection, `n_in` of them,
 * or *d_n_in of them if `d_n_in` is non-NULL) only those rows are tested, so
 * the result is the AND of both predicates.  `sel_out` holds n_in (or col.n)
 * ids.  Single pass: one read of the column, decoupled look-back for the
 * tile offsets (Merrill & Garland 2016) whose waits are bounded. */
pq_status pq_filter(pq_ctx* ctx, pq_col col, int op, int64_t c, const int64_t* sel_in,
                    int64_t n_in, const int64_t* d_n_in, int64_t* sel_out, int64_t* d_count,
                    void* stream);

/* Radix hash partition by join key (the step ahead of the exchange,
 * Sec. 3.1): bucket(k) = (uint64(k) * 0x9E3779B97F4A7C15 mod 2^64)
 * >> (64 - log2P) (Fibonacci hashing; bucket 0 when log2P = 0).  Rows are
 * written to out_key / out_payload[j] grouped by bucket, in input order
 * within a bucket (stable); d_offsets[b] .. d_offsets[b+1] (device, P + 1
 * int64) delimit bucket b.  0 <= log2P <= PQ_MAX_LOG2P, npay <=
 * PQ_MAX_PAYLOAD, payload columns have key.n rows; output arrays have the
 * element types of their inputs. */
pq_status pq_partition(pq_ctx* ctx, pq_col key, const pq_col* payload, int npay, int log2P,
                       void* out_key, void* const* out_payload, int64_t* d_offsets,
                       void* stream);

/* Hash-join build on the materialised left side (Sec. 3.1, 3.2): an
 * open-addressing table (linear probing, power-of-two capacity >= n /
 * load_factor) of (key, value) pairs in the arena.  `val` may have data NULL
 * (value = build row id); otherwise val.n == key.n.  Duplicate keys occupy
 * one slot each.  load_factor <= 0 takes the context default. */
pq_status pq_join_build(pq_ctx* ctx, pq_col key, pq_col val, float load_factor, pq_ht** out,
                        void* stream);

/* Hash-join probe (Sec. 3.1): for every probe row i and every build row with
 * an equal key, one output pair (i, build value).  Pairs come in no defined
 * order; *d_count receives the total.  At most `cap` pairs are written. */
pq_status pq_join_probe(pq_ctx* ctx, const pq_ht* ht, pq_col probe_key, int64_t* out_probe_row,
                        int64_t* out_build_val, int64_t cap, int64_t* d_count, void* stream);

/* Group-by SUM (Sec. 3.2): one (key, exact int64 sum) per distinct key, in no
 * defined order; *d_ngroups receives the number of groups.  `val` is int8,
 * int32 or int64 (summed in int64).  At most `cap` groups are written; the
 * hash table is sized for min(key.n, cap) groups.  Inputs of 2^20 rows or
 * more (outside stream capture) first measure the key range, which waits
 * for the stream once; when the range is at most 4 keys per row the groups
 * are summed in a slot array over the range instead of the hash table. */
pq_status pq_groupby_sum(pq_ctx* ctx, pq_col key, pq_col val, int64_t* out_keys,
                         int64_t* out_sums, int64_t cap, int64_t* d_ngroups, void* stream);

/* Top-k (ORDER BY sum DESC, key ASC LIMIT k; not in the paper): the first
 * min(k, n) pairs of (keys[i], sums[i]) in that order, count to *d_nout.
 * If `d_n` is non-NULL the pair count is read from it on the device (at most
 * n).  1 <= k <= PQ_MAX_K. */
pq_status pq_topk(pq_ctx* ctx, const int64_t* keys, const int64_t* sums, int64_t n,
                  const int64_t* d_n, int k, int64_t* out_keys, int64_t* out_sums,
                  int64_t* d_nout, void* stream);

/* Allocation-free selection (no counterpart in the paper): the same result
 * as pq_filter, for callers that cannot allocate device memory -- code that
 * runs while a CUDA graph is being captured, or inside a runtime that owns
 * every allocation -- and that may have no context.  Its scratch is a fixed
 * static device array inside libpq (about 1 MiB, held by every GPU that loads
 * the library until the process exits), so it needs neither an arena nor any
 * allocation; the caller passes the inputs and outputs as for pq_filter.
 * Limits: at most 536,870,912 rows tested per call (col.n, or n_in with a
 * selection vector); larger inputs return PQ_ERR_CAPACITY before any GPU
 * work.  The first call on a device looks up the array's device address
 * (once per device, with that device current), so make that first call
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller; each call clears what it uses first.  If
 * `d_error` (device int32) is non-NULL it receives 0, or PQ_ERR_TIMEOUT if a
 * bounded wait gave up.  Returns PQ_ERR_INVALID_ARG for bad arguments and
 * PQ_ERR_CUDA if the set-up or a launch fails. */
pq_status pq_filter_noalloc(pq_col col, int op, int64_t c, const int64_t* sel_in, int64_t n_in,
                            int64_t* sel_out, int64_t* d_count, int32_t* d_error, void* stream);

/* ---- the plan ------------------------------------------------------------- */

enum pq_plan_flags {
  PQ_PLAN_PARTITIONED = 1,  /* radix-partition the build side and the filtered
                               probe side into 2^log2P buckets and probe bucket
                               by bucket (out-of-core style)                   */
  PQ_PLAN_CACHE_DSET = 2,   /* keep the filtered dimension key set resident and
                               reuse it for later plans with the same D table,
                               row range and predicate                         */
  PQ_PLAN_NO_GRAPH = 4,     /* never replay a captured CUDA graph              */
  PQ_PLAN_AGG_FIRST = 8     /* the aggregate-first plan (below)                */
};

/* The three-table plan (the running example's shape, Sec. 5.1):
 *   D' = { D.key : D.seg op_d c_d },
 *   M' = { M rows : M.date op_m c_m and M.dref in D' },
 *   for each pair (F row, M' row) with F.date2 op_f c_f and F.mkey = M.key:
 *       sum[M.key] += F.price * (100 - F.disc)
 *   result = top-k of (M.key, sum) by sum desc, key asc, and the number of
 *   groups (M keys with at least one pair).
 * Column order and types: D = [key int32, seg int8]; M = [key int64,
 * dref int32, date int32]; F = [mkey int64, price int64, disc int8,
 * date2 int32].  Each table may be restricted to the rows
 * [row0, row0 + rows) (rows < 0: to the end).
 *
 * With PQ_PLAN_AGG_FIRST the plan aggregates first (a large materialised
 * group-by filtered on its aggregate, the shape of Sec. 6.3's Q18 remark):
 *   G = F rows with F.date2 op_f c_f grouped by F.mkey, sum = sum of
 *       F.price * (100 - F.disc) over the group (every group materialised);
 *   result = the groups with sum > `having` whose key is an M' key (a
 *   semi-join: a key held by several M' rows counts once), top-k by sum
 *   desc, key asc, and their number; `hits` = the F rows aggregated.
 * It needs resident tables whose F keys span at most 4 * (rows of the F
 * table) + 4096 values (PQ_ERR_INVALID_ARG otherwise).  Overflow is reported when the
 * magnitudes of all summed revenues reach 2^62, the bound below which no
 * group sum can leave int64. */
typedef struct pq_plan {
  const pq_table* D;
  const pq_table* M;
  const pq_table* F;
  int64_t d_row0, d_rows, m_row0, m_rows, f_row0, f_rows;
  int32_t d_op; int32_t m_op; int32_t f_op; int32_t k;
  int64_t d_c, m_c, f_c;
  int32_t flags;        /* pq_plan_flags */
  int32_t log2P;        /* <= 0: context default */
  float load_factor;    /* <= 0: context default */
  int32_t reserved;
  int64_t having;       /* PQ_PLAN_AGG_FIRST: keep groups whose sum > having */
} pq_plan;

/* Result of one plan; the device writes it with one copy. */
typedef struct pq_result {
  int64_t n;                  /* rows in keys/sums: min(k, ngroups)            */
  int64_t ngroups;            /* number of groups                              */
  int64_t keys[PQ_MAX_K];
  int64_t sums[PQ_MAX_K];
  int32_t status;             /* pq_status of this plan's device work          */
  int32_t reserved;
  int64_t hits;               /* F rows that joined (the probe's inputs)       */
} pq_result;

/* Run one plan on `stream`.  Resident tables run as one chain of kernels with
 * no host synchronisation (deferred synchronisation, Sec. 3.3); repeated
 * identical plans replay a captured CUDA graph.  Streaming tables are fed
 * through the ingest ring with copies on side streams overlapped with compute.
 * If `result` is pinned host memory the call returns at once and the result
 * is valid after pq_sync(ctx, stream); otherwise the call waits.
 *
 * Out of core: when a join-first plan over resident or mapped tables does
 * not fit the arena and its M keys are dense (a key-range bitmap), the build
 * side is radix-partitioned by key range (1024 buckets of the M key
 * column, counted once per table) and the plan runs in passes over groups of
 * consecutive buckets whose dictionary fits (Sec. 3.4, chunks bound the
 * memory; Sec. 3.1, build and probe per partition); F is scanned once per
 * pass.  The passes' groups are disjoint and their results are merged on
 * the host, so such a call returns when the plan is done;
 * pq_stats.out_of_core_passes counts the passes.  PQ_ERR_BUDGET when not
 * even one bucket fits. */
pq_status pq_run_plan(pq_ctx* ctx, const pq_plan* plan, pq_result* result, void* stream);

/* Run `n` plans in one batch: each kernel of the chain is launched once for
 * all plans, its persistent blocks stealing tiles from a flattened work list,
 * so plans of very different sizes share the GPU.  When the plans stream
 * their tables and all name the same D, M and F tables, each chunk of a
 * streamed table is read and copied once for the whole batch and every plan
 * scans its own rows of it (reader combining, Sec. 5.2); plans over
 * different streamed tables run one after another.  Results as for
 * pq_run_plan (pinned -> asynchronous). */
pq_status pq_run_batch(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                       void* stream);

/* ---- serving ---------------------------------------------------------------- */

/* Continuous batching: hand a plan to the context's serving loop, which
 * admits it as soon as a slot and arena memory are free, batches it with the
 * other admitted requests and runs the batch on one of `serve_slots` streams
 * while earlier batches are still on the GPU.  Plans over streamed tables are
 * batched like pq_run_batch batches them: one ingest pass per batch for the
 * tables they share.
 * *ticket identifies the request.  PQ_ERR_BUSY if `serve_queue` requests are
 * already pending. */
pq_status pq_submit(pq_ctx* ctx, const pq_plan* plan, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: forever, 0: do not wait) for request `ticket`;
 * on completion copy its result to *result and forget the ticket.  Returns
 * PQ_ERR_TIMEOUT if it is not done in time (poll again later). */
pq_status pq_poll(pq_ctx* ctx, uint64_t ticket, pq_result* result, int timeout_ms);

/* Submit-to-completion latency of a finished request in microseconds
 * (valid for the ticket of the last successful pq_poll). */
double pq_last_latency_us(pq_ctx* ctx);

/* ---- tuning ------------------------------------------------------------------ */

typedef struct pq_tuning {
  int32_t block_threads;  /* threads per block of the plan kernels (always
                             256: they are written for 8 warps)           */
  int32_t blocks_per_sm;  /* resident blocks per SM of the persistent grids */
  int32_t log2P;          /* fan-out exponent of the partitioned plan      */
  int32_t partitioned;    /* 1 if the partitioned plan was fastest         */
  float load_factor;      /* hash-table load factor                        */
  float best_ms;          /* median time of the chosen setting             */
  int32_t tried;          /* settings measured                             */
  int32_t reserved[5];
} pq_tuning;

/* Time `sample` (a join-first plan over resident tables; the tuning of
 * Sec. 3.1 applied to this engine's launch and partition parameters) by
 * coordinate descent: resident blocks per SM of the persistent kernels
 * (1, 2, 3, 4, 6, 8), then the hash-table load factor (0.25, 0.4, 0.5, 0.7),
 * then the partitioned plan with 2^4, 2^6, 2^8 and 2^10 buckets -- 14
 * settings, each the median of 5 timed runs.  The fastest goes to *out; its
 * blocks per SM and load factor become the context's defaults, and when
 * the partitioned plan won, its fan-out becomes the default log2P of plans
 * that set PQ_PLAN_PARTITIONED (the caller sets that flag: results are the
 * same either way).  The sample's result is not returned. */
pq_status pq_autotune(pq_ctx* ctx, const pq_plan* sample, pq_tuning* out);

#ifdef __cplusplus
}
#endif

#endif /* PQ_H_ */
