// pq_stream.cu -- streaming plan driver: host-resident (pinned, pageable or
// file) tables are fed to the plan kernels chunk by chunk.
//
// Pipeline (chunked execution on several streams, Sec. 3.2; overlapped scan,
// Sec. 4.2; queue-based scheduling with a bounded queue, Sec. 5.4):
//   * the chunks of D, M and F form one sequence ("reader combining",
//     Sec. 5.2: one ingest pool serves every scan of the plan);
//   * pinned host columns are copied straight from their rows; pageable
//     memory and files are first filled into pinned staging buffers by
//     reader threads (multiple producers), in chunk order, and consumed by
//     the plan thread (single consumer);
//   * copies run on the context's copy streams into a ring of device slots,
//     each copy waits (on the GPU) for the kernel that last used its slot, and
//     each scan kernel waits for its copy -- the host never blocks on the GPU
//     except once after the D and M scans to size the tables exactly;
//   * the staging buffers and device slots bound the memory in flight
//     (adaptive regulation, Sec. 5.4).
#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>

#include "pq_plan_host.h"

using namespace pqk;

namespace pqh {

namespace {

size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct Chunk {
  int table;   // 0 D, 1 M, 2 F
  i64 row0;    // first row inside the plan's row range
  i64 rows;
};

struct TableIn {
  const pq_table* t = nullptr;
  i64 row0 = 0;    // plan row offset inside the table
  int ncols = 0;
  size_t esize[4] = {0, 0, 0, 0};
  size_t row_bytes = 0;
  bool packed = false;  // some column is packed (chunks start on pack blocks)
};

// Column j of chunk c laid out in a slot: columns one after another, each
// starting on a 256-byte boundary.
size_t col_offset(const TableIn& T, i64 rows, int j) {
  size_t o = 0;
  for (int i = 0; i < j; ++i) o += al(T.esize[i] * rows);
  return o;
}

// Multi-producer single-consumer staging queue.  Producers claim chunks in
// order after taking a free staging buffer, so the chunk the consumer waits
// for always owns a buffer and the queue cannot deadlock.
class Stager {
 public:
  Stager(pq_ctx* ctx, const TableIn* tabs, const std::vector<Chunk>& chunks, size_t buf_bytes,
         int nbuf, int nthreads)
      : ctx_(ctx), tabs_(tabs), chunks_(chunks), buf_bytes_(buf_bytes) {
    bufs_.resize(nbuf, nullptr);
    evs_.resize(nbuf, nullptr);
    for (int i = 0; i < nbuf; ++i) {
      if (cudaHostAlloc((void**)&bufs_[i], buf_bytes, 0) != cudaSuccess ||
          cudaEventCreateWithFlags(&evs_[i], cudaEventDisableTiming) != cudaSuccess) {
        ok_ = false;
        return;
      }
      free_.push_back(i);
    }
    ready_.assign(chunks.size(), -1);
    for (int i = 0; i < nthreads; ++i) th_.emplace_back([this] { run(); });
  }

  ~Stager() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
    for (size_t i = 0; i < bufs_.size(); ++i) {
      if (evs_[i]) cudaEventSynchronize(evs_[i]), cudaEventDestroy(evs_[i]);
      if (bufs_[i]) cudaFreeHost(bufs_[i]);
    }
  }

  bool ok() const { return ok_; }

  // Wait until chunk c is staged; returns its buffer index or -1 (I/O error).
  int wait(size_t c) {
    std::unique_lock<std::mutex> g(mu_);
    cv_.wait(g, [&] { return ready_[c] != -1 || err_; });
    return err_ ? -1 : ready_[c];
  }

  char* buf(int i) const { return bufs_[i]; }

  // The consumer enqueued the copies out of buffer i; it is free again once
  // event `after` (recorded after those copies) completes.
  void release(int i, cudaStream_t s) {
    cudaEventRecord(evs_[i], s);
    {
      std::lock_guard<std::mutex> g(mu_);
      free_.push_back(i);
    }
    cv_.notify_all();
  }

  std::string error() const { return msg_; }

 private:
  void run() {
    while (true) {
      int b;
      size_t c;
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&] { return stop_ || err_ || (!free_.empty() && next_ < chunks_.size()); });
        if (stop_ || err_ || next_ >= chunks_.size()) return;
        b = free_.front();
        free_.pop_front();
        c = next_++;
      }
      cudaEventSynchronize(evs_[b]);  // previous copies out of this buffer are done
      std::string m;
      bool good = fill(chunks_[c], bufs_[b], &m);
      {
        std::lock_guard<std::mutex> g(mu_);
        if (good) ready_[c] = b;
        else err_ = true, msg_ = m;
      }
      cv_.notify_all();
    }
  }

  bool fill(const Chunk& ch, char* dst, std::string* msg) {
    const TableIn& T = tabs_[ch.table];
    for (int j = 0; j < T.ncols; ++j) {
      const Column& col = T.t->cols[j];
      if (col.packed) continue;  // copied straight from its page-locked buffer
      const size_t es = T.esize[j];
      const size_t bytes = es * ch.rows;
      const size_t src_off = es * (T.row0 + ch.row0);
      char* d = dst + col_offset(T, ch.rows, j);
      if (col.src.kind == PQ_SRC_FILE) {
        int fd = open(col.path.c_str(), O_RDONLY);
        if (fd < 0) {
          *msg = "open " + col.path;
          return false;
        }
        size_t got = 0;
        while (got < bytes) {
          ssize_t r = pread(fd, d + got, bytes - got, (off_t)(col.src.offset + src_off + got));
          if (r <= 0) break;
          got += (size_t)r;
        }
        close(fd);
        if (got != bytes) {
          *msg = "short read from " + col.path;
          return false;
        }
      } else {
        memcpy(d, (const char*)col.src.ptr + src_off, bytes);
      }
    }
    return true;
  }

  pq_ctx* ctx_;
  const TableIn* tabs_;
  const std::vector<Chunk>& chunks_;
  size_t buf_bytes_;
  std::vector<char*> bufs_;
  std::vector<cudaEvent_t> evs_;
  std::deque<int> free_;
  std::vector<int> ready_;
  size_t next_ = 0;
  bool stop_ = false, err_ = false, ok_ = true;
  std::string msg_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::vector<std::thread> th_;
};

}  // namespace

pq_status run_plan_streaming(pq_ctx* ctx, const pq_plan* plan, pq_result* result,
                             cudaStream_t s) {
  ResolvedPlan r;
  pq_status st = resolve_plan(ctx, *plan, r, false);
  if (st != PQ_OK) return st;
  const pq_table* T3[3] = {plan->D, plan->M, plan->F};
  const i64 row0[3] = {r.d_row0, r.m_row0, r.f_row0};
  const i64 nrows[3] = {r.n_d, r.n_m, r.n_f};
  TableIn tabs[3];
  const size_t chunk_bytes = (size_t)ctx->opt.chunk_bytes;
  std::vector<Chunk> chunks;
  bool need_stage = false;
  for (int t = 0; t < 3; ++t) {
    TableIn& T = tabs[t];
    T.t = T3[t];
    T.row0 = row0[t];
    T.ncols = t == 0 ? 2 : t == 1 ? 3 : 4;
    for (int j = 0; j < T.ncols; ++j) {
      T.esize[j] = dtype_size(T.t->cols[j].type);
      T.row_bytes += T.esize[j];
    }
    if (r.resident[t]) continue;
    for (int j = 0; j < T.ncols; ++j) {
      const Column& c = T.t->cols[j];
      if (c.dev) return fail(ctx, PQ_ERR_INVALID_ARG, "streaming table mixes device columns");
      if (c.packed) T.packed = true;
      else if (!(c.src.kind == PQ_SRC_HOST && c.pinned)) need_stage = true;
    }
    i64 rows_per = (i64)((chunk_bytes - 4 * 256) / T.row_bytes) / 64 * 64;
    rows_per = std::max<i64>(rows_per, 64);
    if (T.packed) rows_per = std::max<i64>(rows_per / PQ_PACK_BLOCK, 1) * PQ_PACK_BLOCK;
    for (i64 a = 0; a < nrows[t]; a += rows_per)
      chunks.push_back({t, a, std::min(rows_per, nrows[t] - a)});
  }

  // Workspace part 1: header, D list, M list (sized by row counts); the D-set,
  // M table and group list are sized after the scans.
  const BatchLayout L = batch_layout(1);
  const int nslots = std::max(2, ctx->opt.ring_slots);
  Scratch scr(ctx, s);
  // F hit list: the rows of one F chunk (or of the resident F table).
  i64 f_hits = r.resident[2] ? r.n_f : 0;
  for (const Chunk& ch : chunks)
    if (ch.table == 2) f_hits = std::max(f_hits, ch.rows);
  char* ws = (char*)scr.get(L.end + al(r.n_d * 8) + al(r.n_m * 8) + al(f_hits * 4 + 4));
  // Partitioned plan: bucket counters and the partitioned hits of one chunk.
  const int plog = r.dev.part_log2;
  char* pws = plog ? (char*)scr.get(al(((1 << plog) + 1) * 8) + al(f_hits * 8 + 8) +
                                    al(f_hits * 4 + 4) + al(f_hits * 8 + 8))
                   : nullptr;
  if (plog && !pws) return fail(ctx, PQ_ERR_BUDGET, "streaming plan: partitioned hits");
  // A slot holds a chunk's plain columns and, for packed columns, their
  // packed bytes behind them (never more than the plain bytes plus the block
  // tables and padding).
  bool any_packed = false;
  for (int t = 0; t < 3; ++t) any_packed = any_packed || (!r.resident[t] && tabs[t].packed);
  const size_t slot_bytes = any_packed ? 2 * chunk_bytes + (64 << 10) : chunk_bytes + 1024;
  char* ring = chunks.empty() ? nullptr : (char*)scr.get(slot_bytes * nslots);
  if (!ws || (!chunks.empty() && !ring))
    return fail(ctx, PQ_ERR_BUDGET, "streaming plan: workspace and %d chunk slots of %zu bytes",
                nslots, chunk_bytes);
  PlanDev& d = r.dev;
  d.build_dset = 1;
  d.dlist = (i64*)(ws + L.end);
  d.mlist = (i64*)(ws + L.end + al(r.n_d * 8));
  d.hlist = (u32*)(ws + L.end + al(r.n_d * 8) + al(r.n_m * 8));
  set_kernel_variants(false, false);
  // Dynamic buffering (Sec. 5.3): a streamed F table's hits are gathered
  // into a buffer that holds `hit_buffer` chunks of rows (so it cannot
  // overflow), and the probe runs after every `hit_buffer` chunks and after
  // the last one instead of after every chunk.
  if (!r.resident[2] && !plog && ctx->opt.hit_buffer > 0 && f_hits > 0) {
    const u64 cap = (u64)f_hits * (u64)ctx->opt.hit_buffer;
    char* hb = (char*)scr.get(al(cap * 8) * 2 + al(cap));
    if (hb) {  // else the probe runs chunk by chunk
      d.hb_key = (i64*)hb;
      d.hb_price = (i64*)(hb + al(cap * 8));
      d.hb_disc = (signed char*)(hb + 2 * al(cap * 8));
      d.hb_cap = cap;
      set_kernel_variants(true, false);
    }
  }
  if (plog) {
    char* q = pws;
    d.part = (u64*)q;
    q += al(((1 << plog) + 1) * 8);
    d.pval0 = (i64*)q;
    q += al(f_hits * 8 + 8);
    d.pslot = (u32*)q;
    q += al(f_hits * 4 + 4);
    d.pval = (i64*)q;
  }
  QCtr* ctr = (QCtr*)(ws + L.ctr);
  d.ctr = ctr;
  d.out = (pq_result*)(ws + L.out);
  // Streamed columns live in ring slots: the kernels get them through the
  // chunk override, so only resident tables' pointers matter in `d`.
  bool vec = true;
  for (int t = 0; t < 3; ++t)
    if (r.resident[t]) {
      const void* ptrs[4] = {t == 0 ? (const void*)d.d_key : t == 1 ? (const void*)d.m_key
                                                                     : (const void*)d.f_mkey,
                             t == 0 ? (const void*)d.d_seg : t == 1 ? (const void*)d.m_dref
                                                                    : (const void*)d.f_price,
                             t == 1 ? (const void*)d.m_date : (const void*)d.f_disc,
                             (const void*)d.f_date};
      for (int j = 0; j < tabs[t].ncols; ++j) vec = vec && (((uintptr_t)ptrs[j]) & 15) == 0;
    }

  std::vector<char> host(L.upload_bytes());
  auto upload_desc = [&](i64 tiles_d, i64 tiles_m, i64 tiles_f) -> cudaError_t {
    memcpy(host.data(), &d, sizeof d);
    i64* tD = (i64*)(host.data() + (L.tD - L.desc));
    i64* tM = (i64*)(host.data() + (L.tM - L.desc));
    i64* tF = (i64*)(host.data() + (L.tF - L.desc));
    tD[0] = tM[0] = tF[0] = 0;
    tD[1] = tiles_d;
    tM[1] = tiles_m;
    tF[1] = tiles_f;
    return ctx->ring.upload(ws + L.desc, host.data(), host.size(), s);
  };
  // D-set region placeholder until the D scan is done: a 64-slot block.
  char* dset_blk = (char*)scr.get(dset_block_bytes(6));
  if (!dset_blk) return fail(ctx, PQ_ERR_BUDGET, "streaming plan: D-set");
  dset_block_assign(dset_blk, 6, d);
  PQ_CUDA(ctx, upload_desc(r.resident[0] ? (r.n_d + d.d_tile - 1) / d.d_tile : 0,
                           r.resident[1] ? (r.n_m + d.m_tile - 1) / d.m_tile : 0,
                           r.resident[2] ? (r.n_f + d.f_tile - 1) / d.f_tile : 0));
  PQ_CUDA(ctx, cudaMemsetAsync(ws + L.work, 0, L.zero_bytes(), s));
  Batch b = make_batch(ctx, ws, 1, L);

  std::unique_ptr<Stager> stager;
  if (need_stage) {
    stager.reset(new Stager(ctx, tabs, chunks, chunk_bytes + 1024,
                            std::max(2, ctx->opt.ring_slots), std::max(1, ctx->opt.ingest_threads)));
    if (!stager->ok()) return fail(ctx, PQ_ERR_CUDA, "streaming plan: pinned staging");
  }
  std::vector<cudaEvent_t> slot_free(nslots), copy_done(nslots);
  for (int i = 0; i < nslots; ++i) {
    cudaEventCreateWithFlags(&slot_free[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&copy_done[i], cudaEventDisableTiming);
  }
  struct EvGuard {
    std::vector<cudaEvent_t>& a;
    std::vector<cudaEvent_t>& b;
    ~EvGuard() {
      for (auto e : a) cudaEventSynchronize(e), cudaEventDestroy(e);
      for (auto e : b) cudaEventSynchronize(e), cudaEventDestroy(e);
    }
  } guard{slot_free, copy_done};

  const int ncs = (int)ctx->copy_streams.size();
  size_t issued = 0;  // chunks whose copies are enqueued
  // Enqueue the copies of chunk c into slot c % nslots.
  auto issue = [&](size_t c) -> pq_status {
    const Chunk& ch = chunks[c];
    const TableIn& T = tabs[ch.table];
    const int slot = (int)(c % nslots);
    cudaStream_t cs = ctx->copy_streams[c % ncs];
    char* dst = ring + slot * slot_bytes;
    PQ_CUDA(ctx, cudaStreamWaitEvent(cs, slot_free[slot], 0));
    int sb = -1;
    if (stager) {
      sb = stager->wait(c);
      if (sb < 0) return fail(ctx, PQ_ERR_IO, "streaming plan: %s", stager->error().c_str());
    }
    size_t total = 0;
    size_t pk_off = col_offset(T, ch.rows, T.ncols);  // packed bytes after the plain columns
    for (int j = 0; j < T.ncols; ++j) {
      const Column& col = T.t->cols[j];
      const size_t off = col_offset(T, ch.rows, j);
      if (col.packed) {
        // The chunk's block table entries and payload words, then the decode
        // into the plain column's place on the same copy stream.
        const i64 row = T.row0 + ch.row0;
        const PackedRange pr = packed_range(col.pk, row, ch.rows);
        const size_t tb = (size_t)(pr.b1 - pr.b0) * sizeof(PackBlock);
        const size_t wb = (size_t)(pr.w1 - pr.w0) * 4;
        char* dtab = dst + pk_off;
        char* dwords = dst + pk_off + al(tb);
        PQ_CUDA(ctx, cudaMemcpyAsync(dtab, col.pk.blocks + pr.b0, tb, cudaMemcpyHostToDevice, cs));
        PQ_CUDA(ctx, cudaMemcpyAsync(dwords, col.pk.words + pr.w0, wb, cudaMemcpyHostToDevice, cs));
        PQ_CUDA(ctx, unpack_launch((const PackBlock*)dtab, (const uint32_t*)dwords, pr.w0, row,
                                   ch.rows, col.type, dst + off, ctx->num_sms, cs));
        ctx->launches++;
        pk_off += al(tb) + al(wb);
        total += tb + wb;
        continue;
      }
      const size_t bytes = T.esize[j] * ch.rows;
      const void* src = stager ? (const void*)(stager->buf(sb) + off)
                               : (const void*)((const char*)col.src.ptr +
                                               T.esize[j] * (T.row0 + ch.row0));
      PQ_CUDA(ctx, cudaMemcpyAsync(dst + off, src, bytes, cudaMemcpyHostToDevice, cs));
      total += bytes;
    }
    PQ_CUDA(ctx, cudaEventRecord(copy_done[slot], cs));
    if (stager) stager->release(sb, cs);
    ctx->h2d += (int64_t)total;
    ctx->chunks++;
    return PQ_OK;
  };
  auto prefetch = [&](size_t upto) -> pq_status {
    while (issued < chunks.size() && issued < upto) {
      pq_status e = issue(issued);
      if (e != PQ_OK) return e;
      ++issued;
    }
    return PQ_OK;
  };
  // The F table's phase is the scan and the probe of its hits (for a
  // partitioned plan: the scan, the partition, scatter and aggregation
  // passes, then the probe kernel's epilogue), chunk by chunk; with buffered
  // hits the probe only after every hit_buffer chunks and the last.
  bool probe_now = true;
  i64 f_seen = 0;
  auto launch_table = [&](int t, const Batch& bt, bool v) -> pq_status {
    if (t < 2) return launch_phase(ctx, t == 0 ? kPhaseD : kPhaseM, bt, v, s);
    if (plog) PQ_CUDA(ctx, cudaMemsetAsync(d.part, 0, ((1 << plog) + 1) * 8, s));
    pq_status e = launch_phase(ctx, kPhaseFscan, bt, v, s);
    for (int ph : {kPhaseFpart, kPhaseFscatter, kPhaseFagg})
      if (e == PQ_OK && plog) e = launch_phase(ctx, ph, bt, v, s);
    if (e == PQ_OK && probe_now) e = launch_phase(ctx, kPhaseF, bt, v, s);
    return e;
  };
  size_t c = 0;
  for (int t = 0; t < 3; ++t) {
    if (r.resident[t]) {
      st = launch_table(t, b, vec && d.vec);
      if (st != PQ_OK) return st;
    } else if (nrows[t] == 0) {
      // An empty streamed table: one launch with no tiles still lets the
      // kernel's last block size the following phases.
      Batch bc = b;
      bc.ov.table = t + 1;
      bc.ov.n = 0;
      bc.ov.tiles = 0;
      st = launch_table(t, bc, true);
      if (st != PQ_OK) return st;
    } else {
      for (; c < chunks.size() && chunks[c].table == t; ++c) {
        st = prefetch(c + nslots);
        if (st != PQ_OK) return st;
        const Chunk& ch = chunks[c];
        const TableIn& T = tabs[t];
        const int slot = (int)(c % nslots);
        char* src = ring + slot * slot_bytes;
        PQ_CUDA(ctx, cudaStreamWaitEvent(s, copy_done[slot], 0));
        Batch bc = b;
        bc.ov.table = t + 1;
        bc.ov.n = ch.rows;
        const bool last = c + 1 == chunks.size() || chunks[c + 1].table != t;
        if (t == 2) ++f_seen;
        probe_now = t != 2 || !d.hb_cap || last || f_seen % ctx->opt.hit_buffer == 0;
        const int tile = t == 0   ? scan_tile(ch.rows, 512, kTD, resident_warps(ctx, 0))
                         : t == 1 ? scan_tile(ch.rows, 128, kTM, resident_warps(ctx, 3))
                                  : scan_tile(ch.rows, 128, kTF, resident_warps(ctx, 8));
        bc.ov.tile = tile;
        bc.ov.tiles = (ch.rows + tile - 1) / tile;
        for (int j = 0; j < T.ncols; ++j) bc.ov.p[j] = src + col_offset(T, ch.rows, j);
        st = launch_table(t, bc, true);
        if (st != PQ_OK) return st;
        PQ_CUDA(ctx, cudaEventRecord(slot_free[slot], s));
      }
    }
    if (t == 2) break;
    // Size the next table exactly from the device count (one host wait per
    // phase; the copies already enqueued keep streaming meanwhile).
    st = prefetch(c + nslots);
    if (st != PQ_OK) return st;
    i64 count = 0;
    {
      SmallPinned h(ctx);
      if (!h.p) return fail(ctx, PQ_ERR_CUDA, "streaming plan: pinned read-back buffer");
      cudaError_t e = cudaMemcpyAsync(h.p, t == 0 ? (void*)&ctr->dcount : (void*)&ctr->mcount, 8,
                                      cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "streaming plan: count read-back");
      count = h.p[0];
    }
    const int e = cap_log2(count, d.lf1024);
    if (t == 0) {
      char* blk = (char*)scr.get(dset_block_bytes(e));
      if (!blk) return fail(ctx, PQ_ERR_BUDGET, "streaming plan: D-set of 2^%d slots", e);
      dset_block_assign(blk, e, d);
      PQ_CUDA(ctx, upload_desc(0, r.resident[1] ? (r.n_m + d.m_tile - 1) / d.m_tile : 0,
                               r.resident[2] ? (r.n_f + d.f_tile - 1) / d.f_tile : 0));
      // The dscan kernel sized the fill/build phases; it wrote the header
      // (log2, bitmap base and bits) into the placeholder, copied here to the
      // real block.
      PQ_CUDA(ctx, cudaMemcpyAsync(d.dset_log2, dset_blk, 24, cudaMemcpyDeviceToDevice, s));
      for (int ph : {kPhaseDfill, kPhaseDbuild}) {
        st = launch_phase(ctx, ph, b, true, s);
        if (st != PQ_OK) return st;
      }
    } else {
      const i64 parts = topk_parts(e), cap = topk_cand_cap(e, d.k);
      char* blk = (char*)scr.get(mtable_bytes(e) + al(parts * 4) +
                                 al(cap * 8) * 2);
      if (!blk) return fail(ctx, PQ_ERR_BUDGET, "streaming plan: M table of 2^%d slots", e);
      char* p = mtable_assign(blk, e, d);
      d.tk_c = (int*)p;
      p += al(parts * 4);
      d.cand_k = (i64*)p;
      p += al(cap * 8);
      d.cand_s = (i64*)p;
      PQ_CUDA(ctx, upload_desc(0, 0, r.resident[2] ? (r.n_f + d.f_tile - 1) / d.f_tile : 0));
      for (int ph : {kPhaseMfill, kPhaseMbuild, kPhaseMrank, kPhaseMdup}) {
        st = launch_phase(ctx, ph, b, true, s);
        if (st != PQ_OK) return st;
      }
    }
  }
  st = launch_phase(ctx, kPhaseTopk, b, true, s);
  if (st != PQ_OK) return st;
  ctx->plans++;
  const size_t bytes = sizeof(pq_result);
  ctx->d2h += (int64_t)bytes;
  if (is_pinned(result)) {
    PQ_CUDA(ctx, cudaMemcpyAsync(result, d.out, bytes, cudaMemcpyDeviceToHost, s));
    return PQ_OK;
  }
  pq_result* tmp = nullptr;
  PQ_CUDA(ctx, cudaHostAlloc((void**)&tmp, bytes, 0));
  cudaError_t e = cudaMemcpyAsync(tmp, d.out, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) memcpy(result, tmp, bytes);
  cudaFreeHost(tmp);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "result read-back");
  return PQ_OK;
}

}  // namespace pqh

namespace pqh {

// A batch of plans over the same streamed tables (reader combining, Sec.
// 5.2): each chunk of a streamed table is read and copied once, and every
// plan scans the rows of the chunk that fall in its own row range -- its
// descriptors point into the chunk's slot for that launch.  Counts are read
// back once per table for all plans (the D-sets and M tables are sized
// exactly, as for one plan); resident tables of the batch are scanned in
// place.  Plans whose streamed tables differ run one after another.
pq_status run_batch_streaming(pq_ctx* ctx, const pq_plan* plans, int n, pq_result* results,
                              cudaStream_t s) {
  set_kernel_variants(false, false);
  std::vector<ResolvedPlan> R(n);
  for (int i = 0; i < n; ++i) {
    pq_status st = resolve_plan(ctx, plans[i], R[i], false);
    if (st != PQ_OK) return st;
  }
  const pq_table* T3[3] = {plans[0].D, plans[0].M, plans[0].F};
  bool shared = true;
  for (int i = 0; i < n; ++i) {
    const pq_table* Ti[3] = {plans[i].D, plans[i].M, plans[i].F};
    for (int t = 0; t < 3; ++t) shared = shared && Ti[t] == T3[t];
  }
  if (!shared || n == 1) {
    for (int i = 0; i < n; ++i) {
      pq_status st = run_plan_streaming(ctx, &plans[i], &results[i], s);
      if (st != PQ_OK) return st;
    }
    return PQ_OK;
  }
  bool streamed[3];
  for (int t = 0; t < 3; ++t) streamed[t] = !R[0].resident[t];
  auto prow0 = [&](int i, int t) { return t == 0 ? R[i].d_row0 : t == 1 ? R[i].m_row0 : R[i].f_row0; };
  auto prows = [&](int i, int t) { return t == 0 ? R[i].n_d : t == 1 ? R[i].n_m : R[i].n_f; };

  // Chunks over the union of the plans' row ranges of each streamed table.
  TableIn tabs[3];
  i64 urows[3] = {0, 0, 0};
  const size_t chunk_bytes = (size_t)ctx->opt.chunk_bytes;
  std::vector<Chunk> chunks;
  bool need_stage = false;
  for (int t = 0; t < 3; ++t) {
    TableIn& T = tabs[t];
    T.t = T3[t];
    T.ncols = t == 0 ? 2 : t == 1 ? 3 : 4;
    for (int j = 0; j < T.ncols; ++j) {
      T.esize[j] = dtype_size(T.t->cols[j].type);
      T.row_bytes += T.esize[j];
    }
    if (!streamed[t]) continue;
    i64 lo = prow0(0, t), hi = lo;
    for (int i = 0; i < n; ++i) {
      if (prows(i, t) == 0) continue;
      if (hi == lo) lo = prow0(i, t), hi = lo + prows(i, t);
      lo = std::min(lo, prow0(i, t));
      hi = std::max(hi, prow0(i, t) + prows(i, t));
    }
    T.row0 = lo;
    urows[t] = hi - lo;
    for (int j = 0; j < T.ncols; ++j) {
      const Column& c = T.t->cols[j];
      if (c.dev) return fail(ctx, PQ_ERR_INVALID_ARG, "streaming table mixes device columns");
      if (c.packed) T.packed = true;
      else if (!(c.src.kind == PQ_SRC_HOST && c.pinned)) need_stage = true;
    }
    i64 rows_per = (i64)((chunk_bytes - 4 * 256) / T.row_bytes) / 64 * 64;
    rows_per = std::max<i64>(rows_per, 64);
    if (T.packed) rows_per = std::max<i64>(rows_per / PQ_PACK_BLOCK, 1) * PQ_PACK_BLOCK;
    for (i64 a = 0; a < urows[t]; a += rows_per) {
      const i64 A = lo + a, B = A + std::min(rows_per, urows[t] - a);
      bool used = false;  // a chunk between the plans' row ranges is not read
      for (int i = 0; i < n && !used; ++i)
        used = prows(i, t) > 0 && prow0(i, t) < B && prow0(i, t) + prows(i, t) > A;
      if (used) chunks.push_back({t, a, B - A});
    }
  }

  // Workspace: the batch header, per plan the D and M key lists, a hit list
  // for its rows of one F chunk (or of a resident F) and a placeholder D-set;
  // the D-sets and M tables are sized after the scans.
  const BatchLayout L = batch_layout(n);
  const int nslots = std::max(2, ctx->opt.ring_slots);
  Scratch scr(ctx, s);
  i64 f_chunk = 0;
  for (const Chunk& ch : chunks)
    if (ch.table == 2) f_chunk = std::max(f_chunk, ch.rows);
  char* ws = (char*)scr.get(L.end);
  bool any_packed = false;
  for (int t = 0; t < 3; ++t) any_packed = any_packed || (streamed[t] && tabs[t].packed);
  const size_t slot_bytes = any_packed ? 2 * chunk_bytes + (64 << 10) : chunk_bytes + 1024;
  char* ring = chunks.empty() ? nullptr : (char*)scr.get(slot_bytes * nslots);
  if (!ws || (!chunks.empty() && !ring))
    return fail(ctx, PQ_ERR_BUDGET, "streaming batch: workspace and %d chunk slots", nslots);
  QCtr* ctr = (QCtr*)(ws + L.ctr);
  pq_result* out = (pq_result*)(ws + L.out);
  std::vector<PlanDev> base(n);
  std::vector<char*> dset_ph(n);
  std::vector<std::pair<void*, size_t>> part_clears;  // bucket counters, per F launch
  for (int i = 0; i < n; ++i) {
    PlanDev& d = R[i].dev;
    d.build_dset = 1;
    const i64 hl = streamed[2] ? std::min(R[i].n_f, f_chunk) : R[i].n_f;
    const int plog = d.part_log2;
    const size_t pbytes =
        plog ? al(((1 << plog) + 1) * 8) + al(hl * 8 + 8) + al(hl * 4 + 4) + al(hl * 8 + 8) : 0;
    char* p = (char*)scr.get(al(R[i].n_d * 8) + al(R[i].n_m * 8) + al(hl * 4 + 4) +
                             dset_block_bytes(6) + pbytes);
    if (!p) return fail(ctx, PQ_ERR_BUDGET, "streaming batch: lists of plan %d", i);
    d.dlist = (i64*)p;
    d.mlist = (i64*)(p + al(R[i].n_d * 8));
    d.hlist = (u32*)(p + al(R[i].n_d * 8) + al(R[i].n_m * 8));
    dset_ph[i] = p + al(R[i].n_d * 8) + al(R[i].n_m * 8) + al(hl * 4 + 4);
    dset_block_assign(dset_ph[i], 6, d);
    if (plog) {
      char* q = dset_ph[i] + dset_block_bytes(6);
      d.part = (u64*)q;
      q += al(((1 << plog) + 1) * 8);
      d.pval0 = (i64*)q;
      q += al(hl * 8 + 8);
      d.pslot = (u32*)q;
      q += al(hl * 4 + 4);
      d.pval = (i64*)q;
      part_clears.push_back({d.part, (size_t)((1 << plog) + 1) * 8});
    }
    d.ctr = ctr + i;
    d.out = out + i;
    base[i] = d;
  }

  // Descriptors for one launch: table t's rows of chunk `ch` (each plan's
  // window of it), or the resident tables in place (ch == nullptr).
  std::vector<char> host(L.upload_bytes());
  bool vec = true;
  auto upload = [&](int t, const Chunk* ch, const char* slot) -> pq_status {
    PlanDev* descs = (PlanDev*)host.data();
    i64* tX[3] = {(i64*)(host.data() + (L.tD - L.desc)), (i64*)(host.data() + (L.tM - L.desc)),
                  (i64*)(host.data() + (L.tF - L.desc))};
    for (int k = 0; k < 3; ++k) tX[k][0] = 0;
    vec = true;
    for (int i = 0; i < n; ++i) {
      PlanDev d = base[i];
      i64 tiles = 0;
      if (t >= 0) {
        const TableIn& T = tabs[t];
        i64 w0 = prow0(i, t), wn = prows(i, t);
        const void* cols[4] = {nullptr, nullptr, nullptr, nullptr};
        if (ch) {  // the plan's rows inside this chunk
          const i64 A = T.row0 + ch->row0, B = A + ch->rows;
          const i64 a = std::max(A, w0), b = std::min(B, w0 + wn);
          w0 = a;
          wn = std::max<i64>(0, b - a);
          for (int j = 0; j < T.ncols; ++j) {
            cols[j] = slot + col_offset(T, ch->rows, j) + (size_t)(a - A) * T.esize[j];
            vec = vec && (((uintptr_t)cols[j]) & 15) == 0;
          }
        } else {
          vec = vec && d.vec;
        }
        if (t == 0) {
          if (ch) d.d_key = (const int*)cols[0], d.d_seg = (const signed char*)cols[1];
          d.n_d = wn;
          d.d_tile = scan_tile(wn, 512, kTD, resident_warps(ctx, 0));
          tiles = (wn + d.d_tile - 1) / d.d_tile;
        } else if (t == 1) {
          if (ch) d.m_key = (const i64*)cols[0], d.m_dref = (const int*)cols[1],
                  d.m_date = (const int*)cols[2];
          d.n_m = wn;
          d.m_tile = scan_tile(wn, 128, kTM, resident_warps(ctx, 3));
          tiles = (wn + d.m_tile - 1) / d.m_tile;
        } else {
          if (ch) d.f_mkey = (const i64*)cols[0], d.f_price = (const i64*)cols[1],
                  d.f_disc = (const signed char*)cols[2], d.f_date = (const int*)cols[3];
          d.n_f = wn;
          d.f_tile = scan_tile(wn, 128, kTF, resident_warps(ctx, 8));
          tiles = (wn + d.f_tile - 1) / d.f_tile;
        }
      }
      descs[i] = d;
      for (int k = 0; k < 3; ++k) tX[k][i + 1] = tX[k][i] + (k == t ? tiles : 0);
    }
    PQ_CUDA(ctx, ctx->ring.upload(ws + L.desc, host.data(), host.size(), s));
    return PQ_OK;
  };

  std::unique_ptr<Stager> stager;
  if (need_stage) {
    stager.reset(new Stager(ctx, tabs, chunks, chunk_bytes + 1024,
                            std::max(2, ctx->opt.ring_slots), std::max(1, ctx->opt.ingest_threads)));
    if (!stager->ok()) return fail(ctx, PQ_ERR_CUDA, "streaming batch: pinned staging");
  }
  std::vector<cudaEvent_t> slot_free(nslots), copy_done(nslots);
  for (int i = 0; i < nslots; ++i) {
    cudaEventCreateWithFlags(&slot_free[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&copy_done[i], cudaEventDisableTiming);
  }
  struct EvGuard {
    std::vector<cudaEvent_t>& a;
    std::vector<cudaEvent_t>& b;
    ~EvGuard() {
      for (auto e : a) cudaEventSynchronize(e), cudaEventDestroy(e);
      for (auto e : b) cudaEventSynchronize(e), cudaEventDestroy(e);
    }
  } guard{slot_free, copy_done};
  const int ncs = (int)ctx->copy_streams.size();
  size_t issued = 0;
  auto issue = [&](size_t c) -> pq_status {
    const Chunk& ch = chunks[c];
    const TableIn& T = tabs[ch.table];
    const int slot = (int)(c % nslots);
    cudaStream_t cs = ctx->copy_streams[c % ncs];
    char* dst = ring + slot * slot_bytes;
    PQ_CUDA(ctx, cudaStreamWaitEvent(cs, slot_free[slot], 0));
    int sb = -1;
    if (stager) {
      sb = stager->wait(c);
      if (sb < 0) return fail(ctx, PQ_ERR_IO, "streaming batch: %s", stager->error().c_str());
    }
    size_t total = 0;
    size_t pk_off = col_offset(T, ch.rows, T.ncols);
    for (int j = 0; j < T.ncols; ++j) {
      const Column& col = T.t->cols[j];
      const size_t off = col_offset(T, ch.rows, j);
      const i64 row = T.row0 + ch.row0;
      if (col.packed) {
        const PackedRange pr = packed_range(col.pk, row, ch.rows);
        const size_t tb = (size_t)(pr.b1 - pr.b0) * sizeof(PackBlock);
        const size_t wb = (size_t)(pr.w1 - pr.w0) * 4;
        char* dtab = dst + pk_off;
        char* dwords = dst + pk_off + al(tb);
        PQ_CUDA(ctx, cudaMemcpyAsync(dtab, col.pk.blocks + pr.b0, tb, cudaMemcpyHostToDevice, cs));
        PQ_CUDA(ctx, cudaMemcpyAsync(dwords, col.pk.words + pr.w0, wb, cudaMemcpyHostToDevice, cs));
        PQ_CUDA(ctx, unpack_launch((const PackBlock*)dtab, (const uint32_t*)dwords, pr.w0, row,
                                   ch.rows, col.type, dst + off, ctx->num_sms, cs));
        ctx->launches++;
        pk_off += al(tb) + al(wb);
        total += tb + wb;
        continue;
      }
      const size_t bytes = T.esize[j] * ch.rows;
      const void* src = stager ? (const void*)(stager->buf(sb) + off)
                               : (const void*)((const char*)col.src.ptr + T.esize[j] * row);
      PQ_CUDA(ctx, cudaMemcpyAsync(dst + off, src, bytes, cudaMemcpyHostToDevice, cs));
      total += bytes;
    }
    PQ_CUDA(ctx, cudaEventRecord(copy_done[slot], cs));
    if (stager) stager->release(sb, cs);
    ctx->h2d += (int64_t)total;
    ctx->chunks++;
    return PQ_OK;
  };
  auto prefetch = [&](size_t upto) -> pq_status {
    while (issued < chunks.size() && issued < upto) {
      pq_status e = issue(issued);
      if (e != PQ_OK) return e;
      ++issued;
    }
    return PQ_OK;
  };

  pq_status st = upload(-1, nullptr, nullptr);
  if (st != PQ_OK) return st;
  PQ_CUDA(ctx, cudaMemsetAsync(ws + L.work, 0, L.zero_bytes(), s));
  const Batch b = make_batch(ctx, ws, n, L);
  auto launch_table = [&](int t, bool v) -> pq_status {
    if (t < 2) return launch_phase(ctx, t == 0 ? kPhaseD : kPhaseM, b, v, s);
    const bool part = !part_clears.empty();
    for (auto& c : part_clears) PQ_CUDA(ctx, cudaMemsetAsync(c.first, 0, c.second, s));
    pq_status e = launch_phase(ctx, kPhaseFscan, b, v, s);
    for (int ph : {kPhaseFpart, kPhaseFscatter, kPhaseFagg})
      if (e == PQ_OK && part) e = launch_phase(ctx, ph, b, v, s);
    if (e == PQ_OK) e = launch_phase(ctx, kPhaseF, b, v, s);
    return e;
  };
  std::vector<QCtr> hctr(n);
  auto read_counters = [&]() -> pq_status {
    PQ_CUDA(ctx, cudaMemcpyAsync(hctr.data(), ctr, sizeof(QCtr) * n, cudaMemcpyDeviceToHost, s));
    PQ_CUDA(ctx, cudaStreamSynchronize(s));
    return PQ_OK;
  };
  size_t c = 0;
  for (int t = 0; t < 3; ++t) {
    if (!streamed[t] || urows[t] == 0) {
      st = upload(t, nullptr, nullptr);
      if (st == PQ_OK) st = launch_table(t, vec);
      if (st != PQ_OK) return st;
    } else {
      for (; c < chunks.size() && chunks[c].table == t; ++c) {
        st = prefetch(c + nslots);
        if (st != PQ_OK) return st;
        const int slot = (int)(c % nslots);
        PQ_CUDA(ctx, cudaStreamWaitEvent(s, copy_done[slot], 0));
        st = upload(t, &chunks[c], ring + slot * slot_bytes);
        if (st == PQ_OK) st = launch_table(t, vec);
        if (st != PQ_OK) return st;
        PQ_CUDA(ctx, cudaEventRecord(slot_free[slot], s));
      }
    }
    if (t == 2) break;
    // Size every plan's next structure from its count (one host wait).
    st = prefetch(c + nslots);
    if (st == PQ_OK) st = read_counters();
    if (st != PQ_OK) return st;
    for (int i = 0; i < n; ++i) {
      PlanDev& d = base[i];
      const i64 count = (i64)(t == 0 ? hctr[i].dcount : hctr[i].mcount);
      const int e = cap_log2(count, d.lf1024);
      if (t == 0) {
        char* blk = (char*)scr.get(dset_block_bytes(e));
        if (!blk) return fail(ctx, PQ_ERR_BUDGET, "streaming batch: D-set of 2^%d slots", e);
        dset_block_assign(blk, e, d);
        // The D scan's last block wrote the header into the placeholder.
        PQ_CUDA(ctx, cudaMemcpyAsync(d.dset_log2, dset_ph[i], 24, cudaMemcpyDeviceToDevice, s));
      } else {
        const i64 parts = topk_parts(e), cap = topk_cand_cap(e, d.k);
        char* blk = (char*)scr.get(mtable_bytes(e) + al(parts * 4) +
                                   al(cap * 8) * 2);
        if (!blk) return fail(ctx, PQ_ERR_BUDGET, "streaming batch: M table of 2^%d slots", e);
        char* p = mtable_assign(blk, e, d);
        d.tk_c = (int*)p;
        p += al(parts * 4);
        d.cand_k = (i64*)p;
        p += al(cap * 8);
        d.cand_s = (i64*)p;
      }
    }
    st = upload(-1, nullptr, nullptr);
    if (st != PQ_OK) return st;
    const int next[2][4] = {{kPhaseDfill, kPhaseDbuild, -1, -1},
                            {kPhaseMfill, kPhaseMbuild, kPhaseMrank, kPhaseMdup}};
    for (int ph : next[t]) {
      if (ph < 0) continue;
      st = launch_phase(ctx, ph, b, true, s);
      if (st != PQ_OK) return st;
    }
  }
  st = launch_phase(ctx, kPhaseTopk, b, true, s);
  if (st != PQ_OK) return st;
  ctx->plans += n;
  return read_back(ctx, results, out, n, s);
}

}  // namespace pqh
