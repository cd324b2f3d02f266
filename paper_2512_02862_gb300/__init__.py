"""Python binding of libpq (the C ABI in ``include/pq.h``).

Argument marshalling only: every step of every operator runs in the CUDA
kernels of ``libpq.so``.  PyTorch provides device memory (the arena and
output tensors) and streams.  If the library is missing, importing the
binding's functions raises: there is no CPU fallback.

Function names follow the C ABI (``pq_filter``, ``pq_partition``,
``pq_join_build``/``pq_join_probe``, ``pq_groupby_sum``, ``pq_topk``,
``pq_load_columns``, ``pq_run_plan``, ``pq_run_batch``, ``pq_submit``/
``pq_poll``, ``pq_autotune``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64,
                    c_uint64, c_void_p)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpq.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pq.h")

PQ_MAX_K = 64
PQ_MAX_PAYLOAD = 8
PQ_MAX_LOG2P = 12

STATUS = {0: "PQ_OK", 1: "PQ_ERR_INVALID_ARG", 2: "PQ_ERR_BUDGET", 3: "PQ_ERR_CAPACITY",
          4: "PQ_ERR_CUDA", 5: "PQ_ERR_IO", 6: "PQ_ERR_TIMEOUT", 7: "PQ_ERR_OVERFLOW",
          8: "PQ_ERR_BUSY", 9: "PQ_ERR_RESERVED_KEY"}
PQ_OK, PQ_ERR_INVALID_ARG, PQ_ERR_BUDGET, PQ_ERR_CAPACITY, PQ_ERR_CUDA = 0, 1, 2, 3, 4
PQ_ERR_IO, PQ_ERR_TIMEOUT, PQ_ERR_OVERFLOW, PQ_ERR_BUSY, PQ_ERR_RESERVED_KEY = 5, 6, 7, 8, 9

PQ_INT8, PQ_INT32, PQ_INT64 = 1, 2, 3
CMP = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5, "all": 6}
PQ_SRC_DEVICE, PQ_SRC_HOST, PQ_SRC_FILE, PQ_SRC_PACKED = 0, 1, 2, 3
PQ_PACK_BLOCK = 4096
PQ_RESIDENT, PQ_STREAMING, PQ_MAPPED = 0, 1, 2
PQ_PLAN_PARTITIONED, PQ_PLAN_CACHE_DSET, PQ_PLAN_NO_GRAPH = 1, 2, 4


class pq_col(Structure):
    _fields_ = [("data", c_void_p), ("n", c_int64), ("type", c_int32), ("reserved", c_int32)]


class pq_options(Structure):
    _fields_ = [("block_threads", c_int32), ("blocks_per_sm", c_int32), ("load_factor", c_float),
                ("log2P", c_int32), ("chunk_bytes", c_int64), ("ingest_threads", c_int32),
                ("copy_streams", c_int32), ("ring_slots", c_int32), ("serve_slots", c_int32),
                ("spin_limit", c_int64), ("serve_queue", c_int32), ("profile", c_int32),
                ("hit_buffer", c_int32), ("reserved", c_int32 * 5)]


class pq_stats(Structure):
    _fields_ = [("kernel_launches", c_int64), ("h2d_bytes", c_int64), ("d2h_bytes", c_int64),
                ("arena_bytes", c_int64), ("arena_in_use", c_int64),
                ("arena_high_water", c_int64), ("chunks_ingested", c_int64),
                ("plans_run", c_int64), ("graph_replays", c_int64),
                ("out_of_core_passes", c_int64), ("reserved", c_int64 * 6)]


class pq_source(Structure):
    _fields_ = [("kind", c_int32), ("type", c_int32), ("ptr", c_void_p), ("path", c_char_p),
                ("offset", c_int64)]


class pq_plan(Structure):
    _fields_ = [("D", c_void_p), ("M", c_void_p), ("F", c_void_p),
                ("d_row0", c_int64), ("d_rows", c_int64), ("m_row0", c_int64),
                ("m_rows", c_int64), ("f_row0", c_int64), ("f_rows", c_int64),
                ("d_op", c_int32), ("m_op", c_int32), ("f_op", c_int32), ("k", c_int32),
                ("d_c", c_int64), ("m_c", c_int64), ("f_c", c_int64),
                ("flags", c_int32), ("log2P", c_int32), ("load_factor", c_float),
                ("reserved", c_int32), ("having", c_int64)]


class pq_result(Structure):
    _fields_ = [("n", c_int64), ("ngroups", c_int64), ("keys", c_int64 * PQ_MAX_K),
                ("sums", c_int64 * PQ_MAX_K), ("status", c_int32), ("reserved", c_int32),
                ("hits", c_int64)]

    def as_dict(self):
        n = int(self.n)
        return dict(keys=list(self.keys[:n]), sums=list(self.sums[:n]),
                    ngroups=int(self.ngroups), status=int(self.status))


class pq_tuning(Structure):
    _fields_ = [("block_threads", c_int32), ("blocks_per_sm", c_int32), ("log2P", c_int32),
                ("partitioned", c_int32), ("load_factor", c_float), ("best_ms", c_float),
                ("tried", c_int32), ("reserved", c_int32 * 5)]


_lib = None


def library():
    """Load libpq.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = c_void_p, c_int64, c_int
    sigs = {
        "pq_default_options": [POINTER(pq_options)],
        "pq_create": [POINTER(pq_options), vp, ctypes.c_size_t, POINTER(vp)],
        "pq_destroy": [vp],
        "pq_sync": [vp, vp],
        "pq_get_stats": [vp, POINTER(pq_stats)],
        "pq_profile_read": [vp, c_char_p, POINTER(c_double), POINTER(c_int64)],
        "pq_profile_reset": [vp],
        "pq_profile_enable": [vp, c_int32],
        "pq_load_columns": [vp, POINTER(pq_source), i32, i64, i32, POINTER(vp), vp],
        "pq_table_free": [vp, vp, vp],
        "pq_ht_free": [vp, vp, vp],
        "pq_filter": [vp, pq_col, i32, i64, vp, i64, vp, vp, vp, vp],
        "pq_partition": [vp, pq_col, POINTER(pq_col), i32, i32, vp, POINTER(vp), vp, vp],
        "pq_join_build": [vp, pq_col, pq_col, c_float, POINTER(vp), vp],
        "pq_join_probe": [vp, vp, pq_col, vp, vp, i64, vp, vp],
        "pq_groupby_sum": [vp, pq_col, pq_col, vp, vp, i64, vp, vp],
        "pq_topk": [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp],
        "pq_run_plan": [vp, POINTER(pq_plan), POINTER(pq_result), vp],
        "pq_run_batch": [vp, POINTER(pq_plan), i32, POINTER(pq_result), vp],
        "pq_submit": [vp, POINTER(pq_plan), POINTER(c_uint64)],
        "pq_poll": [vp, c_uint64, POINTER(pq_result), i32],
        "pq_autotune": [vp, POINTER(pq_plan), POINTER(pq_tuning)],
        "pq_filter_noalloc": [pq_col, i32, i64, vp, i64, vp, vp, vp, vp],
        "pq_pack_column": [vp, i32, i64, vp, i64, POINTER(c_int64)],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c_int
    lib.pq_last_error.argtypes = [vp]
    lib.pq_last_error.restype = c_char_p
    lib.pq_status_string.argtypes = [c_int]
    lib.pq_status_string.restype = c_char_p
    lib.pq_table_rows.argtypes = [vp]
    lib.pq_table_rows.restype = c_int64
    lib.pq_table_column.argtypes = [vp, c_int]
    lib.pq_table_column.restype = c_void_p
    lib.pq_last_latency_us.argtypes = [vp]
    lib.pq_last_latency_us.restype = c_double
    lib.pq_pack_bound.argtypes = [i64, c_int32]
    lib.pq_pack_bound.restype = c_int64
    _lib = lib
    return lib


def header_symbols() -> list[str]:
    """Function names declared in include/pq.h."""
    import re
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(pq_[a-z0-9_]+)\(", text)))


class PQError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


# --------------------------------------------------------------- helpers ----
def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    return {torch.int8: PQ_INT8, torch.int32: PQ_INT32, torch.int64: PQ_INT64}[t.dtype]


def col(t) -> pq_col:
    """pq_col view of a 1-D contiguous int8/int32/int64 CUDA tensor."""
    assert t.is_cuda and t.dim() == 1 and t.is_contiguous(), "columns are 1-D contiguous CUDA"
    return pq_col(t.data_ptr() if t.numel() else None, t.numel(), _dtype_code(t), 0)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


# Arenas of contexts that pq_destroy could not release (kept until exit).
_KEPT_ALIVE: list = []


class Context:
    """A libpq context over a device arena of ``arena_bytes`` (the budget)."""

    def __init__(self, arena_bytes: int = 4 << 30, device=None, **options):
        torch = _torch()
        lib = library()
        self.device = torch.device(device) if device is not None else torch.device("cuda", 0)
        torch.cuda.set_device(self.device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        opt = pq_options()
        lib.pq_default_options(ctypes.byref(opt))
        for k, v in options.items():
            setattr(opt, k, v)
        h = c_void_p()
        self._check(lib.pq_create(ctypes.byref(opt), c_void_p(self.arena.data_ptr()),
                                  int(arena_bytes), ctypes.byref(h)), None)
        self.h = h
        self.tables = []

    def _check(self, st, h=None):
        if st != PQ_OK:
            lib = library()
            msg = lib.pq_last_error(h if h is not None else getattr(self, "h", None))
            raise PQError(st, (msg or b"").decode())

    def check(self, st):
        self._check(st, self.h)

    def close(self):
        """pq_destroy.  If a served batch did not finish in time the library
        keeps the context (its memory may still be in use on the device), so
        the arena is kept alive too and PQError(PQ_ERR_TIMEOUT) is raised."""
        if getattr(self, "h", None):
            st = library().pq_destroy(self.h)
            self.h = None
            if st != PQ_OK:
                _KEPT_ALIVE.append(self.arena)
                raise PQError(st, "pq_destroy: a served batch did not complete")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        """pq_sync: wait for the stream, raise the first device-latched error."""
        self.check(library().pq_sync(self.h, _stream(stream)))

    def stats(self) -> dict:
        s = pq_stats()
        self.check(library().pq_get_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in pq_stats._fields_ if f != "reserved"}

    def profile(self, name: str):
        ms, n = c_double(0), c_int64(0)
        self.check(library().pq_profile_read(self.h, name.encode(), ctypes.byref(ms),
                                             ctypes.byref(n)))
        return ms.value, n.value

    def profile_reset(self):
        self.check(library().pq_profile_reset(self.h))

    def profile_enable(self, on: bool):
        """Per-kernel event timing on or off for the calls issued after this."""
        self.check(library().pq_profile_enable(self.h, 1 if on else 0))


# -------------------------------------------------------------- operators ----
def pq_filter(ctx: Context, column, op: str, c: int, sel_in=None, d_n_in=None, stream=None):
    """Ascending row ids with ``column op c`` (AND ``sel_in`` if given).
    Returns (sel_out tensor sized to capacity, d_count device tensor)."""
    torch = _torch()
    n_cap = column.numel() if sel_in is None else sel_in.numel()
    out = torch.empty(max(n_cap, 1), dtype=torch.int64, device=column.device)
    d_count = torch.empty(1, dtype=torch.int64, device=column.device)
    ctx.check(library().pq_filter(ctx.h, col(column), CMP[op], int(c), _ptr(sel_in), n_cap,
                                  _ptr(d_n_in), out.data_ptr(), d_count.data_ptr(),
                                  _stream(stream)))
    return out, d_count


def pq_partition(ctx: Context, key, payloads=(), log2P: int = 6, stream=None):
    """Radix partition by Fibonacci hash of ``key``.  Returns
    (out_key, [out_payloads], d_offsets[P + 1])."""
    torch = _torch()
    out_key = torch.empty_like(key)
    out_pay = [torch.empty_like(p) for p in payloads]
    d_off = torch.empty((1 << log2P) + 1, dtype=torch.int64, device=key.device)
    pc = (pq_col * max(1, len(payloads)))(*[col(p) for p in payloads])
    op = (c_void_p * max(1, len(payloads)))(*[p.data_ptr() if p.numel() else None
                                              for p in out_pay])
    ctx.check(library().pq_partition(ctx.h, col(key), pc, len(payloads), int(log2P),
                                     _ptr(out_key) if key.numel() else None, op,
                                     d_off.data_ptr(), _stream(stream)))
    return out_key, out_pay, d_off


class HashTable:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def free(self, stream=None):
        if self.h:
            self.ctx.check(library().pq_ht_free(self.ctx.h, self.h, _stream(stream)))
            self.h = None


def pq_join_build(ctx: Context, key, val=None, load_factor: float = 0.0, stream=None):
    h = c_void_p()
    v = col(val) if val is not None else pq_col(None, key.numel(), PQ_INT64, 0)
    ctx.check(library().pq_join_build(ctx.h, col(key), v, float(load_factor), ctypes.byref(h),
                                      _stream(stream)))
    return HashTable(ctx, h)


def pq_join_probe(ctx: Context, ht: HashTable, probe_key, cap: int, stream=None):
    """Returns (out_probe_row, out_build_val, d_count); at most ``cap`` pairs."""
    torch = _torch()
    rows = torch.empty(max(cap, 1), dtype=torch.int64, device=probe_key.device)
    vals = torch.empty(max(cap, 1), dtype=torch.int64, device=probe_key.device)
    d_count = torch.empty(1, dtype=torch.int64, device=probe_key.device)
    ctx.check(library().pq_join_probe(ctx.h, ht.h, col(probe_key), rows.data_ptr(),
                                      vals.data_ptr(), int(cap), d_count.data_ptr(),
                                      _stream(stream)))
    return rows, vals, d_count


def pq_groupby_sum(ctx: Context, key, val, cap: int, stream=None):
    """Returns (out_keys, out_sums, d_ngroups); at most ``cap`` groups."""
    torch = _torch()
    ok = torch.empty(max(cap, 1), dtype=torch.int64, device=key.device)
    os_ = torch.empty(max(cap, 1), dtype=torch.int64, device=key.device)
    d_ng = torch.empty(1, dtype=torch.int64, device=key.device)
    ctx.check(library().pq_groupby_sum(ctx.h, col(key), col(val), ok.data_ptr(), os_.data_ptr(),
                                       int(cap), d_ng.data_ptr(), _stream(stream)))
    return ok, os_, d_ng


def pq_topk(ctx: Context, keys, sums, k: int, d_n=None, stream=None):
    """Returns (out_keys[k], out_sums[k], d_nout)."""
    torch = _torch()
    ok = torch.empty(k, dtype=torch.int64, device=keys.device)
    os_ = torch.empty(k, dtype=torch.int64, device=keys.device)
    d_nout = torch.empty(1, dtype=torch.int64, device=keys.device)
    ctx.check(library().pq_topk(ctx.h, _ptr(keys) if keys.numel() else None,
                                _ptr(sums) if sums.numel() else None, keys.numel(), _ptr(d_n),
                                int(k), ok.data_ptr(), os_.data_ptr(), d_nout.data_ptr(),
                                _stream(stream)))
    return ok, os_, d_nout


# ------------------------------------------------------------------ tables ----
class Table:
    def __init__(self, ctx, h, keep):
        self.ctx, self.h, self._keep = ctx, h, keep

    @property
    def rows(self) -> int:
        return library().pq_table_rows(self.h)

    def column_ptr(self, i: int):
        return library().pq_table_column(self.h, i)

    def free(self, stream=None):
        if self.h:
            self.ctx.check(library().pq_table_free(self.ctx.h, self.h, _stream(stream)))
            self.h = None


class Packed:
    """A packed column (frame of reference + bit packing, pq_pack_column) in a
    byte buffer: ``data`` (a pinned uint8 tensor unless packed with
    ``pinned=False``), the column type code and its row count."""

    def __init__(self, data, type_code: int, nrows: int):
        self.data, self.type, self.nrows = data, type_code, nrows

    @property
    def nbytes(self) -> int:
        return int(self.data.numel())


def pq_pack_column(column, pinned: bool = True) -> Packed:
    """Pack a host column (numpy array or CPU tensor) on the host."""
    import numpy as np
    torch = _torch()
    a = column.numpy() if isinstance(column, torch.Tensor) else np.ascontiguousarray(column)
    code = {np.dtype(np.int8): PQ_INT8, np.dtype(np.int32): PQ_INT32,
            np.dtype(np.int64): PQ_INT64}[a.dtype]
    n = len(a)
    cap = library().pq_pack_bound(n, code)
    buf = torch.empty(cap, dtype=torch.uint8, pin_memory=pinned)
    used = c_int64(0)
    st = library().pq_pack_column(a.ctypes.data if n else None, code, n, buf.data_ptr(), cap,
                                  ctypes.byref(used))
    if st != 0:
        raise PQError(st, "pq_pack_column")
    return Packed(buf[:used.value], code, n)


def pq_load_columns(ctx: Context, columns, mode: int = PQ_RESIDENT, stream=None) -> Table:
    """Load a table.  ``columns`` are CUDA tensors (borrowed), CPU tensors or
    numpy arrays (host memory; pinned tensors are copied directly), or
    ``(path, dtype_code, offset)`` tuples for raw column files."""
    import numpy as np
    torch = _torch()
    srcs = (pq_source * len(columns))()
    keep = []
    nrows = None
    for i, c in enumerate(columns):
        if isinstance(c, Packed):
            keep.append(c)
            n = c.nrows
            srcs[i] = pq_source(PQ_SRC_PACKED, c.type, c.data.data_ptr(), None, 0)
        elif isinstance(c, tuple):
            path, code, off, n = c
            p = path.encode()
            keep.append(p)
            srcs[i] = pq_source(PQ_SRC_FILE, code, None, p, int(off))
        elif isinstance(c, np.ndarray):
            code = {np.dtype(np.int8): PQ_INT8, np.dtype(np.int32): PQ_INT32,
                    np.dtype(np.int64): PQ_INT64}[c.dtype]
            assert c.flags["C_CONTIGUOUS"]
            keep.append(c)
            n = len(c)
            srcs[i] = pq_source(PQ_SRC_HOST, code, c.ctypes.data, None, 0)
        else:
            assert isinstance(c, torch.Tensor) and c.dim() == 1 and c.is_contiguous()
            keep.append(c)
            n = c.numel()
            kind = PQ_SRC_DEVICE if c.is_cuda else PQ_SRC_HOST
            srcs[i] = pq_source(kind, _dtype_code(c), c.data_ptr(), None, 0)
        nrows = n if nrows is None else nrows
        assert n == nrows, "all columns need the same row count"
    h = c_void_p()
    ctx.check(library().pq_load_columns(ctx.h, srcs, len(columns), int(nrows or 0), int(mode),
                                        ctypes.byref(h), _stream(stream)))
    t = Table(ctx, h, keep)
    ctx.tables.append(t)
    return t


# ------------------------------------------------------------------- plans ----
PQ_PLAN_AGG_FIRST = 8


def make_plan(D: Table, M: Table, F: Table, seg=1, m_date_lt=1200, f_date_gt=1200, k=10,
              d_op="==", m_op="<", f_op=">", rows=None, flags=0, log2P=0,
              load_factor=0.0, having=None) -> pq_plan:
    """The three-table plan: D.seg d_op seg, M.date m_op m_date_lt,
    F.date2 f_op f_date_gt; ``rows`` = dict(d=(row0, n), m=..., f=...).
    ``having`` given: the aggregate-first plan (groups of F by mkey with
    sum > having whose key is in M')."""
    rows = rows or {}
    d0, dn = rows.get("d", (0, -1))
    m0, mn = rows.get("m", (0, -1))
    f0, fn = rows.get("f", (0, -1))
    if having is not None:
        flags |= PQ_PLAN_AGG_FIRST
    return pq_plan(D.h, M.h, F.h, d0, dn, m0, mn, f0, fn, CMP[d_op], CMP[m_op], CMP[f_op], k,
                   seg, m_date_lt, f_date_gt, flags, log2P, load_factor, 0,
                   int(having) if having is not None else 0)


def pinned_results(n: int):
    """A page-locked array of n pq_result records (asynchronous read-back)."""
    torch = _torch()
    buf = torch.empty(n * ctypes.sizeof(pq_result), dtype=torch.uint8, pin_memory=True)
    arr = (pq_result * n).from_address(buf.data_ptr())
    arr._buf = buf
    return arr


def pq_run_plan(ctx: Context, plan: pq_plan, result=None, stream=None):
    """Run one plan.  With ``result`` from pinned_results() the call is
    asynchronous (valid after ctx.sync()); otherwise it waits."""
    res = result if result is not None else pq_result()
    ctx.check(library().pq_run_plan(ctx.h, ctypes.byref(plan), ctypes.byref(res),
                                    _stream(stream)))
    return res


def pq_run_batch(ctx: Context, plans, results=None, stream=None):
    n = len(plans)
    arr = (pq_plan * n)(*plans)
    res = results if results is not None else (pq_result * n)()
    ctx.check(library().pq_run_batch(ctx.h, arr, n, res, _stream(stream)))
    return res


def pq_submit(ctx: Context, plan: pq_plan) -> int:
    t = c_uint64(0)
    ctx.check(library().pq_submit(ctx.h, ctypes.byref(plan), ctypes.byref(t)))
    return t.value


def pq_poll(ctx: Context, ticket: int, timeout_ms: int = -1):
    """(status, pq_result, latency_us); status PQ_ERR_TIMEOUT if not done."""
    res = pq_result()
    st = library().pq_poll(ctx.h, c_uint64(ticket), ctypes.byref(res), int(timeout_ms))
    if st not in (PQ_OK, PQ_ERR_TIMEOUT) and res.status == 0:
        ctx.check(st)
    return st, res, library().pq_last_latency_us(ctx.h)


def pq_autotune(ctx: Context, plan: pq_plan) -> dict:
    t = pq_tuning()
    ctx.check(library().pq_autotune(ctx.h, ctypes.byref(plan), ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in pq_tuning._fields_ if f != "reserved"}
