"""CPU oracle for the relational hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``oracle.cpp`` (plain single-threaded
C++17 written from the relational definitions) through ctypes and numpy, and
shares no code with the CUDA library.

Parity status of each function (the pins live in ``tests/test_oracle_pins.py``):
  filter, partition, join, groupby_sum, topk, run_plan, plan_groups -- pinned
  by brute force on tiny inputs, closed forms, invariants, a hand-worked
  example (``tests/golden/``); ``tests/test_oracle_mutations.py`` compiles
  copies of oracle.cpp with one deliberate mistake each and checks that the
  pins catch every one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPE_CODE = {np.dtype(np.int8): 1, np.dtype(np.int32): 2, np.dtype(np.int64): 3}
CMP = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5, "all": 6}


def build(force: bool = False) -> str:
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    if True:  # argument types of every exported routine
        lib.oracle_filter.argtypes = [vp, i32, i64, i32, i64, vp, i64, vp]
        lib.oracle_filter.restype = i64
        lib.oracle_partition.argtypes = [vp, i32, i64, i32, i32, vp, vp, vp, vp, vp]
        lib.oracle_partition.restype = i32
        lib.oracle_join.argtypes = [vp, i32, vp, i64, vp, i32, i64, vp, vp, i64]
        lib.oracle_join.restype = i64
        lib.oracle_groupby_sum.argtypes = [vp, i32, vp, i64, vp, vp, i64, vp]
        lib.oracle_groupby_sum.restype = i64
        lib.oracle_topk.argtypes = [vp, vp, i64, i32, vp, vp]
        lib.oracle_topk.restype = i64
        plan = [vp, vp, i64, vp, vp, vp, i64, vp, vp, vp, vp, i64, i32, i64, i32, i64, i32, i64]
        lib.oracle_run_plan.argtypes = plan + [i32, vp, vp, vp, vp]
        lib.oracle_run_plan.restype = i32
        lib.oracle_plan_groups.argtypes = plan + [vp, vp, i64]
        lib.oracle_plan_groups.restype = i64
        lib.oracle_run_plan_aggfirst.argtypes = plan + [i64, i32, vp, vp, vp, vp]
        lib.oracle_run_plan_aggfirst.restype = i32
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_LIB)
    return _lib


class variant:
    """Context manager for the mutation tests: while it is active, every
    function of this module calls the library compiled at ``path`` (a copy
    of oracle.cpp with one deliberate mistake) instead of the oracle."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _p(a):
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], type(a)
    return a.ctypes.data


def filter(col: np.ndarray, op: str, c: int, sel_in: np.ndarray | None = None) -> np.ndarray:
    n_in = len(sel_in) if sel_in is not None else len(col)
    out = np.empty(max(n_in, 1), dtype=np.int64)
    cnt = _load().oracle_filter(_p(col), DTYPE_CODE[col.dtype], len(col), CMP[op], int(c),
                                _p(sel_in), n_in, _p(out))
    return out[:cnt].copy()


def partition(key: np.ndarray, log2P: int, payloads=()):
    n = len(key)
    P = 1 << log2P
    out_key = np.empty(max(n, 1), dtype=key.dtype)
    out_pay = [np.empty(max(n, 1), dtype=p.dtype) for p in payloads]
    offsets = np.empty(P + 1, dtype=np.int64)
    pay_ptrs = (ctypes.c_void_p * max(1, len(payloads)))(*[_p(p) for p in payloads])
    out_ptrs = (ctypes.c_void_p * max(1, len(payloads)))(*[_p(p) for p in out_pay])
    types = (ctypes.c_int * max(1, len(payloads)))(*[DTYPE_CODE[p.dtype] for p in payloads])
    rc = _load().oracle_partition(_p(key), DTYPE_CODE[key.dtype], n, log2P, len(payloads),
                                  ctypes.cast(pay_ptrs, ctypes.c_void_p),
                                  ctypes.cast(types, ctypes.c_void_p), _p(out_key),
                                  ctypes.cast(out_ptrs, ctypes.c_void_p), _p(offsets))
    if rc != 0:
        raise ValueError(f"oracle_partition status {rc}")
    return out_key[:n], [p[:n] for p in out_pay], offsets


def join(build_key: np.ndarray, probe_key: np.ndarray, build_val: np.ndarray | None = None):
    """All (probe row, build value) pairs, sorted."""
    lib = _load()
    args = (_p(build_key), DTYPE_CODE[build_key.dtype], _p(build_val), len(build_key),
            _p(probe_key), DTYPE_CODE[probe_key.dtype], len(probe_key))
    total = lib.oracle_join(*args, None, None, 0)
    rows = np.empty(max(total, 1), dtype=np.int64)
    vals = np.empty(max(total, 1), dtype=np.int64)
    lib.oracle_join(*args, _p(rows), _p(vals), total)
    return rows[:total], vals[:total]


def groupby_sum(key: np.ndarray, val: np.ndarray):
    """(keys sorted ascending, exact sums, overflow flag)."""
    val = np.ascontiguousarray(val, dtype=np.int64)
    n = len(key)
    ok = np.empty(max(n, 1), dtype=np.int64)
    os_ = np.empty(max(n, 1), dtype=np.int64)
    ovf = ctypes.c_int(0)
    g = _load().oracle_groupby_sum(_p(key), DTYPE_CODE[key.dtype], _p(val), n, _p(ok), _p(os_),
                                   n, ctypes.addressof(ovf))
    return ok[:g].copy(), os_[:g].copy(), bool(ovf.value)


def topk(keys: np.ndarray, sums: np.ndarray, k: int):
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    sums = np.ascontiguousarray(sums, dtype=np.int64)
    ok = np.empty(max(k, 1), dtype=np.int64)
    os_ = np.empty(max(k, 1), dtype=np.int64)
    m = _load().oracle_topk(_p(keys), _p(sums), len(keys), k, _p(ok), _p(os_))
    return ok[:m].copy(), os_[:m].copy()


def _plan_args(D, M, F, d_op, d_c, m_op, m_c, f_op, f_c):
    return (_p(D["key"]), _p(D["seg"]), len(D["key"]), _p(M["key"]), _p(M["dref"]),
            _p(M["date"]), len(M["key"]), _p(F["mkey"]), _p(F["price"]), _p(F["disc"]),
            _p(F["date2"]), len(F["mkey"]), CMP[d_op], int(d_c), CMP[m_op], int(m_c),
            CMP[f_op], int(f_c))


def run_plan(D: dict, M: dict, F: dict, seg=1, m_date_lt=1200, f_date_gt=1200, k=10,
             d_op="==", m_op="<", f_op=">"):
    """Top-k (keys, sums), number of groups and status (0 ok, 7 overflow)."""
    ok = np.empty(max(k, 1), dtype=np.int64)
    os_ = np.empty(max(k, 1), dtype=np.int64)
    n_out = ctypes.c_int64(0)
    ng = ctypes.c_int64(0)
    st = _load().oracle_run_plan(*_plan_args(D, M, F, d_op, seg, m_op, m_date_lt, f_op,
                                             f_date_gt), k, _p(ok), _p(os_),
                                 ctypes.addressof(n_out), ctypes.addressof(ng))
    return dict(keys=ok[:n_out.value].copy(), sums=os_[:n_out.value].copy(),
                ngroups=int(ng.value), status=int(st))


def run_plan_aggfirst(D: dict, M: dict, F: dict, seg=1, m_date_lt=1200, f_date_gt=1200,
                      having=-(1 << 63), k=10, d_op="==", m_op="<", f_op=">"):
    """The aggregate-first plan: F grouped by mkey (date2 filter), groups with
    sum > having whose key is in M' (semi-join), top-k."""
    ok = np.empty(max(k, 1), dtype=np.int64)
    os_ = np.empty(max(k, 1), dtype=np.int64)
    n_out = ctypes.c_int64(0)
    ng = ctypes.c_int64(0)
    st = _load().oracle_run_plan_aggfirst(
        *_plan_args(D, M, F, d_op, seg, m_op, m_date_lt, f_op, f_date_gt), int(having), k,
        _p(ok), _p(os_), ctypes.addressof(n_out), ctypes.addressof(ng))
    return dict(keys=ok[:n_out.value].copy(), sums=os_[:n_out.value].copy(),
                ngroups=int(ng.value), status=int(st))


def plan_groups(D: dict, M: dict, F: dict, seg=1, m_date_lt=1200, f_date_gt=1200,
                d_op="==", m_op="<", f_op=">"):
    """Every group of the plan as (keys ascending, sums)."""
    lib = _load()
    args = _plan_args(D, M, F, d_op, seg, m_op, m_date_lt, f_op, f_date_gt)
    g = lib.oracle_plan_groups(*args, None, None, 0)
    ok = np.empty(max(g, 1), dtype=np.int64)
    os_ = np.empty(max(g, 1), dtype=np.int64)
    lib.oracle_plan_groups(*args, _p(ok), _p(os_), g)
    return ok[:g].copy(), os_[:g].copy()
