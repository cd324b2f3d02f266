"""Seeded synthetic inputs for the three-table plan (D, M, F).

This module draws inputs only; it contains none of the relational arithmetic.
Both the CUDA path and the CPU oracle read the arrays it returns, so parity
does not depend on the generator.  The C generator (``pqgen.c``) is built on
first use with gcc (OpenMP, ``-O2``), or ahead of time by ``build()``.

Workloads (sizes as named; the query shape follows the paper's running
example, a three-table filter / join / group-by / top-k plan, Sec. 5.1):

* ``small``  -- D 15k, M 150k, F 600k rows (seed 1)
* ``x100``   -- D 1.5M, M 15M, F 60M rows (seed 2)
* ``x2000``  -- D 30M, M 300M, F 1.2B rows (seed 3)
* ``skew``   -- D 4M, M 40M, F 200M rows, Zipf(1.0) foreign keys (seed 4)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pqgen.c")
_LIB = os.path.join(_HERE, "libpqgen.so")
_lock = threading.Lock()
_lib = None

WORKLOADS = {
    "small": dict(n_d=15_000, n_m=150_000, n_f=600_000, seed=1, fk="clustered"),
    "x100": dict(n_d=1_500_000, n_m=15_000_000, n_f=60_000_000, seed=2, fk="clustered"),
    "x2000": dict(n_d=30_000_000, n_m=300_000_000, n_f=1_200_000_000, seed=3, fk="clustered"),
    "skew": dict(n_d=4_000_000, n_m=40_000_000, n_f=200_000_000, seed=4, fk="zipf", zipf_s=1.0),
}

# Predicate constants of the plan: D.seg == 1, M.date < 1200, F.date2 > 1200.
# The skewed workload runs with pass-all predicates so that ~20M groups exist.
QUERY = dict(seg=1, m_date_lt=1200, f_date_gt=1200, k=10)

D_COLS = (("key", np.int32), ("seg", np.int8))
M_COLS = (("key", np.int64), ("dref", np.int32), ("date", np.int32))
F_COLS = (("mkey", np.int64), ("price", np.int64), ("disc", np.int8), ("date2", np.int32))


def build(force: bool = False) -> str:
    """Compile ``libpqgen.so`` next to its source if it is missing or stale."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u64, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.pqgen_d.argtypes = [u64, i64, vp, vp]
        lib.pqgen_m.argtypes = [u64, i64, i64, vp, vp, vp]
        lib.pqgen_f_clustered.argtypes = [u64, i64, i64, vp, vp, vp, vp, vp, vp]
        lib.pqgen_f_zipf.argtypes = [u64, i64, i64, ctypes.c_double, vp, vp, vp, vp, vp, vp]
        lib.pqgen_f_starts.argtypes = [u64, i64, i64, vp]
        lib.pqgen_uniform_i64.argtypes = [u64, u64, i64, i64, i64, vp]
        lib.pqgen_uniform_f64.argtypes = [u64, u64, i64, vp]
        lib.pqgen_threads.restype = ctypes.c_int
        for f in (lib.pqgen_d, lib.pqgen_m, lib.pqgen_f_clustered, lib.pqgen_f_zipf,
                  lib.pqgen_f_starts, lib.pqgen_uniform_i64, lib.pqgen_uniform_f64):
            f.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _alloc(cols, n, out):
    res = {}
    for name, dt in cols:
        if out is not None and name in out:
            a = out[name]
            assert a.dtype == dt and a.shape == (n,), (name, a.dtype, a.shape)
        else:
            a = np.empty(n, dtype=dt)
        res[name] = a
    return res


def gen_d(seed: int, n_d: int, out=None) -> dict:
    d = _alloc(D_COLS, n_d, out)
    _load().pqgen_d(seed, n_d, _p(d["key"]), _p(d["seg"]))
    return d


def gen_m(seed: int, n_m: int, n_d: int, out=None) -> dict:
    m = _alloc(M_COLS, n_m, out)
    _load().pqgen_m(seed, n_m, n_d, _p(m["key"]), _p(m["dref"]), _p(m["date"]))
    return m


def gen_f(seed: int, n_f: int, m: dict, fk: str = "clustered", zipf_s: float = 1.0,
          out=None) -> dict:
    n_m = len(m["key"])
    f = _alloc(F_COLS, n_f, out)
    lib = _load()
    args = (_p(m["key"]), _p(m["date"]), _p(f["mkey"]), _p(f["price"]), _p(f["disc"]),
            _p(f["date2"]))
    if fk == "clustered":
        lib.pqgen_f_clustered(seed, n_f, n_m, *args)
    elif fk == "zipf":
        lib.pqgen_f_zipf(seed, n_f, n_m, float(zipf_s), *args)
    else:
        raise ValueError(fk)
    return f


def f_starts(seed: int, n_m: int, n_f: int) -> np.ndarray:
    """First F row of each M row in the first lap of the clustered generator."""
    s = np.empty(n_m + 1, dtype=np.int64)
    _load().pqgen_f_starts(seed, n_m, n_f, _p(s))
    return s


def make(n_d: int, n_m: int, n_f: int, seed: int, fk: str = "clustered",
         zipf_s: float = 1.0, out=None):
    """Generate (D, M, F) as dicts of numpy arrays.  ``out`` may map
    ``"D"/"M"/"F"`` to dicts of preallocated arrays (e.g. pinned buffers)."""
    out = out or {}
    d = gen_d(seed, n_d, out.get("D"))
    m = gen_m(seed, n_m, n_d, out.get("M"))
    f = gen_f(seed, n_f, m, fk, zipf_s, out.get("F"))
    return d, m, f


def workload(name: str, out=None):
    w = dict(WORKLOADS[name])
    return make(w["n_d"], w["n_m"], w["n_f"], w["seed"], w["fk"], w.get("zipf_s", 1.0), out)


def uniform_i64(seed: int, tag: int, n: int, lo: int, hi: int) -> np.ndarray:
    a = np.empty(n, dtype=np.int64)
    _load().pqgen_uniform_i64(seed, tag, n, lo, hi, _p(a))
    return a


def uniform_f64(seed: int, tag: int, n: int) -> np.ndarray:
    a = np.empty(n, dtype=np.float64)
    _load().pqgen_uniform_f64(seed, tag, n, _p(a))
    return a


def query_stream(seed: int, n_queries: int, n_m: int, starts: np.ndarray, rate_qps: float,
                 median_f: int = 500_000, sigma: float = 1.5, f_min: int = 10_000,
                 f_max: int = 50_000_000, align: int = 16):
    """Serving workload: per query an (M slice, F slice) pair cut from a
    clustered dataset, randomised predicate constants and a Poisson arrival
    time.  F sizes are lognormal(ln median_f, sigma) clipped to [f_min, f_max];
    slice starts are multiples of ``align`` rows.  Returns a list of dicts."""
    n_f_total = int(starts[-1])
    u1 = uniform_f64(seed, 1, n_queries)
    u2 = uniform_f64(seed, 2, n_queries)
    # Box-Muller normal deviates from two uniform streams.
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    sizes = np.clip(np.exp(np.log(median_f) + sigma * z), f_min, min(f_max, n_f_total // 2))
    sizes = sizes.astype(np.int64)
    a_rand = uniform_i64(seed, 3, n_queries, 0, n_m - 1)
    seg = uniform_i64(seed, 4, n_queries, 0, 4)
    c = uniform_i64(seed, 5, n_queries, 0, 2405)
    gaps = -np.log(uniform_f64(seed, 6, n_queries)) / float(rate_qps)
    arrive = np.cumsum(gaps)
    qs = []
    for i in range(n_queries):
        a = int(a_rand[i]) // align * align
        f0 = int(starts[a]) // align * align
        want = int(sizes[i])
        f1 = min(n_f_total, f0 + want)
        b = int(np.searchsorted(starts, f1, side="left"))
        b = min(n_m, (b + align - 1) // align * align)
        f1 = f1 // align * align if f1 < n_f_total else f1
        if f1 <= f0:
            f1 = min(n_f_total, f0 + align)
        qs.append(dict(m_row0=a, m_rows=max(0, b - a), f_row0=f0, f_rows=f1 - f0,
                       seg=int(seg[i]), c=int(c[i]), arrive_s=float(arrive[i])))
    return qs
