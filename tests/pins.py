"""Pins for the CPU oracle: checks against things other than the oracle itself
(brute force on tiny inputs, closed forms, invariants, hand-worked examples,
an independently derived hash constant).  Each ``pin_*`` returns None when the
oracle agrees and raises AssertionError otherwise; ``tests/test_oracle_pins.py``
runs them, and ``tests/test_oracle_mutations.py`` shows that every planted
mistake in the oracle trips at least one of them.
"""
from __future__ import annotations

import decimal
import operator
import os

import numpy as np

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PY_OPS = {"<": operator.lt, "<=": operator.le, ">": operator.gt, ">=": operator.ge,
          "==": operator.eq, "!=": operator.ne, "all": lambda a, b: True}


def read_golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            out.setdefault(parts[0], []).append([int(x) for x in parts[1:]])
    return out


def golden_constant() -> int:
    """floor(2^64 / phi) re-derived with 60-digit decimal arithmetic."""
    ctx = decimal.Context(prec=60)
    phi = (decimal.Decimal(1) + decimal.Decimal(5).sqrt(ctx)) / 2
    return int(ctx.divide(decimal.Decimal(2) ** 64, phi).to_integral_value(decimal.ROUND_FLOOR))


def py_bucket(key: int, log2P: int, constant: int) -> int:
    if log2P == 0:
        return 0
    return ((key % 2**64) * constant % 2**64) >> (64 - log2P)


# --------------------------------------------------------------------------
def pin_filter_bruteforce(seed: int = 0):
    rng = np.random.default_rng(seed)
    for dt in (np.int8, np.int32, np.int64):
        for n in (0, 1, 7, 33, 257):
            col = rng.integers(-5, 6, size=n).astype(dt)
            for op in PY_OPS:
                c = int(rng.integers(-6, 7))
                want = [i for i in range(n) if PY_OPS[op](int(col[i]), c)]
                got = oracle.filter(col, op, c)
                assert got.tolist() == want, (dt, n, op, c)
                sel = np.array(sorted(rng.choice(n, size=n // 2, replace=False)) if n else [],
                               dtype=np.int64)
                want2 = [int(r) for r in sel if PY_OPS[op](int(col[r]), c)]
                assert oracle.filter(col, op, c, sel).tolist() == want2


def pin_filter_known():
    col = np.array([5, 1, 7, 3, 5], dtype=np.int32)
    assert oracle.filter(col, "<", 5).tolist() == [1, 3]
    assert oracle.filter(col, "<=", 5).tolist() == [0, 1, 3, 4]
    assert oracle.filter(col, ">", 5).tolist() == [2]
    assert oracle.filter(col, "==", 5).tolist() == [0, 4]
    assert oracle.filter(col, "!=", 5).tolist() == [1, 2, 3]
    assert oracle.filter(col, "all", 0).tolist() == [0, 1, 2, 3, 4]
    assert oracle.filter(col, "<", -100).tolist() == []


def pin_partition_constant_and_known_buckets():
    g = read_golden("fib_hash.txt")
    assert golden_constant() == g["constant"][0][0]
    keys = np.array([k for k, _ in g["bucket4"]], dtype=np.int64)
    rows = np.arange(len(keys), dtype=np.int64)
    _, (prow,), off = oracle.partition(keys, 4, [rows])
    for k, b in g["bucket4"]:
        i = keys.tolist().index(k)
        pos = prow.tolist().index(i)
        assert off[b] <= pos < off[b + 1], (k, b, off)


def pin_partition_invariants(seed: int = 1):
    rng = np.random.default_rng(seed)
    C = golden_constant()
    for dt in (np.int32, np.int64):
        for log2P in (0, 1, 3, 6, 10):
            n = int(rng.integers(0, 3000))
            keys = rng.integers(-10**6, 10**6, size=n).astype(dt)
            rows = np.arange(n, dtype=np.int64)
            tag = rng.integers(-128, 127, size=n).astype(np.int8)
            ok, (orow, otag), off = oracle.partition(keys, log2P, [rows, tag])
            P = 1 << log2P
            assert off[0] == 0 and off[P] == n and np.all(np.diff(off) >= 0)
            assert sorted(orow.tolist()) == list(range(n))           # a permutation
            assert np.array_equal(ok, keys[orow]) and np.array_equal(otag, tag[orow])
            for b in range(P):
                seg = orow[off[b]:off[b + 1]]
                assert np.all(np.diff(seg) > 0)                       # stable
                for r in seg[:20]:
                    assert py_bucket(int(keys[r]), log2P, C) == b
            if log2P == 0:
                assert np.array_equal(ok, keys)                        # identity


def pin_join_bruteforce(seed: int = 2):
    rng = np.random.default_rng(seed)
    for nb, npr in ((0, 5), (5, 0), (40, 60), (200, 300)):
        bk = rng.integers(0, 25, size=nb).astype(np.int64)
        pk = rng.integers(0, 30, size=npr).astype(np.int32)
        bv = rng.integers(-1000, 1000, size=nb).astype(np.int64)
        want = sorted((i, int(bv[j])) for i in range(npr) for j in range(nb)
                      if int(pk[i]) == int(bk[j]))
        rows, vals = oracle.join(bk, pk, bv)
        assert list(zip(rows.tolist(), vals.tolist())) == want
        # closed form: |join| = sum over values v of a_v * b_v
        a = np.bincount(bk, minlength=40) if nb else np.zeros(40, int)
        b = np.bincount(pk, minlength=40) if npr else np.zeros(40, int)
        assert len(rows) == int((a[:40] * b[:40]).sum())
        r2, v2 = oracle.join(bk, pk)                                    # default value: row id
        assert sorted(zip(r2.tolist(), v2.tolist())) == sorted(
            (i, j) for i in range(npr) for j in range(nb) if int(pk[i]) == int(bk[j]))


def pin_groupby_bruteforce(seed: int = 3):
    rng = np.random.default_rng(seed)
    for dt in (np.int8, np.int32, np.int64):
        for n in (0, 1, 50, 999):
            k = rng.integers(-20, 20, size=n).astype(dt)
            v = rng.integers(-10**12, 10**12, size=n).astype(np.int64)
            want = {}
            for i in range(n):
                want[int(k[i])] = want.get(int(k[i]), 0) + int(v[i])
            keys, sums, ovf = oracle.groupby_sum(k, v)
            assert keys.tolist() == sorted(want) and not ovf
            assert sums.tolist() == [want[x] for x in sorted(want)]
            assert int(sums.astype(object).sum()) == int(v.astype(object).sum())  # conservation
    big = np.array([2**62, 2**62, -5], dtype=np.int64)
    _, _, ovf = oracle.groupby_sum(np.array([7, 7, 8], dtype=np.int64), big)
    assert ovf


def pin_topk_bruteforce(seed: int = 4):
    rng = np.random.default_rng(seed)
    for n, k in ((0, 3), (1, 1), (10, 3), (100, 10), (500, 64), (7, 20)):
        keys = rng.permutation(10 * n + 1)[:n].astype(np.int64)
        sums = rng.integers(-5, 5, size=n).astype(np.int64)   # many ties
        order = sorted(range(n), key=lambda i: (-int(sums[i]), int(keys[i])))[:k]
        ok, os_ = oracle.topk(keys, sums, k)
        assert ok.tolist() == [int(keys[i]) for i in order]
        assert os_.tolist() == [int(sums[i]) for i in order]
    ok, os_ = oracle.topk(np.array([3, 1, 2], np.int64), np.array([5, 5, 9], np.int64), 3)
    assert ok.tolist() == [2, 1, 3] and os_.tolist() == [9, 5, 5]


def brute_plan(D, M, F, seg, mc, fc, d_op="==", m_op="<", f_op=">"):
    dset = {int(D["key"][i]) for i in range(len(D["key"]))
            if PY_OPS[d_op](int(D["seg"][i]), seg)}
    sums = {}
    for j in range(len(M["key"])):
        if not (PY_OPS[m_op](int(M["date"][j]), mc) and int(M["dref"][j]) in dset):
            continue
        mk = int(M["key"][j])
        for i in range(len(F["mkey"])):                       # nested-loop join
            if int(F["mkey"][i]) == mk and PY_OPS[f_op](int(F["date2"][i]), fc):
                sums[mk] = sums.get(mk, 0) + int(F["price"][i]) * (100 - int(F["disc"][i]))
    return sums


def pin_plan_golden():
    g = read_golden("tiny_plan.txt")
    D = dict(key=np.array(g["D.key"][0], np.int32), seg=np.array(g["D.seg"][0], np.int8))
    M = dict(key=np.array(g["M.key"][0], np.int64), dref=np.array(g["M.dref"][0], np.int32),
             date=np.array(g["M.date"][0], np.int32))
    F = dict(mkey=np.array(g["F.mkey"][0], np.int64), price=np.array(g["F.price"][0], np.int64),
             disc=np.array(g["F.disc"][0], np.int8), date2=np.array(g["F.date2"][0], np.int32))
    r = oracle.run_plan(D, M, F, seg=1, m_date_lt=1200, f_date_gt=1200, k=10)
    assert r["ngroups"] == g["expect.ngroups"][0][0]
    assert r["keys"].tolist() == g["expect.keys"][0]
    assert r["sums"].tolist() == g["expect.sums"][0]
    r1 = oracle.run_plan(D, M, F, k=1)
    assert r1["keys"].tolist() == g["expect.keys"][0][:1]


def pin_plan_bruteforce(seed: int = 5):
    for trial in range(3):
        D, M, F = datagen.make(50, 500, 2000, seed=100 + seed + trial)
        for (seg, mc, fc) in ((1, 1200, 1200), (0, 2000, 300), (4, 600, 2000)):
            want = brute_plan(D, M, F, seg, mc, fc)
            keys, sums = oracle.plan_groups(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc)
            assert keys.tolist() == sorted(want)
            assert sums.tolist() == [want[x] for x in sorted(want)]
            r = oracle.run_plan(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc, k=10)
            order = sorted(want, key=lambda x: (-want[x], x))[:10]
            assert r["keys"].tolist() == order and r["ngroups"] == len(want)
            assert r["sums"].tolist() == [want[x] for x in order]


def pin_plan_duplicate_build_keys():
    D = dict(key=np.array([1, 2], np.int32), seg=np.array([1, 1], np.int8))
    M = dict(key=np.array([7, 7, 8], np.int64), dref=np.array([1, 2, 1], np.int32),
             date=np.array([0, 0, 0], np.int32))
    F = dict(mkey=np.array([7, 8, 8], np.int64), price=np.array([10, 20, 30], np.int64),
             disc=np.array([0, 0, 50], np.int8), date2=np.array([9, 9, 9], np.int32))
    want = brute_plan(D, M, F, 1, 10, 0)
    assert want == {7: 2 * 1000, 8: 2000 + 1500}
    keys, sums = oracle.plan_groups(D, M, F, seg=1, m_date_lt=10, f_date_gt=0)
    assert dict(zip(keys.tolist(), sums.tolist())) == want


def pin_plan_pass_all_closed_form():
    D, M, F = datagen.make(1000, 10_000, 40_000, seed=11)
    keys, sums = oracle.plan_groups(D, M, F, d_op="all", m_op="all", f_op="all")
    # every foreign key exists and every predicate passes: groups are the
    # distinct F.mkey values and the grand total is sum(price * (100 - disc)).
    assert np.array_equal(keys, np.unique(F["mkey"]))
    total = int((F["price"].astype(np.int64) * (100 - F["disc"].astype(np.int64))).sum())
    assert int(sums.sum()) == total
    r = oracle.run_plan(D, M, F, d_op="all", m_op="all", f_op="all", k=5)
    assert r["ngroups"] == len(keys)
    # the k-th reported sum is >= every sum left out
    assert int(r["sums"][-1]) >= int(np.sort(sums)[-6])


def brute_aggfirst(D, M, F, seg, mc, fc, having):
    """Aggregate-first plan by definition: every group of F (date2 filter),
    kept when sum > having and its key is held by at least one M' row."""
    dset = {int(D["key"][i]) for i in range(len(D["key"])) if int(D["seg"][i]) == seg}
    mkeys = {int(M["key"][j]) for j in range(len(M["key"]))
             if int(M["date"][j]) < mc and int(M["dref"][j]) in dset}
    g = {}
    for i in range(len(F["mkey"])):
        if int(F["date2"][i]) > fc:
            mk = int(F["mkey"][i])
            g[mk] = g.get(mk, 0) + int(F["price"][i]) * (100 - int(F["disc"][i]))
    return {k: v for k, v in g.items() if v > having and k in mkeys}


def pin_aggfirst_bruteforce(seed: int = 12):
    """Brute force with M keys held by several rows and D rows that fail."""
    for trial in range(3):
        D, M, F = datagen.make(40, 300, 1200, seed=200 + seed + trial)
        M = dict(M)
        M["key"] = M["key"].copy()
        M["key"][1::7] = M["key"][0:-1:7][:len(M["key"][1::7])]      # repeated keys
        for (seg, mc, fc) in ((1, 1200, 1200), (0, 2000, 300)):
            for having in (-(1 << 63), 0, 2_000_000_000):
                want = brute_aggfirst(D, M, F, seg, mc, fc, having)
                r = oracle.run_plan_aggfirst(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc,
                                             having=having, k=20)
                order = sorted(want, key=lambda x: (-want[x], x))[:20]
                assert r["ngroups"] == len(want) and r["status"] == 0
                assert r["keys"].tolist() == order
                assert r["sums"].tolist() == [want[x] for x in order]


def pin_aggfirst_threshold_is_strict():
    """A group whose sum equals the threshold is left out; one unit lower
    keeps it (hand-computed: groups 7 -> 1000, 8 -> 2500)."""
    D = dict(key=np.array([1], np.int32), seg=np.array([1], np.int8))
    M = dict(key=np.array([7, 8], np.int64), dref=np.array([1, 1], np.int32),
             date=np.array([0, 0], np.int32))
    F = dict(mkey=np.array([7, 8, 8], np.int64), price=np.array([10, 20, 10], np.int64),
             disc=np.array([0, 0, 50], np.int8), date2=np.array([9, 9, 9], np.int32))
    r = oracle.run_plan_aggfirst(D, M, F, seg=1, m_date_lt=10, f_date_gt=0, having=1000, k=5)
    assert r["keys"].tolist() == [8] and r["sums"].tolist() == [2500] and r["ngroups"] == 1
    r = oracle.run_plan_aggfirst(D, M, F, seg=1, m_date_lt=10, f_date_gt=0, having=999, k=5)
    assert r["keys"].tolist() == [8, 7] and r["sums"].tolist() == [2500, 1000]


def _overflow_tables(prices, discs):
    """One D row, one M row (key 5) and F rows of key 5 that all pass."""
    D = dict(key=np.array([1], np.int32), seg=np.array([1], np.int8))
    M = dict(key=np.array([5], np.int64), dref=np.array([1], np.int32),
             date=np.array([0], np.int32))
    n = len(prices)
    F = dict(mkey=np.full(n, 5, np.int64), price=np.array(prices, np.int64),
             disc=np.array(discs, np.int8), date2=np.full(n, 2000, np.int32))
    return D, M, F


def pin_plan_overflow_status():
    """Status 7 exactly when a group sum leaves int64 (hand-computed edges:
    2^63 - 1 = 73 * 126347562148695559, -2^63 = 64 * -2^57)."""
    top = 126347562148695559          # * (100 - 27) = 2^63 - 1
    cases = [([top], [27], 0, 2**63 - 1),                   # exactly INT64_MAX: fits
             ([top, 1], [27, 99], 7, None),                  # INT64_MAX + 1
             ([-(2**57)], [36], 0, -(2**63)),                # exactly INT64_MIN: fits
             ([-(2**57), -1], [36, 99], 7, None),            # INT64_MIN - 1
             ([2**56, 2**56], [0, 0], 7, None),              # 2 * 100 * 2^56 > 2^63
             ([top, -5], [27, 0], 0, 2**63 - 1 - 500)]       # back inside by a negative row
    for prices, discs, status, total in cases:
        D, M, F = _overflow_tables(prices, discs)
        for agg in (False, True):
            run = oracle.run_plan_aggfirst if agg else oracle.run_plan
            r = run(D, M, F, seg=1, m_date_lt=10, f_date_gt=0)
            assert r["status"] == status, (prices, discs, r["status"])
            if total is None:
                continue
            # the aggregate-first plan keeps sums > having (INT64_MIN by default)
            kept = not agg or total > -(2**63)
            assert r["keys"].tolist() == ([5] if kept else []), (agg, prices)
            assert r["sums"].tolist() == ([total] if kept else [])


ALL_PINS = [pin_filter_bruteforce, pin_filter_known, pin_partition_constant_and_known_buckets,
            pin_partition_invariants, pin_join_bruteforce, pin_groupby_bruteforce,
            pin_topk_bruteforce, pin_plan_golden, pin_plan_bruteforce,
            pin_plan_duplicate_build_keys, pin_plan_pass_all_closed_form,
            pin_aggfirst_bruteforce, pin_aggfirst_threshold_is_strict,
            pin_plan_overflow_status]
