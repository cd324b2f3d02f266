"""Helpers shared by the GPU tests: device copies of generated tables and the
plan/oracle comparison."""
import numpy as np

import oracle


def to_dev(tab: dict):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in tab.items()}


def load_tables(pq, ctx, D, M, F, stream=None, mode=None):
    d, m, f = to_dev(D), to_dev(M), to_dev(F)
    TD = pq.pq_load_columns(ctx, [d["key"], d["seg"]], stream=stream)
    TM = pq.pq_load_columns(ctx, [m["key"], m["dref"], m["date"]], stream=stream)
    TF = pq.pq_load_columns(ctx, [f["mkey"], f["price"], f["disc"], f["date2"]], stream=stream)
    return TD, TM, TF, (d, m, f)


def oracle_plan(D, M, F, seg=1, mc=1200, fc=1200, k=10, d_op="==", m_op="<", f_op=">",
                rows=None):
    rows = rows or {}

    def cut(tab, key):
        if key not in rows:
            return tab
        r0, n = rows[key]
        n = len(next(iter(tab.values()))) - r0 if n < 0 else n
        return {c: v[r0:r0 + n] for c, v in tab.items()}

    return oracle.run_plan(cut(D, "d"), cut(M, "m"), cut(F, "f"), seg=seg, m_date_lt=mc,
                           f_date_gt=fc, k=k, d_op=d_op, m_op=m_op, f_op=f_op)


def assert_same(got: dict, want: dict, ctx=""):
    assert got["status"] == want.get("status", 0), (ctx, got["status"])
    assert got["ngroups"] == want["ngroups"], (ctx, got["ngroups"], want["ngroups"])
    assert got["keys"] == list(map(int, want["keys"])), (ctx, got["keys"][:5],
                                                         list(want["keys"][:5]))
    assert got["sums"] == list(map(int, want["sums"])), (ctx, got["sums"][:5],
                                                         list(want["sums"][:5]))
