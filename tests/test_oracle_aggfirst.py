"""Pins of the oracle's aggregate-first plan (F grouped by mkey under the
date2 filter, groups with sum > having whose key is in M', top-k), no GPU:
Python brute force on tiny inputs, the join-first plan it must equal when
nothing is filtered on the aggregate and the M keys are unique, and the
group count as a function of the threshold."""
import numpy as np
import pytest

import datagen
import oracle


def brute(D, M, F, seg, mc, fc, having, k):
    dset = {int(k_) for k_, s in zip(D["key"], D["seg"]) if s == seg}
    mkeys = {int(k_) for k_, dr, dt in zip(M["key"], M["dref"], M["date"])
             if dt < mc and int(dr) in dset}
    g = {}
    for mk, p, d, d2 in zip(F["mkey"], F["price"], F["disc"], F["date2"]):
        if d2 > fc:
            g[int(mk)] = g.get(int(mk), 0) + int(p) * (100 - int(d))
    keep = [(s, k_) for k_, s in g.items() if s > having and k_ in mkeys]
    keep.sort(key=lambda x: (-x[0], x[1]))
    return [k_ for _, k_ in keep[:k]], [s for s, _ in keep[:k]], len(keep)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("having", [-(1 << 63), 0, 50_000_000_000, 300_000_000_000])
def test_brute_force(seed, having):
    D, M, F = datagen.make(30, 200, 800, seed=seed)
    rng = np.random.default_rng(seed)
    M = dict(M)
    M["key"] = M["key"].copy()
    M["key"][rng.integers(0, 200, 20)] = M["key"][rng.integers(0, 200, 20)]   # repeated keys
    for seg, mc, fc in ((1, 1200, 1200), (0, 2400, 0), (3, 600, 900)):
        want_k, want_s, want_n = brute(D, M, F, seg, mc, fc, having, 15)
        got = oracle.run_plan_aggfirst(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc,
                                       having=having, k=15)
        assert got["status"] == 0
        assert got["keys"].tolist() == want_k and got["sums"].tolist() == want_s
        assert got["ngroups"] == want_n


def test_equals_join_first_plan_without_a_threshold():
    """Unique M keys and no threshold: the groups of the aggregate-first plan
    are those of the join-first plan (same keys, same sums)."""
    D, M, F = datagen.make(2000, 20_000, 80_000, seed=5)
    for seg, mc, fc in ((1, 1200, 1200), (4, 2000, 300)):
        a = oracle.run_plan_aggfirst(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc, k=50)
        b = oracle.run_plan(D, M, F, seg=seg, m_date_lt=mc, f_date_gt=fc, k=50)
        assert a["ngroups"] == b["ngroups"]
        assert a["keys"].tolist() == b["keys"].tolist()
        assert a["sums"].tolist() == b["sums"].tolist()


def test_group_count_follows_the_threshold():
    """ngroups(T) = groups of the unthresholded plan whose sum exceeds T."""
    D, M, F = datagen.make(2000, 20_000, 80_000, seed=6)
    keys, sums = oracle.plan_groups(D, M, F)
    for t in (np.int64(0), np.percentile(sums, 50).astype(np.int64),
              np.percentile(sums, 99).astype(np.int64), sums.max()):
        got = oracle.run_plan_aggfirst(D, M, F, having=int(t), k=10)
        assert got["ngroups"] == int((sums > t).sum())
