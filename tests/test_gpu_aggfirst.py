"""The aggregate-first plan (PQ_PLAN_AGG_FIRST) through the C ABI against the
oracle, bit-exact: predicates, thresholds and k on the small workload,
repeated M keys (a semi-join counts a key once), row ranges, the x100
workload, overflow, and the dense-key requirement."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import load_tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02862_gb300 as pq  # noqa: E402

I64_MIN = -(1 << 63)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = pq.Context(arena_bytes=8 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.Stream()


@pytest.fixture(scope="module")
def small():
    return datagen.workload("small")


@pytest.fixture(scope="module")
def small_tables(ctx, stream, small):
    with torch.cuda.stream(stream):
        return load_tables(pq, ctx, *small, stream=stream)


def run(ctx, stream, plan):
    with torch.cuda.stream(stream):
        res = pq.pq_run_plan(ctx, plan, stream=stream)
        ctx.sync(stream)
    return res


def same(got, want, what=""):
    assert got.status == want["status"], (what, got.status)
    assert got.ngroups == want["ngroups"], (what, got.ngroups, want["ngroups"])
    d = got.as_dict()
    assert d["keys"] == want["keys"].tolist(), (what, d["keys"][:4], want["keys"][:4])
    assert d["sums"] == want["sums"].tolist(), (what, d["sums"][:4], want["sums"][:4])


PREDS = [dict(seg=1, mc=1200, fc=1200), dict(seg=0, mc=2000, fc=300), dict(seg=4, mc=100, fc=2300),
         dict(seg=9, mc=1200, fc=1200)]


@pytest.mark.parametrize("p", PREDS, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
# group sums of the small workload: 0 keeps every M' group, 2e9 and 4e9 a
# few hundred and a dozen, 8e9 none
@pytest.mark.parametrize("having", [I64_MIN, 0, 2_000_000_000, 4_000_000_000, 8_000_000_000])
@pytest.mark.parametrize("k", [1, 10, 64])
def test_small_workload_matches_oracle(ctx, stream, small, small_tables, p, having, k):
    TD, TM, TF, _ = small_tables
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                        f_date_gt=p["fc"], k=k, having=having))
    want = oracle.run_plan_aggfirst(*small, seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"],
                                    having=having, k=k)
    same(got, want, str((p, having, k)))
    if having == I64_MIN:       # unique M keys: the join-first plan gives the same groups
        jf = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                           f_date_gt=p["fc"], k=k))
        assert jf.as_dict()["keys"] == got.as_dict()["keys"] and jf.ngroups == got.ngroups


def test_repeated_keys_and_row_ranges(ctx, stream):
    D, M, F = datagen.make(3000, 40_000, 160_000, seed=8)
    rng = np.random.default_rng(8)
    M = dict(M)
    M["key"] = M["key"].copy()
    dup = rng.integers(0, 40_000, size=5000)
    M["key"][dup] = M["key"][(dup + 1) % 40_000]
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for having in (I64_MIN, 1_000_000_000):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=2, m_date_lt=1800, f_date_gt=600,
                                            k=64, having=having))
        same(got, oracle.run_plan_aggfirst(D, M, F, seg=2, m_date_lt=1800, f_date_gt=600,
                                           having=having, k=64), f"dup {having}")
    rows = dict(f=(1000, 100_000), m=(50, 30_000))
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, k=20, having=0, rows=rows))
    cut = lambda t, r0, n: {c: v[r0:r0 + n] for c, v in t.items()}
    same(got, oracle.run_plan_aggfirst(D, cut(M, 50, 30_000), cut(F, 1000, 100_000), having=0,
                                       k=20), "rows")
    for t in (TD, TM, TF):
        t.free(stream)


def test_x100_workload(ctx, stream):
    D, M, F = datagen.workload("x100")
    having = 4_000_000_000
    want = oracle.run_plan_aggfirst(D, M, F, having=having, k=10)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, k=10, having=having))
    same(got, want, "x100")
    assert got.hits == int((F["date2"] > 1200).sum())   # every date-passing F row aggregated
    for t in (TD, TM, TF):
        t.free(stream)


@pytest.mark.parametrize("price", [2**56, 2**60], ids=["sum-overflows", "product-overflows"])
def test_overflow_is_reported(ctx, stream, price):
    D = dict(key=np.array([1], np.int32), seg=np.array([1], np.int8))
    M = dict(key=np.array([5], np.int64), dref=np.array([1], np.int32),
             date=np.array([0], np.int32))
    F = dict(mkey=np.full(4, 5, np.int64), price=np.full(4, price, np.int64),
             disc=np.zeros(4, np.int8), date2=np.full(4, 2000, np.int32))
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
        res = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, having=0), stream=stream)
        with pytest.raises(pq.PQError) as e:
            ctx.sync(stream)
    assert e.value.status == pq.PQ_ERR_OVERFLOW and res.status == pq.PQ_ERR_OVERFLOW
    assert oracle.run_plan_aggfirst(D, M, F, having=0)["status"] == 7


def test_sparse_keys_are_refused(ctx, stream):
    D, M, F = datagen.make(200, 2000, 8000, seed=3)
    F = dict(F)
    F["mkey"] = F["mkey"].copy()
    F["mkey"][0] = 1 << 50                       # the F keys now span 2^50 values
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
        with pytest.raises(pq.PQError) as e:
            pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, having=0), stream=stream)
    assert e.value.status == pq.PQ_ERR_INVALID_ARG
