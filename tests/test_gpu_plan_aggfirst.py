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
    # an odd first row: the scan's unaligned (scalar) path
    rows = dict(f=(1001, 99_999), m=(3, 39_000))
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=1, k=64, having=I64_MIN, rows=rows))
    same(got, oracle.run_plan_aggfirst(D, cut(M, 3, 39_000), cut(F, 1001, 99_999), seg=1,
                                       having=I64_MIN, k=64), "odd rows")
    for t in (TD, TM, TF):
        t.free(stream)


@pytest.mark.parametrize("having", [I64_MIN, 0, 10_000_000_000])
def test_zipf_keys(ctx, stream, having):
    """Keys in no order with heavy hitters: one group's rows fall in many
    tiles and many runs."""
    D, M, F = datagen.make(2000, 30_000, 300_000, seed=5, fk="zipf", zipf_s=1.1)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for p in PREDS[:3]:
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                            f_date_gt=p["fc"], k=64, having=having))
        same(got, oracle.run_plan_aggfirst(D, M, F, seg=p["seg"], m_date_lt=p["mc"],
                                           f_date_gt=p["fc"], having=having, k=64),
             f"zipf {p} {having}")
    for t in (TD, TM, TF):
        t.free(stream)


def sorted_chunks(nseg, seed, narrow=False):
    """F as nseg chunks, each in key order, over overlapping keys (nseg - 1
    descents), with a few keys of hundreds of rows, so that runs span whole
    128-row tiles and a key's rows fall in several chunks."""
    rng = np.random.default_rng(seed)
    R = 5000
    D = dict(key=np.arange(1, 101, dtype=np.int32), seg=rng.integers(0, 5, 100).astype(np.int8))
    M = dict(key=np.arange(R, dtype=np.int64) * 2, dref=rng.integers(1, 101, R).astype(np.int32),
             date=rng.integers(0, 2406, R).astype(np.int32))
    keys = []
    for i in range(nseg):
        if narrow and i > 0:        # later chunks over narrow key ranges
            lo = 600 * (nseg - i)     # each lower than the last: a descent
            k = np.concatenate([rng.integers(lo, lo + 500, 800), np.full(400, lo + 250)])
        else:
            k = rng.integers(0, 2 * R, 6000)
            k = np.concatenate([k, np.full(700, rng.integers(0, 2 * R)), np.full(300, 2 * R - 2)])
        keys.append(np.sort(k))
    mk = np.concatenate(keys).astype(np.int64)
    n = len(mk)
    F = dict(mkey=mk, price=rng.integers(90_000, 10_500_000, n).astype(np.int64),
             disc=rng.integers(0, 11, n).astype(np.int8),
             date2=rng.integers(0, 2406, n).astype(np.int32))
    return D, M, F


@pytest.mark.parametrize("nseg,narrow", [(1, False), (2, False), (9, False), (10, False),
                                         (3, True), (9, True)])
def test_key_ordered_segments(ctx, stream, nseg, narrow):
    """The scan of F in key-ordered segments (up to 8 descents) and the
    reduction path beyond; row ranges that cut segments; later segments
    over narrow key ranges (groups outside them are final at commit)."""
    D, M, F = sorted_chunks(nseg, seed=nseg, narrow=narrow)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    cut = lambda t, r0, n: {c: v[r0:r0 + n] for c, v in t.items()}
    n_f = len(F["mkey"])
    for having in (I64_MIN, 0, 1_000_000_000, 20_000_000_000):
        for p in PREDS[:2]:
            got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                                f_date_gt=p["fc"], k=64, having=having))
            same(got, oracle.run_plan_aggfirst(D, M, F, seg=p["seg"], m_date_lt=p["mc"],
                                               f_date_gt=p["fc"], having=having, k=64),
                 f"{nseg} {p} {having}")
        for r0, n in ((1, n_f - 1), (7001, n_f - 9000), (3, 6500), (4999, 1)):
            if n <= 0:
                continue
            got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=1, m_date_lt=2000, f_date_gt=300,
                                                k=64, having=having, rows=dict(f=(r0, n))))
            same(got, oracle.run_plan_aggfirst(D, M, cut(F, r0, n), seg=1, m_date_lt=2000,
                                               f_date_gt=300, having=having, k=64),
                 f"{nseg} rows {r0} {n} {having}")
    for t in (TD, TM, TF):
        t.free(stream)


def gapless_chunks(seed, big_price=False, R=3000):
    """F as key-ordered segments whose distinct keys are consecutive among
    F's keys (gapless: every key once, with 1..7 rows, plus runs of 2047,
    2048, 2049 and 6000 rows, so that runs cut 2048-row units and cover whole
    ones; then a prefix of the keys; then a range that starts below the
    prefix's end), followed by one segment with gaps (every third key of a
    range).  big_price: prices up to
    2^40, beyond the 32-bit revenue bound.  Every segment but the last is
    padded with its last key to a multiple of 16 rows, so that each starts
    16-byte aligned in every column (the staged scan); R keys."""
    rng = np.random.default_rng(seed)
    D = dict(key=np.arange(1, 101, dtype=np.int32), seg=rng.integers(0, 5, 100).astype(np.int8))
    M = dict(key=np.arange(R, dtype=np.int64) * 4, dref=rng.integers(1, 101, R).astype(np.int32),
             date=rng.integers(0, 2406, R).astype(np.int32))
    rep = rng.integers(1, 8, R)
    rep[[10, 500, 1200, R - 1]] = [2047, 2048, 6000, 2049]
    a, b, c = R * 2 // 15, R // 10, R * 17 // 30
    segs = [np.repeat(M["key"], rep),
            np.repeat(M["key"][:a], rng.integers(1, 8, a)),
            np.repeat(M["key"][b:c], rng.integers(1, 5, c - b)),
            np.repeat(M["key"][R // 30:R * 2 // 3:3], rng.integers(1, 4, len(range(R // 30, R * 2 // 3, 3))))]
    for i in range(3):
        segs[i] = np.concatenate([segs[i], np.full(-len(segs[i]) % 16, segs[i][-1])])
    mk = np.concatenate(segs).astype(np.int64)
    n = len(mk)
    hi = 1 << 40 if big_price else 10_500_000
    F = dict(mkey=mk, price=rng.integers(-hi // 50, hi, n).astype(np.int64),
             disc=rng.integers(0, 11, n).astype(np.int8),
             date2=rng.integers(0, 2406, n).astype(np.int32))
    return D, M, F


@pytest.mark.parametrize("big_price,R", [(False, 3000), (True, 3000), (False, 600_000)],
                         ids=["bounded", "tracked", "bounded-large"])
def test_gapless_segments(ctx, stream, big_price, R):
    """Gapless key-ordered segments (staged scan: a unit of rows per warp,
    runs carried between its 128-row steps; R = 600,000 gives units of
    several steps) beside a segment with gaps, whole and cut by row ranges
    at aligned, odd and step-edge rows."""
    D, M, F = gapless_chunks(11, big_price, R)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    cut = lambda t, r0, n: {c: v[r0:r0 + n] for c, v in t.items()}
    n_f = len(F["mkey"])
    for having in (I64_MIN, 0, 3_000_000_000):
        for p in PREDS[:2]:
            got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                                f_date_gt=p["fc"], k=64, having=having))
            same(got, oracle.run_plan_aggfirst(D, M, F, seg=p["seg"], m_date_lt=p["mc"],
                                               f_date_gt=p["fc"], having=having, k=64),
                 f"gapless {p} {having}")
        for r0, n in ((0, 12_000), (16, n_f - 16), (2048, 4096), (1, n_f - 1), (2047, 6002),
                      (n_f - 3000, 3000), (5, 1)):
            got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=1, m_date_lt=2000, f_date_gt=300,
                                                k=64, having=having, rows=dict(f=(r0, n))))
            same(got, oracle.run_plan_aggfirst(D, M, cut(F, r0, n), seg=1, m_date_lt=2000,
                                               f_date_gt=300, having=having, k=64),
                 f"gapless rows {r0} {n} {having}")
    for t in (TD, TM, TF):
        t.free(stream)


def mixed_plans(tables):
    """Aggregate-first and join-first plans over the same tables, with the
    oracle call that gives each one's result."""
    TD, TM, TF = tables
    out = []
    for i, p in enumerate(PREDS * 2):
        q = dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=[1, 10, 64][i % 3])
        if i % 2 == 0:
            h = [I64_MIN, 0, 2_000_000_000, 4_000_000_000][i % 4]
            out.append((pq.make_plan(TD, TM, TF, having=h, **q),
                        lambda D, M, F, q=q, h=h: oracle.run_plan_aggfirst(D, M, F, having=h, **q)))
        else:
            out.append((pq.make_plan(TD, TM, TF, **q),
                        lambda D, M, F, q=q: oracle.run_plan(D, M, F, **q)))
    return out


def test_batch_mixing_plan_shapes(ctx, stream, small, small_tables):
    plans = mixed_plans(small_tables[:3])
    with torch.cuda.stream(stream):
        res = pq.pq_run_batch(ctx, [p for p, _ in plans], stream=stream)
        ctx.sync(stream)
    for i, (_, want) in enumerate(plans):
        same(res[i], want(*small), f"batch {i}")


def test_serving_mixing_plan_shapes(ctx, small, small_tables):
    """Served aggregate-first requests (each in a batch of its own) beside
    batched join-first ones: every result equals the oracle's."""
    plans = mixed_plans(small_tables[:3]) * 3
    tickets = [pq.pq_submit(ctx, p) for p, _ in plans]
    for i, t in enumerate(tickets):
        st, res, lat = pq.pq_poll(ctx, t, timeout_ms=15_000)
        assert st == pq.PQ_OK and lat > 0
        same(res, plans[i][1](*small), f"served {i}")


def test_serving_refuses_aggfirst_over_streamed_tables(ctx, small):
    D, M, F = small
    pin = lambda t, names: [torch.from_numpy(np.ascontiguousarray(t[c])).pin_memory()
                            for c in names]
    TD = pq.pq_load_columns(ctx, pin(D, ("key", "seg")), mode=pq.PQ_STREAMING)
    TM = pq.pq_load_columns(ctx, pin(M, ("key", "dref", "date")), mode=pq.PQ_STREAMING)
    TF = pq.pq_load_columns(ctx, pin(F, ("mkey", "price", "disc", "date2")),
                            mode=pq.PQ_STREAMING)
    with pytest.raises(pq.PQError) as e:
        pq.pq_submit(ctx, pq.make_plan(TD, TM, TF, having=0))
    assert e.value.status == pq.PQ_ERR_INVALID_ARG


@pytest.mark.parametrize("rows", [dict(f=(5, 0)), dict(m=(0, 0)), dict(d=(7, 0)),
                                  dict(f=(599_999, 1)), dict(m=(0, 800), f=(0, 3000)),
                                  dict(m=(0, 1), f=(0, 9))],
                         ids=["no-F", "no-M", "no-D", "one-F", "few", "one-M"])
def test_empty_and_tiny_ranges(ctx, stream, small, small_tables, rows):
    """Empty row ranges and ranges of a few rows, with every predicate
    passing (so that the few rows form groups)."""
    TD, TM, TF, _ = small_tables
    D, M, F = small
    cut = lambda t, key: ({c: v[rows[key][0]:rows[key][0] + rows[key][1]] for c, v in t.items()}
                          if key in rows else t)
    q = dict(d_op="all", m_op="all", f_op="all", k=64)
    for having in (I64_MIN, 0, 500_000_000):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, having=having, rows=rows, **q))
        same(got, oracle.run_plan_aggfirst(cut(D, "d"), cut(M, "m"), cut(F, "f"), having=having,
                                           **q), f"{rows} {having}")


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
