"""The partitioned plan (PQ_PLAN_PARTITIONED) through the C ABI against the
oracle, bit-exact: the F hits are radix-partitioned by group into 2^log2P
buckets and aggregated bucket by bucket.  Dense keys (the M dictionary) and
sparse keys (hash tables), every fan-out from 2 to 1024, pass-all and empty
hit sets, duplicate build keys, row ranges, batches mixing partitioned and
plain plans, graph replay, streamed tables, and a skewed (Zipf) workload at
a tenth of the benchmark's size."""
import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same, load_tables, oracle_plan

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02862_gb300 as pq  # noqa: E402
from test_gpu_plan import remap_keys, random_plans  # noqa: E402

PART = pq.PQ_PLAN_PARTITIONED


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
    return res.as_dict()


PREDS = [dict(seg=1, mc=1200, fc=1200), dict(seg=0, mc=2000, fc=300),
         dict(seg=9, mc=1200, fc=1200),                                  # no hit
         dict(seg=0, mc=0, fc=0, d_op="all", m_op="all", f_op="all")]    # every row hits


def kw(p, k):
    return dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=k,
                d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"), f_op=p.get("f_op", ">"))


def want_of(data, p, k, rows=None):
    return oracle_plan(*data, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=k,
                       d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"),
                       f_op=p.get("f_op", ">"), rows=rows)


@pytest.mark.parametrize("p", PREDS, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
@pytest.mark.parametrize("log2P", [1, 6, 10])
@pytest.mark.parametrize("k", [1, 64])
def test_small_workload_matches_oracle(ctx, stream, small, small_tables, p, log2P, k):
    TD, TM, TF, _ = small_tables
    plan = pq.make_plan(TD, TM, TF, flags=PART | pq.PQ_PLAN_NO_GRAPH, log2P=log2P, **kw(p, k))
    assert_same(run(ctx, stream, plan), want_of(small, p, k), f"{p} {log2P}")


def test_graph_replay_and_plain_plan_agree(ctx, stream, small, small_tables):
    TD, TM, TF, _ = small_tables
    want = want_of(small, PREDS[0], 10)
    for rep in range(3):   # capture, then replays
        assert_same(run(ctx, stream, pq.make_plan(TD, TM, TF, flags=PART, log2P=7, k=10)),
                    want, f"rep {rep}")
    assert run(ctx, stream, pq.make_plan(TD, TM, TF, k=10)) == \
        run(ctx, stream, pq.make_plan(TD, TM, TF, flags=PART, log2P=3, k=10))


@pytest.mark.parametrize("sparse,shift", [(True, 0), (False, -(10**15))],
                         ids=["sparse-hash", "dense-negative"])
@pytest.mark.parametrize("log2P", [2, 9])
def test_renamed_keys(ctx, stream, sparse, shift, log2P):
    """Sparse keys: the M side is a hash table and the buckets are the top
    bits of the Fibonacci product; dense keys of any sign: key-range bits."""
    D, M, F = remap_keys(*datagen.make(5000, 60_000, 250_000, seed=31), seed=32, sparse=sparse,
                         shift=shift)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for p in (PREDS[0], dict(seg=3, mc=2000, fc=300), PREDS[3]):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, flags=PART, log2P=log2P, **kw(p, 10)))
        assert_same(got, want_of((D, M, F), p, 10), f"{p}")
    for t in (TD, TM, TF):
        t.free(stream)


def test_duplicate_build_keys(ctx, stream):
    rng = np.random.default_rng(41)
    D, M, F = datagen.make(3000, 40_000, 160_000, seed=41)
    M = dict(M)
    dup = rng.integers(0, 40_000, size=5000)
    M["key"] = M["key"].copy()
    M["key"][dup] = M["key"][(dup + 1) % 40_000]
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for p in (dict(seg=2, mc=1800, fc=600), PREDS[3]):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, flags=PART, log2P=5, **kw(p, 64)))
        assert_same(got, want_of((D, M, F), p, 64), str(p))


@pytest.mark.parametrize("rows", [dict(m=(16, 30_000), f=(4096, 200_000)),
                                  dict(d=(1, 5000), m=(3, 77_777), f=(5, 123_457)),
                                  dict(f=(599_999, 1)), dict(f=(0, 0))])
def test_row_ranges(ctx, stream, small, small_tables, rows):
    TD, TM, TF, _ = small_tables
    for p in (PREDS[0], PREDS[3]):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, rows=rows, flags=PART, log2P=4,
                                            **kw(p, 10)))
        assert_same(got, want_of(small, p, 10, rows=rows), f"{rows} {p}")


def test_batch_mixing_partitioned_and_plain_plans(ctx, stream, small, small_tables):
    D, M, F = small
    starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
    rng = np.random.default_rng(51)
    plans, specs = random_plans(rng, small_tables[:3], 48, len(M["key"]), len(F["mkey"]), starts)
    for i in range(0, 48, 2):   # every other plan partitioned, fan-outs 2 .. 1024
        plans[i].flags |= PART
        plans[i].log2P = 1 + (i // 2) % 10
    with torch.cuda.stream(stream):
        res = pq.pq_run_batch(ctx, plans, stream=stream)
        ctx.sync(stream)
    for i, sp in enumerate(specs):
        assert_same(res[i].as_dict(), oracle_plan(D, M, F, **sp), f"plan {i}")


def test_skewed_workload_tenth_scale(ctx, stream):
    """Zipf(1.0) foreign keys in no order, pass-all predicates: every F row
    hits and hot groups repeat (the shared aggregation table's path)."""
    D, M, F = datagen.make(400_000, 4_000_000, 20_000_000, seed=4, fk="zipf", zipf_s=1.0)
    q = dict(d_op="all", m_op="all", f_op="all", seg=0, m_date_lt=0, f_date_gt=0, k=10)
    want = oracle.run_plan(D, M, F, **q)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for log2P in (4, 8):
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, flags=PART, log2P=log2P, **q))
        assert_same(got, want, f"log2P {log2P}")
    assert run(ctx, stream, pq.make_plan(TD, TM, TF, **q))["keys"] == list(map(int, want["keys"]))
    for t in (TD, TM, TF):
        t.free(stream)


@pytest.mark.parametrize("source", ["pinned", "packed"])
def test_streamed_tables(stream, small, source):
    """Streamed F chunks: each chunk's hits are partitioned and aggregated;
    a single plan and a batch sharing one ingest pass."""
    D, M, F = small
    c = pq.Context(arena_bytes=2 << 30, chunk_bytes=1 << 20, ring_slots=3)

    def col(a):
        a = np.ascontiguousarray(a)
        return pq.pq_pack_column(a) if source == "packed" else torch.from_numpy(a).pin_memory()

    with torch.cuda.stream(stream):
        TD = pq.pq_load_columns(c, [col(D[x]) for x in ("key", "seg")], mode=pq.PQ_STREAMING)
        TM = pq.pq_load_columns(c, [col(M[x]) for x in ("key", "dref", "date")],
                                mode=pq.PQ_STREAMING)
        TF = pq.pq_load_columns(c, [col(F[x]) for x in ("mkey", "price", "disc", "date2")],
                                mode=pq.PQ_STREAMING)
        for p in (PREDS[0], PREDS[3]):
            got = pq.pq_run_plan(c, pq.make_plan(TD, TM, TF, flags=PART, log2P=6, **kw(p, 32)),
                                 stream=stream)
            c.sync(stream)
            assert_same(got.as_dict(), want_of(small, p, 32), f"{source} {p}")
        starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
        rng = np.random.default_rng(61)
        plans, specs = random_plans(rng, (TD, TM, TF), 12, len(M["key"]), len(F["mkey"]), starts)
        for i in range(0, 12, 3):
            plans[i].flags |= PART
            plans[i].log2P = 5
        res = pq.pq_run_batch(c, plans, stream=stream)
        c.sync(stream)
    for i, sp in enumerate(specs):
        assert_same(res[i].as_dict(), oracle_plan(D, M, F, **sp), f"{source} plan {i}")
    c.close()


def test_partitioned_argument_errors(ctx, stream, small_tables):
    TD, TM, TF, _ = small_tables
    for bad in (dict(flags=PART, log2P=11), dict(flags=PART, having=0)):
        with pytest.raises(pq.PQError) as e:
            with torch.cuda.stream(stream):
                pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, **bad), stream=stream)
        assert e.value.status == pq.PQ_ERR_INVALID_ARG
