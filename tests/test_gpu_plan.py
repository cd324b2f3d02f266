"""Parity of the whole plan (CUDA through the C ABI) with the CPU oracle,
bit-exact: the hand-worked example, the small workload under many
predicates, the full x100 workload in the benchmark's launch configuration,
duplicate build keys, row ranges, unaligned views, CUDA-graph replay,
batches, streaming (pinned, pageable, file sources), serving and errors."""
import os

import numpy as np
import pytest

import datagen
import oracle
from gpu_util import assert_same, load_tables, oracle_plan, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02862_gb300 as pq  # noqa: E402
import pins  # noqa: E402


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


def test_hand_worked_example(ctx, stream):
    g = pins.read_golden("tiny_plan.txt")
    D = dict(key=np.array(g["D.key"][0], np.int32), seg=np.array(g["D.seg"][0], np.int8))
    M = dict(key=np.array(g["M.key"][0], np.int64), dref=np.array(g["M.dref"][0], np.int32),
             date=np.array(g["M.date"][0], np.int32))
    F = dict(mkey=np.array(g["F.mkey"][0], np.int64), price=np.array(g["F.price"][0], np.int64),
             disc=np.array(g["F.disc"][0], np.int8), date2=np.array(g["F.date2"][0], np.int32))
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    got = run(ctx, stream, pq.make_plan(TD, TM, TF))
    assert got["ngroups"] == g["expect.ngroups"][0][0]
    assert got["keys"] == g["expect.keys"][0] and got["sums"] == g["expect.sums"][0]


PREDS = [dict(seg=1, mc=1200, fc=1200), dict(seg=0, mc=2000, fc=300), dict(seg=4, mc=100, fc=2300),
         dict(seg=1, mc=1200, fc=1200, d_op="!=", m_op=">=", f_op="<="),
         dict(seg=9, mc=1200, fc=1200),                            # no D row passes
         dict(seg=0, mc=0, fc=0, d_op="all", m_op="all", f_op="all")]


@pytest.mark.parametrize("p", PREDS, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
@pytest.mark.parametrize("k", [1, 10, 64])
def test_small_workload_matches_oracle(ctx, stream, small, small_tables, p, k):
    TD, TM, TF, _ = small_tables
    plan = pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=k,
                        d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"),
                        f_op=p.get("f_op", ">"), flags=pq.PQ_PLAN_NO_GRAPH)
    want = oracle_plan(*small, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=k,
                       d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"), f_op=p.get("f_op", ">"))
    assert_same(run(ctx, stream, plan), want, str(p))


def test_pass_all_closed_form(ctx, stream, small, small_tables):
    """Every foreign key exists: groups = distinct F.mkey, and the top group
    sum is the largest per-key sum of price * (100 - disc)."""
    D, M, F = small
    TD, TM, TF, _ = small_tables
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, d_op="all", m_op="all", f_op="all", k=64))
    assert got["ngroups"] == len(np.unique(F["mkey"]))
    rev = F["price"].astype(np.int64) * (100 - F["disc"].astype(np.int64))
    keys, inv = np.unique(F["mkey"], return_inverse=True)
    sums = np.bincount(inv, weights=rev.astype(np.float64))
    assert got["sums"][0] == int(np.max(sums))


def test_x100_workload_full_size(ctx, stream):
    """The benchmark's workload (D 1.5M, M 15M, F 60M rows) and launch shape."""
    D, M, F = datagen.workload("x100")
    want = oracle.run_plan(D, M, F, k=10)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    plan = pq.make_plan(TD, TM, TF, k=10)
    for rep in range(3):   # first run captures a graph, later runs replay it
        assert_same(run(ctx, stream, plan), want, f"rep {rep}")
    assert ctx.stats()["graph_replays"] >= 2
    for t in (TD, TM, TF):
        t.free(stream)


def test_duplicate_build_keys(ctx, stream):
    rng = np.random.default_rng(8)
    D, M, F = datagen.make(3000, 40_000, 160_000, seed=8)
    M = dict(M)
    dup = rng.integers(0, 40_000, size=5000)
    M["key"] = M["key"].copy()
    M["key"][dup] = M["key"][(dup + 1) % 40_000]       # some keys now appear twice
    want = oracle_plan(D, M, F, seg=2, mc=1800, fc=600, k=64)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=2, m_date_lt=1800, f_date_gt=600, k=64))
    assert_same(got, want)


@pytest.mark.parametrize("n_m", [131_072, 131_073, 262_144, 262_145, 262_176])
def test_topk_tiles_at_the_bound(ctx, stream, n_m):
    """Distinct member counts around 128 and 256 top-k tiles of 32 bitmap
    words: the tiling must stay within 256 tiles (the tile lists' and the
    last tile's scratch size)."""
    D, M, F = datagen.make(2000, n_m, 300_000, seed=11)
    ops = dict(d_op="all", m_op="all", f_op="all")
    want = oracle_plan(D, M, F, seg=0, mc=0, fc=0, k=10, **ops)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=0, m_date_lt=0, f_date_gt=0, k=10,
                                        flags=pq.PQ_PLAN_NO_GRAPH, **ops))
    assert_same(got, want, str(n_m))
    for t in (TD, TM, TF):
        t.free(stream)


@pytest.mark.parametrize("k", [1, 10, 32, 33, 64])
def test_topk_lane_lists_overflow(ctx, stream, k):
    """Every M key a group, one F row each, the largest sums on slots 32
    apart: in the top-k scan those records land on one lane of each warp,
    more of them than a lane keeps, so the tiles fall back to the exact
    per-warp lists (k <= 32); k > 32 takes them always."""
    n = 40_000
    D = dict(key=np.arange(1, 11, dtype=np.int32), seg=np.ones(10, np.int8))
    M = dict(key=np.arange(n, dtype=np.int64), dref=np.ones(n, np.int32),
             date=np.zeros(n, np.int32))
    key = np.arange(n, dtype=np.int64)
    F = dict(mkey=key, price=1000 + key + np.where(key % 32 == 0, 10**7, 0),
             disc=np.zeros(n, np.int8), date2=np.full(n, 2000, np.int32))
    ops = dict(d_op="all", m_op="all", f_op="all")
    want = oracle_plan(D, M, F, seg=0, mc=0, fc=0, k=k, **ops)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, seg=0, m_date_lt=0, f_date_gt=0, k=k, **ops))
    assert_same(got, want, str(k))
    for t in (TD, TM, TF):
        t.free(stream)


def test_mapped_tables_match_oracle(ctx, stream, small):
    """PQ_MAPPED: the plan kernels read pinned host columns in place."""
    D, M, F = small
    pin = lambda t: {k: torch.from_numpy(v).pin_memory() for k, v in t.items()}
    d, m, f = pin(D), pin(M), pin(F)
    with torch.cuda.stream(stream):
        TD = pq.pq_load_columns(ctx, [d["key"], d["seg"]], mode=pq.PQ_MAPPED, stream=stream)
        TM = pq.pq_load_columns(ctx, [m[c] for c in ("key", "dref", "date")],
                                mode=pq.PQ_MAPPED, stream=stream)
        TF = pq.pq_load_columns(ctx, [f[c] for c in ("mkey", "price", "disc", "date2")],
                                mode=pq.PQ_MAPPED, stream=stream)
    assert TF.column_ptr(0) == f["mkey"].data_ptr()   # in place, not copied
    for p in PREDS[:3] + PREDS[-1:]:
        kw = dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=10,
                  d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"), f_op=p.get("f_op", ">"))
        want = oracle_plan(*small, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=10,
                           d_op=kw["d_op"], m_op=kw["m_op"], f_op=kw["f_op"])
        for flags in (pq.PQ_PLAN_NO_GRAPH, 0, 0):   # separate launches, capture, replay
            assert_same(run(ctx, stream, pq.make_plan(TD, TM, TF, flags=flags, **kw)), want,
                        str(p))
    for t in (TD, TM, TF):
        t.free(stream)


def test_mapped_refuses_pageable_and_files(ctx, small, tmp_path):
    D, _, _ = small
    with pytest.raises(pq.PQError, match="INVALID_ARG"):
        pq.pq_load_columns(ctx, [D["key"], D["seg"]], mode=pq.PQ_MAPPED)
    path = tmp_path / "key.bin"
    D["key"].tofile(path)
    with pytest.raises(pq.PQError, match="INVALID_ARG"):
        pq.pq_load_columns(ctx, [(str(path), pq.PQ_INT32, 0, len(D["key"])),
                                 torch.from_numpy(D["seg"]).pin_memory()], mode=pq.PQ_MAPPED)


def test_joined_row_count(ctx, stream, small, small_tables):
    """The result's hit count: every F row joins when all predicates pass."""
    TD, TM, TF, _ = small_tables
    with torch.cuda.stream(stream):
        res = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, d_op="all", m_op="all", f_op="all",
                                               flags=pq.PQ_PLAN_NO_GRAPH), stream=stream)
        ctx.sync(stream)
    assert res.hits == len(small[2]["mkey"])


def remap_keys(D, M, F, seed, sparse=True, shift=0):
    """The same plan with the keys renamed: M keys to distinct random int64
    values of both signs (sparse: no key-range bitmap, hash tables) or to
    key + shift (dense, possibly negative), D keys to distinct random int32
    values; references (M.dref, F.mkey) follow."""
    rng = np.random.default_rng(seed)
    M, D, F = dict(M), dict(D), dict(F)
    old_m = M["key"]
    if sparse:
        new_m = rng.choice(np.iinfo(np.int64).max, size=len(old_m), replace=False)
        new_m = (new_m - (np.iinfo(np.int64).max // 2)).astype(np.int64)
    else:
        new_m = (old_m + shift).astype(np.int64)
    order = np.argsort(old_m)
    F["mkey"] = new_m[order[np.searchsorted(old_m[order], F["mkey"])]]
    M["key"] = new_m
    old_d = D["key"]
    new_d = rng.choice(2**31 - 1, size=len(old_d), replace=False).astype(np.int32) - 2**30
    od = np.argsort(old_d)
    M["dref"] = new_d[od[np.searchsorted(old_d[od], M["dref"])]].astype(np.int32)
    D["key"] = new_d.astype(np.int32)
    return D, M, F


@pytest.mark.parametrize("sparse,shift", [(True, 0), (False, -(10**15)), (False, -7)],
                         ids=["sparse-hash", "dense-negative", "dense-around-zero"])
def test_renamed_keys(ctx, stream, sparse, shift):
    """Sparse keys take the hash-table paths (D-set and M table); dense keys
    of any sign take the bitmap and the rank dictionary."""
    D, M, F = datagen.make(5000, 60_000, 250_000, seed=21)
    D, M, F = remap_keys(D, M, F, seed=22, sparse=sparse, shift=shift)
    for p in ({}, dict(seg=3, mc=2000, fc=300)):
        want = oracle_plan(D, M, F, k=10, **p)
        with torch.cuda.stream(stream):
            TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
        kw = dict(seg=p.get("seg", 1), m_date_lt=p.get("mc", 1200), f_date_gt=p.get("fc", 1200))
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, k=10, **kw))
        assert_same(got, want, str(p))
        for t in (TD, TM, TF):
            t.free(stream)


def test_batch_mixing_hash_and_dense_plans(ctx, stream, small, small_tables):
    D, M, F = remap_keys(*datagen.make(4000, 50_000, 200_000, seed=23), seed=24, sparse=True)
    with torch.cuda.stream(stream):
        SD, SM, SF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    TD, TM, TF, _ = small_tables
    plans = [pq.make_plan(SD, SM, SF, k=10), pq.make_plan(TD, TM, TF, k=10),
             pq.make_plan(SD, SM, SF, seg=2, m_date_lt=2000, f_date_gt=100, k=10)]
    wants = [oracle_plan(D, M, F, k=10), oracle_plan(*small, k=10),
             oracle_plan(D, M, F, seg=2, mc=2000, fc=100, k=10)]
    with torch.cuda.stream(stream):
        res = pq.pq_run_batch(ctx, plans, stream=stream)
        ctx.sync(stream)
    for r, w in zip(res, wants):
        assert_same(r.as_dict(), w)
    for t in (SD, SM, SF):
        t.free(stream)


@pytest.mark.parametrize("rows", [dict(m=(16, 30_000), f=(4096, 200_000)),
                                  dict(d=(1, 5000), m=(3, 77_777), f=(5, 123_457)),
                                  dict(f=(599_999, 1)), dict(m=(0, 0))])
def test_row_ranges_and_unaligned_views(ctx, stream, small, small_tables, rows):
    TD, TM, TF, _ = small_tables
    got = run(ctx, stream, pq.make_plan(TD, TM, TF, rows=rows, k=10))
    assert_same(got, oracle_plan(*small, rows=rows, k=10), str(rows))


def random_plans(rng, tables, n, n_m, n_f, starts):
    TD, TM, TF = tables
    plans, specs = [], []
    for _ in range(n):
        a = int(rng.integers(0, n_m - 1)) // 16 * 16
        b = min(n_m, a + int(rng.integers(1, n_m // 4)))
        f0 = int(starts[a]) // 16 * 16
        f1 = max(f0, int(starts[b]) // 16 * 16)
        seg, c, k = int(rng.integers(0, 5)), int(rng.integers(0, 2406)), int(rng.integers(1, 65))
        rows = dict(m=(a, b - a), f=(f0, f1 - f0))
        plans.append(pq.make_plan(TD, TM, TF, seg=seg, m_date_lt=c, f_date_gt=c, k=k, rows=rows))
        specs.append(dict(seg=seg, mc=c, fc=c, k=k, rows=rows))
    return plans, specs


def test_batch_of_uneven_plans(ctx, stream, small, small_tables):
    D, M, F = small
    starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
    rng = np.random.default_rng(21)
    plans, specs = random_plans(rng, small_tables[:3], 64, len(M["key"]), len(F["mkey"]), starts)
    with torch.cuda.stream(stream):
        res = pq.pq_run_batch(ctx, plans, stream=stream)
        ctx.sync(stream)
    for i, sp in enumerate(specs):
        assert_same(res[i].as_dict(), oracle_plan(D, M, F, **sp), f"plan {i}")
    # the same plans one at a time give the same results
    for i in (0, 17, 63):
        assert run(ctx, stream, plans[i]) == res[i].as_dict()


def test_batch_with_cached_dimension_sets(ctx, stream, small, small_tables):
    D, M, F = small
    TD, TM, TF, _ = small_tables
    plans = [pq.make_plan(TD, TM, TF, seg=s % 5, m_date_lt=300 + 97 * s, f_date_gt=2000 - 50 * s,
                          k=10, flags=pq.PQ_PLAN_CACHE_DSET) for s in range(20)]
    for rep in range(2):     # second pass hits the resident D-sets
        with torch.cuda.stream(stream):
            res = pq.pq_run_batch(ctx, plans, stream=stream)
            ctx.sync(stream)
        for s in range(20):
            assert_same(res[s].as_dict(), oracle_plan(D, M, F, seg=s % 5, mc=300 + 97 * s,
                                                      fc=2000 - 50 * s), f"rep {rep} plan {s}")


@pytest.fixture(scope="module")
def stream_ctx():
    c = pq.Context(arena_bytes=2 << 30, chunk_bytes=1 << 20, ring_slots=3, copy_streams=2,
                   ingest_threads=3)
    yield c
    c.close()


@pytest.mark.parametrize("source", ["pinned", "pageable", "file", "packed", "mixed"])
def test_streaming_plan_matches_oracle(stream_ctx, stream, small, tmp_path, source):
    D, M, F = small
    ctx = stream_ctx

    def cols(tab, names):
        out = []
        for i, nm in enumerate(names):
            a = np.ascontiguousarray(tab[nm])
            if source == "packed" or (source == "mixed" and i % 2 == 0):
                out.append(pq.pq_pack_column(a))      # decoded on the device per chunk
            elif source == "mixed" and i % 3 == 1:
                out.append(a)
            elif source in ("pinned", "mixed"):
                out.append(torch.from_numpy(a).pin_memory())
            elif source == "pageable":
                out.append(a)
            else:
                p = tmp_path / f"{id(tab)}_{nm}.bin"
                a.tofile(p)
                code = {1: pq.PQ_INT8, 4: pq.PQ_INT32, 8: pq.PQ_INT64}[a.itemsize]
                out.append((str(p), code, 0, len(a)))
        return out

    with torch.cuda.stream(stream):
        TD = pq.pq_load_columns(ctx, cols(D, ["key", "seg"]), mode=pq.PQ_STREAMING)
        TM = pq.pq_load_columns(ctx, cols(M, ["key", "dref", "date"]), mode=pq.PQ_STREAMING)
        TF = pq.pq_load_columns(ctx, cols(F, ["mkey", "price", "disc", "date2"]),
                                mode=pq.PQ_STREAMING)
        for p in (dict(seg=1, mc=1200, fc=1200), dict(seg=3, mc=2200, fc=100)):
            got = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, seg=p["seg"], m_date_lt=p["mc"],
                                                   f_date_gt=p["fc"], k=32), stream=stream)
            ctx.sync(stream)
            assert_same(got.as_dict(), oracle_plan(D, M, F, k=32, **p), source)
        assert ctx.stats()["chunks_ingested"] > 20


@pytest.mark.parametrize("hit_buffer", [-1, 1, 2, 16])
def test_streaming_hit_buffer(stream, small, hit_buffer):
    """Dynamic buffering of a streamed F table's hits: probe every chunk
    (-1), or keep the hits of up to 1, 2, 16 chunks of rows on the device
    and probe when the buffer could not take another chunk or after the
    last; with every row a hit the small buffers force probes mid-stream."""
    D, M, F = small
    c = pq.Context(arena_bytes=2 << 30, chunk_bytes=1 << 20, ring_slots=3,
                   hit_buffer=hit_buffer)
    pin = lambda t, names: [torch.from_numpy(np.ascontiguousarray(t[x])).pin_memory()
                            for x in names]
    with torch.cuda.stream(stream):
        TD = pq.pq_load_columns(c, pin(D, ("key", "seg")), mode=pq.PQ_STREAMING)
        TM = pq.pq_load_columns(c, pin(M, ("key", "dref", "date")), mode=pq.PQ_STREAMING)
        TF = pq.pq_load_columns(c, pin(F, ("mkey", "price", "disc", "date2")),
                                mode=pq.PQ_STREAMING)
        for p in (dict(seg=1, mc=1200, fc=1200, k=10),
                  dict(seg=0, mc=0, fc=0, k=64, d_op="all", m_op="all", f_op="all")):
            kw = dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=p["k"],
                      d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"),
                      f_op=p.get("f_op", ">"))
            got = pq.pq_run_plan(c, pq.make_plan(TD, TM, TF, **kw), stream=stream)
            c.sync(stream)
            want = oracle_plan(D, M, F, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=p["k"],
                               d_op=kw["d_op"], m_op=kw["m_op"], f_op=kw["f_op"])
            assert_same(got.as_dict(), want, f"hit_buffer {hit_buffer} {p}")
            assert got.hits == (len(F["mkey"]) if "f_op" in p else got.hits)
    c.close()


class _DevView:
    """A device array seen through __cuda_array_interface__ (the test only reads it)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def test_packed_columns_resident_and_row_ranges(stream_ctx, stream, small):
    """Packed sources: a resident table decodes them once (bit-exact copies of
    the plain columns); a streamed packed F table with row ranges that do not
    start on a pack block matches the oracle."""
    D, M, F = small
    ctx = stream_ctx
    names = ("mkey", "price", "disc", "date2")
    with torch.cuda.stream(stream):
        TF = pq.pq_load_columns(ctx, [pq.pq_pack_column(F[c]) for c in names], stream=stream)
        ctx.sync(stream)
        for j, c in enumerate(names):
            a = F[c]
            v = _DevView(TF.column_ptr(j), len(a), np.dtype(a.dtype).str)
            assert np.array_equal(torch.as_tensor(v, device="cuda").cpu().numpy(), a), c
        TF.free(stream)
        d, m = to_dev(D), to_dev(M)
        TD = pq.pq_load_columns(ctx, [d["key"], d["seg"]])
        TM = pq.pq_load_columns(ctx, [m["key"], m["dref"], m["date"]])
        PF = pq.pq_load_columns(ctx, [pq.pq_pack_column(F[c]) for c in names],
                                mode=pq.PQ_STREAMING)
        for rows in (dict(f=(1000, 500_000)), dict(f=(4096 * 3 - 7, 9000))):
            got = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, PF, rows=rows), stream=stream)
            ctx.sync(stream)
            assert_same(got.as_dict(), oracle_plan(D, M, F, rows=rows), str(rows))
        assert ctx.stats()["chunks_ingested"] > 0


@pytest.mark.parametrize("source", ["pinned", "packed", "pageable"])
def test_streamed_batch_shares_one_ingest(stream_ctx, stream, small, source):
    """A batch of plans over the same streamed tables (random M and F slices,
    predicates and k): every result matches the oracle, and the batch copies
    each chunk of the tables once -- no more chunks than one plan over the
    whole tables."""
    D, M, F = small
    ctx = stream_ctx

    def col(a):
        a = np.ascontiguousarray(a)
        return (pq.pq_pack_column(a) if source == "packed" else
                torch.from_numpy(a).pin_memory() if source == "pinned" else a)

    with torch.cuda.stream(stream):
        TD = pq.pq_load_columns(ctx, [col(D[c]) for c in ("key", "seg")], mode=pq.PQ_STREAMING)
        TM = pq.pq_load_columns(ctx, [col(M[c]) for c in ("key", "dref", "date")],
                                mode=pq.PQ_STREAMING)
        TF = pq.pq_load_columns(ctx, [col(F[c]) for c in ("mkey", "price", "disc", "date2")],
                                mode=pq.PQ_STREAMING)
        c0 = ctx.stats()["chunks_ingested"]
        pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF), stream=stream)
        ctx.sync(stream)
        whole = ctx.stats()["chunks_ingested"] - c0
        starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
        rng = np.random.default_rng(55)
        plans, specs = random_plans(rng, (TD, TM, TF), 24, len(M["key"]), len(F["mkey"]),
                                    starts)
        c0 = ctx.stats()["chunks_ingested"]
        res = pq.pq_run_batch(ctx, plans, stream=stream)
        ctx.sync(stream)
        assert ctx.stats()["chunks_ingested"] - c0 <= whole
    for i, sp in enumerate(specs):
        assert_same(res[i].as_dict(), oracle_plan(D, M, F, **sp), f"{source} plan {i}")


def test_streamed_batch_with_resident_dimensions(stream_ctx, stream, small):
    """A batch whose D and M are resident and whose F is streamed (packed):
    the resident tables are scanned in place, F once for all plans."""
    D, M, F = small
    ctx = stream_ctx
    with torch.cuda.stream(stream):
        d, m = to_dev(D), to_dev(M)
        TD = pq.pq_load_columns(ctx, [d["key"], d["seg"]])
        TM = pq.pq_load_columns(ctx, [m["key"], m["dref"], m["date"]])
        TF = pq.pq_load_columns(ctx, [pq.pq_pack_column(F[c])
                                      for c in ("mkey", "price", "disc", "date2")],
                                mode=pq.PQ_STREAMING)
        starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
        rng = np.random.default_rng(91)
        plans, specs = random_plans(rng, (TD, TM, TF), 16, len(M["key"]), len(F["mkey"]),
                                    starts)
        res = pq.pq_run_batch(ctx, plans, stream=stream)
        ctx.sync(stream)
    for i, sp in enumerate(specs):
        assert_same(res[i].as_dict(), oracle_plan(D, M, F, **sp), f"plan {i}")


def test_serving_over_streamed_tables(stream_ctx, stream, small):
    """Requests over host-resident (streamed) tables: served results equal
    the oracle's."""
    D, M, F = small
    ctx = stream_ctx
    pin = lambda t, names: [torch.from_numpy(np.ascontiguousarray(t[c])).pin_memory()
                            for c in names]
    TD = pq.pq_load_columns(ctx, pin(D, ("key", "seg")), mode=pq.PQ_STREAMING)
    TM = pq.pq_load_columns(ctx, pin(M, ("key", "dref", "date")), mode=pq.PQ_STREAMING)
    TF = pq.pq_load_columns(ctx, pin(F, ("mkey", "price", "disc", "date2")),
                            mode=pq.PQ_STREAMING)
    starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
    rng = np.random.default_rng(77)
    plans, specs = random_plans(rng, (TD, TM, TF), 40, len(M["key"]), len(F["mkey"]), starts)
    tickets = [pq.pq_submit(ctx, p) for p in plans]
    for i, t in enumerate(tickets):
        st, res, lat = pq.pq_poll(ctx, t, timeout_ms=15_000)
        assert st == pq.PQ_OK
        assert_same(res.as_dict(), oracle_plan(D, M, F, **specs[i]), f"served {i}")


def test_streaming_fact_table_with_resident_dimensions(stream_ctx, stream, small):
    D, M, F = small
    ctx = stream_ctx
    with torch.cuda.stream(stream):
        d, m = to_dev(D), to_dev(M)
        TD = pq.pq_load_columns(ctx, [d["key"], d["seg"]])
        TM = pq.pq_load_columns(ctx, [m["key"], m["dref"], m["date"]])
        TF = pq.pq_load_columns(ctx, [torch.from_numpy(F[c]).pin_memory()
                                      for c in ("mkey", "price", "disc", "date2")],
                                mode=pq.PQ_STREAMING)
        got = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, rows=dict(f=(1000, 500_000))),
                             stream=stream)
        ctx.sync(stream)
    assert_same(got.as_dict(), oracle_plan(D, M, F, rows=dict(f=(1000, 500_000))))


def test_serving_results_same_alone_and_in_the_mix(ctx, stream, small, small_tables):
    D, M, F = small
    starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
    rng = np.random.default_rng(33)
    plans, specs = random_plans(rng, small_tables[:3], 150, len(M["key"]), len(F["mkey"]),
                                starts)
    tickets = [pq.pq_submit(ctx, p) for p in plans]
    for i, t in enumerate(tickets):
        st, res, lat = pq.pq_poll(ctx, t, timeout_ms=15_000)
        assert st == pq.PQ_OK and lat > 0
        want = oracle_plan(D, M, F, **specs[i])
        assert_same(res.as_dict(), want, f"served {i}")
        if i % 37 == 0:
            assert run(ctx, stream, plans[i]) == res.as_dict()   # alone


def test_serving_tiny_requests_one_by_one(ctx, small, small_tables):
    """Requests submitted and polled one at a time: each batch is a single
    tiny plan that can finish before the serving thread has finished queuing
    it, which must still complete its ticket."""
    D, M, F = small
    TD, TM, TF, _ = small_tables
    for i in range(300):
        rows = dict(m=(16 * i, 16), f=(64 * i, 64))
        t = pq.pq_submit(ctx, pq.make_plan(TD, TM, TF, d_op="all", m_op="all", f_op="all",
                                           rows=rows, k=4))
        st, res, lat = pq.pq_poll(ctx, t, timeout_ms=15_000)
        assert st == pq.PQ_OK, (i, st)
        if i % 50 == 0:
            assert_same(res.as_dict(), oracle_plan(D, M, F, d_op="all", m_op="all", f_op="all",
                                                   rows=rows, k=4), f"request {i}")


def test_close_with_requests_in_flight(stream, small):
    """Closing a context while requests are queued and batches run: the
    batches on the GPU finish, the queued requests are dropped, and close
    returns (bounded) without error."""
    import time
    D, M, F = small
    c = pq.Context(arena_bytes=1 << 30)
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, c, D, M, F, stream=stream)
        torch.cuda.current_stream().synchronize()
    for i in range(400):
        pq.pq_submit(c, pq.make_plan(TD, TM, TF, seg=i % 5, k=10))
    t0 = time.monotonic()
    c.close()
    assert time.monotonic() - t0 < 35


def test_autotune_keeps_results(ctx, stream, small, small_tables):
    """The tuner measures its 14 settings (blocks per SM, load factor,
    partition fan-out), reports a choice inside the grid, and plans run with
    the tuned defaults, partitioned or not, give the oracle's result."""
    TD, TM, TF, _ = small_tables
    plan = pq.make_plan(TD, TM, TF)
    t = pq.pq_autotune(ctx, plan)
    assert t["tried"] == 14 and t["best_ms"] > 0 and t["block_threads"] == 256
    assert t["blocks_per_sm"] in (1, 2, 3, 4, 6, 8)
    assert t["load_factor"] in (0.25, pytest.approx(0.4), 0.5, pytest.approx(0.7))
    assert t["partitioned"] in (0, 1) and t["log2P"] in range(1, 11)
    want = oracle_plan(*small)
    assert_same(run(ctx, stream, plan), want)
    assert_same(run(ctx, stream, pq.make_plan(TD, TM, TF, flags=pq.PQ_PLAN_PARTITIONED)), want)


@pytest.mark.parametrize("flags,log2P", [(0, 0), (pq.PQ_PLAN_PARTITIONED, 5)],
                         ids=["plain", "partitioned"])
def test_exact_commit_path(ctx, stream, small, flags, log2P):
    """One F row with a price of 2^55 that the date filter drops: the bound
    on the revenues (hits x max |price| x 228) no longer excludes an int64
    overflow, so the probe commits with checked atomics; no group overflows
    and the result equals the oracle's."""
    D, M, F = small
    F = dict(F)
    F["price"] = F["price"].copy()
    F["date2"] = F["date2"].copy()
    F["price"][0], F["date2"][0] = 2**55, 0
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
    for p in (dict(seg=1, mc=1200, fc=1200), dict(seg=0, mc=0, fc=0, d_op="all", m_op="all")):
        kw = dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=10,
                  d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"))
        got = run(ctx, stream, pq.make_plan(TD, TM, TF, flags=flags, log2P=log2P, **kw))
        assert_same(got, oracle_plan(D, M, F, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=10,
                                     d_op=kw["d_op"], m_op=kw["m_op"]), str(p))
    for t in (TD, TM, TF):
        t.free(stream)


@pytest.mark.parametrize("price", [2**56, 2**60], ids=["sum-overflows", "product-overflows"])
def test_overflow_is_reported(ctx, stream, price):
    D = dict(key=np.array([1], np.int32), seg=np.array([1], np.int8))
    M = dict(key=np.array([5], np.int64), dref=np.array([1], np.int32),
             date=np.array([0], np.int32))
    n = 4
    F = dict(mkey=np.full(n, 5, np.int64), price=np.full(n, price, np.int64),
             disc=np.zeros(n, np.int8), date2=np.full(n, 2000, np.int32))
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, ctx, D, M, F, stream=stream)
        res = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, flags=pq.PQ_PLAN_NO_GRAPH),
                             stream=stream)
        with pytest.raises(pq.PQError) as e:
            ctx.sync(stream)
    assert e.value.status == pq.PQ_ERR_OVERFLOW and res.status == pq.PQ_ERR_OVERFLOW
    assert oracle.run_plan(D, M, F)["status"] == 7


def test_budget_and_argument_errors(stream, small):
    # The small plan's workspace (hit list 2.4 MB, dictionary 1.9 MB, D-set)
    # does not fit in 2 MB.
    c = pq.Context(arena_bytes=2 << 20)
    D, M, F = small
    with torch.cuda.stream(stream):
        TD, TM, TF, keep = load_tables(pq, c, D, M, F, stream=stream)
        with pytest.raises(pq.PQError) as e:
            pq.pq_run_plan(c, pq.make_plan(TD, TM, TF), stream=stream)
        assert e.value.status == pq.PQ_ERR_BUDGET
        with pytest.raises(pq.PQError) as e:
            pq.pq_run_plan(c, pq.make_plan(TD, TM, TF, k=0), stream=stream)
        assert e.value.status == pq.PQ_ERR_INVALID_ARG
        with pytest.raises(pq.PQError) as e:
            pq.pq_run_plan(c, pq.make_plan(TD, TM, TF, rows=dict(f=(0, 10**9))), stream=stream)
        assert e.value.status == pq.PQ_ERR_INVALID_ARG
    c.close()
