"""Out-of-core plans: when a join-first plan does not fit its arena (the
device budget), the build side is radix-partitioned by key range and the
plan runs in passes whose dictionaries fit, with F scanned once per pass.
Against the oracle, bit-exact, for arenas that force 1 to many passes,
with repeated M keys, several predicates and k, and for tables in pinned
host memory read in place (mapped)."""
import numpy as np
import pytest

import datagen
from gpu_util import assert_same, oracle_plan

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02862_gb300 as pq  # noqa: E402

MB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.Stream()


def tables(ctx, D, M, F, mode):
    if mode == "mapped":
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        cols = lambda t, names: [pin(t[c]) for c in names]
        kw = dict(mode=pq.PQ_MAPPED)
    else:
        cols = lambda t, names: [torch.from_numpy(np.ascontiguousarray(t[c])).cuda()
                                 for c in names]
        kw = {}
    keep = [cols(D, ("key", "seg")), cols(M, ("key", "dref", "date")),
            cols(F, ("mkey", "price", "disc", "date2"))]
    return [pq.pq_load_columns(ctx, c, **kw) for c in keep], keep


def sweep(stream, D, M, F, mode, preds, arenas):
    """Run the plans under each arena; returns the pass counts seen."""
    seen = []
    for ab in arenas:
        ctx = pq.Context(arena_bytes=ab)
        (TD, TM, TF), keep = tables(ctx, D, M, F, mode)
        for p in preds:
            kw = dict(seg=p["seg"], m_date_lt=p["mc"], f_date_gt=p["fc"], k=p["k"],
                      d_op=p.get("d_op", "=="), m_op=p.get("m_op", "<"))
            before = ctx.stats()["out_of_core_passes"]
            try:
                with torch.cuda.stream(stream):
                    res = pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, **kw), stream=stream)
                    ctx.sync(stream)
            except pq.PQError as e:
                assert e.status == pq.PQ_ERR_BUDGET, (ab, p, e)
                continue
            passes = ctx.stats()["out_of_core_passes"] - before
            seen.append(passes)
            want = oracle_plan(D, M, F, seg=p["seg"], mc=p["mc"], fc=p["fc"], k=p["k"],
                               d_op=kw["d_op"], m_op=kw["m_op"])
            assert_same(res.as_dict(), want, f"arena {ab / MB:.2f} MB, {p}, {passes} passes")
        ctx.close()
    return seen


PREDS = [dict(seg=1, mc=1200, fc=1200, k=10), dict(seg=0, mc=2000, fc=300, k=64),
         dict(seg=0, mc=0, fc=0, k=1, d_op="all", m_op="all")]
ARENAS = [int(x * MB) for x in (16, 5.5, 4.5, 4.0, 3.7, 3.5, 3.3, 3.1, 2.9)]


@pytest.mark.parametrize("mode", ["resident", "mapped"])
def test_small_workload_in_passes(stream, mode):
    D, M, F = datagen.workload("small")
    seen = sweep(stream, D, M, F, mode, PREDS, ARENAS)
    assert 0 in seen, "the large arena runs the plan in one piece"
    assert max(seen) >= 3, f"the small arenas force passes: {seen}"


def test_repeated_build_keys_in_passes(stream):
    """M keys held by two rows: the copy counts of each pass's window."""
    rng = np.random.default_rng(17)
    D, M, F = datagen.make(3000, 40_000, 160_000, seed=17)
    M = dict(M)
    dup = rng.integers(0, 40_000, size=6000)
    M["key"] = M["key"].copy()
    M["key"][dup] = M["key"][(dup + 1) % 40_000]
    seen = sweep(stream, D, M, F, "resident", PREDS[:2],
                 [int(x * MB) for x in (8, 1.9, 1.7, 1.5, 1.4, 1.3, 1.2)])
    assert max(seen) >= 2, seen
