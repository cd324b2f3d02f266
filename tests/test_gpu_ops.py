"""Parity of the standalone operators (CUDA, through the C ABI) with the CPU
oracle: bit-exact ids, keys, sums and counts on seeded inputs that span many
tiles with ragged tails, plus the edge cases (empty input, all / none
passing, one bucket, the largest fan-out, duplicate keys, ties, capacity
overflow, the reserved key, unaligned columns)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02862_gb300 as pq  # noqa: E402

NP = {np.int8: torch.int8, np.int32: torch.int32, np.int64: torch.int64}


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    c = pq.Context(arena_bytes=6 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.Stream()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# 6,000,007 rows: more tiles than 8 per SM, the two-pass (count, scan, write) path
SIZES = [0, 1, 15, 16, 17, 4095, 4096, 4097, 100_003, 1_000_001, 6_000_007]


@pytest.mark.parametrize("dt", [np.int8, np.int32, np.int64])
@pytest.mark.parametrize("n", SIZES)
def test_filter_matches_oracle(ctx, stream, dt, n):
    rng = np.random.default_rng(n * 7 + np.dtype(dt).itemsize)
    a = rng.integers(-60, 60, size=n).astype(dt)
    x = dev(a)
    for op in ("<", "<=", ">", ">=", "==", "!=", "all"):
        c = int(rng.integers(-70, 70))
        with torch.cuda.stream(stream):
            out, cnt = pq.pq_filter(ctx, x, op, c, stream=stream)
            ctx.sync(stream)
        want = oracle.filter(a, op, c)
        k = int(cnt.item())
        assert k == len(want), (op, c)
        assert np.array_equal(out[:k].cpu().numpy(), want), (op, c)


@pytest.mark.parametrize("n", [5, 4097, 300_001, 12_000_001])
def test_filter_with_selection_vector(ctx, stream, n):
    rng = np.random.default_rng(n)
    a = rng.integers(0, 100, size=n).astype(np.int32)
    b = rng.integers(0, 100, size=n).astype(np.int64)
    sel = oracle.filter(a, "<", 50)
    want = oracle.filter(b, ">=", 30, sel)
    with torch.cuda.stream(stream):
        s1, c1 = pq.pq_filter(ctx, dev(a), "<", 50, stream=stream)
        k1 = int(c1.item())
        s2, c2 = pq.pq_filter(ctx, dev(b), ">=", 30, sel_in=s1[:k1].contiguous(), stream=stream)
        # count of the selection read on the device (deferred synchronisation)
        s3, c3 = pq.pq_filter(ctx, dev(b), ">=", 30, sel_in=s1, d_n_in=c1, stream=stream)
        ctx.sync(stream)
    assert np.array_equal(s2[:int(c2.item())].cpu().numpy(), want)
    assert np.array_equal(s3[:int(c3.item())].cpu().numpy(), want)


@pytest.mark.parametrize("n", [50_001, 6_000_001])
def test_filter_unaligned_column_takes_scalar_path(ctx, stream, n):
    rng = np.random.default_rng(3)
    a = rng.integers(0, 1000, size=n).astype(np.int32)
    x = dev(a)[1:]                      # 4-byte offset: not 16-byte aligned
    with torch.cuda.stream(stream):
        out, cnt = pq.pq_filter(ctx, x, "<", 500, stream=stream)
        ctx.sync(stream)
    want = oracle.filter(a[1:], "<", 500)
    assert np.array_equal(out[:int(cnt.item())].cpu().numpy(), want)


@pytest.mark.parametrize("kt", [np.int32, np.int64])
@pytest.mark.parametrize("log2P", [0, 1, 4, 6, 10, 12])
@pytest.mark.parametrize("n", [0, 1, 8191, 8193, 300_007])
def test_partition_matches_oracle(ctx, stream, kt, log2P, n):
    rng = np.random.default_rng(n + log2P)
    keys = rng.integers(-2**31, 2**31 - 1, size=n).astype(kt)
    rows = np.arange(n, dtype=np.int64)
    tag = rng.integers(-128, 127, size=n).astype(np.int8)
    w32 = rng.integers(-1000, 1000, size=n).astype(np.int32)
    with torch.cuda.stream(stream):
        ok, (orow, otag, ow), off = pq.pq_partition(ctx, dev(keys), [dev(rows), dev(tag), dev(w32)],
                                                    log2P=log2P, stream=stream)
        ctx.sync(stream)
    wk, (wrow, wtag, ww), woff = oracle.partition(keys, log2P, [rows, tag, w32])
    assert np.array_equal(off.cpu().numpy(), woff)
    assert np.array_equal(ok.cpu().numpy()[:n], wk)
    assert np.array_equal(orow.cpu().numpy()[:n], wrow)
    assert np.array_equal(otag.cpu().numpy()[:n], wtag)
    assert np.array_equal(ow.cpu().numpy()[:n], ww)


@pytest.mark.parametrize("log2P", [3, 9, 10])
@pytest.mark.parametrize("dist", ["uniform", "one-hot"])
def test_partition_large_and_skewed(ctx, stream, log2P, dist):
    """Several sub-tiles per block and a ragged tail (sub-tiles of 4096 rows
    from 512 buckets on, 2048 below); with one-hot keys most rows fall in
    one bucket (a run spanning whole sub-tiles)."""
    n = 3_000_017
    rng = np.random.default_rng(log2P)
    keys = rng.integers(-2**62, 2**62, size=n).astype(np.int64)
    if dist == "one-hot":
        keys[rng.random(n) < 0.9] = 12345
    rows = np.arange(n, dtype=np.int64)
    with torch.cuda.stream(stream):
        ok, (orow,), off = pq.pq_partition(ctx, dev(keys), [dev(rows)], log2P=log2P,
                                           stream=stream)
        ctx.sync(stream)
    wk, (wrow,), woff = oracle.partition(keys, log2P, [rows])
    assert np.array_equal(off.cpu().numpy(), woff)
    assert np.array_equal(ok.cpu().numpy()[:n], wk)
    assert np.array_equal(orow.cpu().numpy()[:n], wrow)


def test_partition_unaligned_columns(ctx, stream):
    """Columns that start off a 16-byte boundary take the scatter without
    bulk copies; the result is the same."""
    n = 1_000_003
    rng = np.random.default_rng(99)
    keys = rng.integers(-2**40, 2**40, size=n + 1).astype(np.int64)
    pay = rng.integers(-100, 100, size=n + 1).astype(np.int32)
    with torch.cuda.stream(stream):
        dk, dp = dev(keys), dev(pay)
        ok, (op,), off = pq.pq_partition(ctx, dk[1:], [dp[1:]], log2P=7, stream=stream)
        ctx.sync(stream)
    wk, (wp,), woff = oracle.partition(keys[1:].copy(), 7, [pay[1:].copy()])
    assert np.array_equal(off.cpu().numpy(), woff)
    assert np.array_equal(ok.cpu().numpy()[:n], wk)
    assert np.array_equal(op.cpu().numpy()[:n], wp)


def join_pairs(rows, vals, cnt):
    k = int(cnt.item())
    r, v = rows[:k].cpu().numpy(), vals[:k].cpu().numpy()
    order = np.lexsort((v, r))
    return r[order], v[order]


@pytest.mark.parametrize("nb,np_", [(0, 100), (100, 0), (1000, 5000), (200_000, 1_000_003)])
def test_join_matches_oracle(ctx, stream, nb, np_):
    rng = np.random.default_rng(nb + np_)
    bk = rng.integers(0, max(nb, 1) // 2 + 1, size=nb).astype(np.int64)   # duplicates
    bv = rng.integers(-10**9, 10**9, size=nb).astype(np.int64)
    pk = rng.integers(0, max(nb, 1), size=np_).astype(np.int32)
    wr, wv = oracle.join(bk, pk, bv)
    with torch.cuda.stream(stream):
        ht = pq.pq_join_build(ctx, dev(bk), dev(bv), stream=stream)
        rows, vals, cnt = pq.pq_join_probe(ctx, ht, dev(pk), cap=len(wr) + 10, stream=stream)
        ctx.sync(stream)
        ht.free(stream)
    r, v = join_pairs(rows, vals, cnt)
    assert np.array_equal(r, wr) and np.array_equal(v, wv)


def test_join_unique_keys_and_row_id_values(ctx, stream):
    rng = np.random.default_rng(11)
    bk = rng.permutation(500_000).astype(np.int64) * 3
    pk = rng.integers(0, 1_500_000, size=700_001).astype(np.int64)
    wr, wv = oracle.join(bk, pk)
    with torch.cuda.stream(stream):
        ht = pq.pq_join_build(ctx, dev(bk), None, load_factor=0.7, stream=stream)
        rows, vals, cnt = pq.pq_join_probe(ctx, ht, dev(pk), cap=len(wr), stream=stream)
        ctx.sync(stream)
        ht.free(stream)
    r, v = join_pairs(rows, vals, cnt)
    assert np.array_equal(r, wr) and np.array_equal(v, wv)


def test_join_capacity_overflow_reports_needed_count(ctx, stream):
    bk = np.arange(1000, dtype=np.int64)
    pk = np.tile(np.arange(1000, dtype=np.int64), 3)
    with torch.cuda.stream(stream):
        ht = pq.pq_join_build(ctx, dev(bk), stream=stream)
        rows, vals, cnt = pq.pq_join_probe(ctx, ht, dev(pk), cap=100, stream=stream)
        with pytest.raises(pq.PQError) as e:
            ctx.sync(stream)
        ht.free(stream)
    assert e.value.status == pq.PQ_ERR_CAPACITY
    assert int(cnt.item()) == 3000


def test_reserved_key_is_reported(ctx, stream):
    bk = np.array([1, 2, np.iinfo(np.int64).min, 4], dtype=np.int64)
    with torch.cuda.stream(stream):
        ht = pq.pq_join_build(ctx, dev(bk), stream=stream)
        with pytest.raises(pq.PQError) as e:
            ctx.sync(stream)
        ht.free(stream)
    assert e.value.status == pq.PQ_ERR_RESERVED_KEY


def groups_sorted(ok, os_, cnt):
    g = int(cnt.item())
    k, s = ok[:g].cpu().numpy(), os_[:g].cpu().numpy()
    o = np.argsort(k, kind="stable")
    return k[o], s[o]


@pytest.mark.parametrize("kt", [np.int32, np.int64])
@pytest.mark.parametrize("vt", [np.int8, np.int64])
@pytest.mark.parametrize("n,distinct", [(0, 1), (1, 1), (5000, 7), (1_000_003, 50_000),
                                        (2_000_000, 1_500_000)])
def test_groupby_matches_oracle(ctx, stream, kt, vt, n, distinct):
    rng = np.random.default_rng(n + distinct)
    # Zipf-like skew: a few hot keys and a long tail
    k = (rng.zipf(1.3, size=n) % distinct).astype(kt) - 3
    lim = 10**12 if vt == np.int64 else 127
    v = rng.integers(-lim, lim, size=n).astype(vt)
    wk, ws, ovf = oracle.groupby_sum(k, v)
    assert not ovf
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_groupby_sum(ctx, dev(k), dev(v), cap=max(len(wk), 1), stream=stream)
        ctx.sync(stream)
    gk, gs = groups_sorted(ok, os_, cnt)
    assert np.array_equal(gk, wk) and np.array_equal(gs, ws)


@pytest.mark.parametrize("layout", ["clustered", "sparse", "capacity"])
def test_groupby_large_inputs(ctx, stream, layout):
    """Inputs of a million rows and more: dense keys take the slot array
    (clustered runs of one key, as F is by mkey: runs cut by the 128-row
    steps), keys spread over 2^40 values take the hash table, and a cap
    below the group count is reported on the dense path too."""
    rng = np.random.default_rng(17)
    n = 3_000_001
    if layout == "sparse":
        k = rng.integers(-(1 << 40), 1 << 40, size=n // 4).astype(np.int64)
        k = np.repeat(k, 4)[:n]
    else:
        k = (np.repeat(np.arange(n // 3 + 1, dtype=np.int64) * 4 - 1_000_000,
                       rng.integers(1, 6, size=n // 3 + 1)))[:n]
    v = rng.integers(-10**9, 10**9, size=len(k)).astype(np.int64)
    wk, ws, ovf = oracle.groupby_sum(k, v)
    assert not ovf
    cap = 1000 if layout == "capacity" else len(wk)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_groupby_sum(ctx, dev(k), dev(v), cap=cap, stream=stream)
        if layout == "capacity":
            with pytest.raises(pq.PQError) as e:
                ctx.sync(stream)
            assert e.value.status == pq.PQ_ERR_CAPACITY and int(cnt.item()) == len(wk)
            return
        ctx.sync(stream)
    gk, gs = groups_sorted(ok, os_, cnt)
    assert np.array_equal(gk, wk) and np.array_equal(gs, ws)


def test_groupby_capacity_overflow(ctx, stream):
    k = np.arange(10_000, dtype=np.int64)
    v = np.ones(10_000, dtype=np.int64)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_groupby_sum(ctx, dev(k), dev(v), cap=100, stream=stream)
        with pytest.raises(pq.PQError) as e:
            ctx.sync(stream)
    assert e.value.status == pq.PQ_ERR_CAPACITY
    assert int(cnt.item()) > 100


@pytest.mark.parametrize("n", [0, 1, 5, 1000, 100_003, 2_000_000])
@pytest.mark.parametrize("k", [1, 10, 32, 33, 64])
def test_topk_matches_oracle(ctx, stream, n, k):
    rng = np.random.default_rng(n * 3 + k)
    keys = rng.permutation(max(4 * n, 1))[:n].astype(np.int64)
    sums = rng.integers(-50, 50, size=n).astype(np.int64)   # heavy ties: key decides
    wk, ws = oracle.topk(keys, sums, k)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_topk(ctx, dev(keys), dev(sums), k, stream=stream)
        ctx.sync(stream)
    m = int(cnt.item())
    assert m == len(wk)
    assert np.array_equal(ok[:m].cpu().numpy(), wk) and np.array_equal(os_[:m].cpu().numpy(), ws)


@pytest.mark.parametrize("k", [10, 32, 64])
def test_topk_identical_entries(ctx, stream, k):
    # Repeated (key, sum) pairs: the list must keep every copy, in order.
    rng = np.random.default_rng(k)
    keys = rng.integers(0, 40, size=50_000).astype(np.int64)
    sums = (keys % 7).astype(np.int64)
    wk, ws = oracle.topk(keys, sums, k)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_topk(ctx, dev(keys), dev(sums), k, stream=stream)
        ctx.sync(stream)
    m = int(cnt.item())
    assert m == len(wk) == k
    assert np.array_equal(ok[:m].cpu().numpy(), wk) and np.array_equal(os_[:m].cpu().numpy(), ws)


@pytest.mark.parametrize("k,where", [(5, "block"), (10, "block"), (32, "block"), (32, "final")])
def test_topk_lane_lists_overflow(ctx, stream, k, where):
    # Blocks of 256 threads take 2048 consecutive pairs each (40 blocks for
    # 81,920 pairs); a thread takes every 256th pair of its block's range and
    # keeps its best 4.  "block": the 8 best pairs all fall to thread 0 of
    # block 0; "final": the best pair of blocks 0, 8, 16, 24 and 32 (each its
    # list's first entry, list entry e = 32 * block) fall to thread 0 of the
    # merge of the 40 lists, which takes entries 0, 256, 512, ...
    n = 40 * 2048
    rng = np.random.default_rng(k)
    keys = rng.permutation(n).astype(np.int64)
    sums = rng.integers(0, 10**6, size=n).astype(np.int64)
    if where == "block":
        rows = np.arange(8) * 256
    else:
        rows = np.array([0, 8, 16, 24, 32]) * 2048
    sums[rows] = 10**9 + np.arange(len(rows))
    wk, ws = oracle.topk(keys, sums, k)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_topk(ctx, dev(keys), dev(sums), k, stream=stream)
        ctx.sync(stream)
    m = int(cnt.item())
    assert m == len(wk) == k
    assert np.array_equal(ok[:m].cpu().numpy(), wk) and np.array_equal(os_[:m].cpu().numpy(), ws)


@pytest.mark.parametrize("order", ["ascending", "descending", "equal"])
@pytest.mark.parametrize("k", [1, 10, 32])
def test_topk_sorted_inputs(ctx, stream, order, k):
    # Pairs sorted by sum (either way) or all of one sum: the block
    # threshold taken from a few spread pairs per thread must keep every
    # pair that can be among the k best.
    n = 2_000_000
    rng = np.random.default_rng(k)
    keys = rng.permutation(n).astype(np.int64)
    sums = np.sort(rng.integers(-10**9, 10**9, size=n)).astype(np.int64)
    if order == "descending":
        sums = sums[::-1].copy()
    elif order == "equal":
        sums[:] = 7
    wk, ws = oracle.topk(keys, sums, k)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_topk(ctx, dev(keys), dev(sums), k, stream=stream)
        ctx.sync(stream)
    m = int(cnt.item())
    assert m == len(wk) == k
    assert np.array_equal(ok[:m].cpu().numpy(), wk) and np.array_equal(os_[:m].cpu().numpy(), ws)


def test_topk_count_from_device(ctx, stream):
    rng = np.random.default_rng(5)
    keys = np.arange(100_000, dtype=np.int64)
    sums = rng.integers(0, 10**12, size=100_000).astype(np.int64)
    n_dev = torch.tensor([60_000], dtype=torch.int64, device="cuda")
    wk, ws = oracle.topk(keys[:60_000], sums[:60_000], 10)
    with torch.cuda.stream(stream):
        ok, os_, cnt = pq.pq_topk(ctx, dev(keys), dev(sums), 10, d_n=n_dev, stream=stream)
        ctx.sync(stream)
    assert np.array_equal(ok.cpu().numpy(), wk) and np.array_equal(os_.cpu().numpy(), ws)
