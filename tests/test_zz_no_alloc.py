"""Allocation-free selection through the C ABI.

pq_filter_noalloc serves callers that cannot allocate device memory (code
running during a CUDA graph capture, or inside a runtime that owns every
allocation): it takes no context and keeps its scratch in a static device
array of the library.  Its output must equal pq_filter's and the CPU
oracle's, exactly (row ids are integers), on two calls in a row that reuse
the same static scratch.
This file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def pq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    return pq


def _call(pq, s, x, op, c, out, cnt, err, sel=None, n_in=None):
    lib = pq.library()
    n = x.numel() if sel is None else n_in
    return lib.pq_filter_noalloc(pq.col(x), pq.CMP[op], int(c),
                                 None if sel is None else sel.data_ptr(), int(n),
                                 out.data_ptr(), cnt.data_ptr(), err.data_ptr(), pq._stream(s))


def test_noalloc_filter_matches_pq_filter_on_two_calls(pq):
    rng = np.random.default_rng(2026)
    a = rng.integers(0, 2406, size=3_000_017).astype(np.int32)   # many tiles, ragged tail
    x = torch.from_numpy(a).cuda()
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=256 << 20)
    # outputs allocated by the caller up front; the entry point allocates nothing
    out = torch.empty(len(a), dtype=torch.int64, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for op, c in (("<", 1200), (">=", 77)):
        assert _call(pq, s, x, op, c, out, cnt, err) == pq.PQ_OK
        with torch.cuda.stream(s):
            want, wcnt = pq.pq_filter(ctx, x, op, c, stream=s)
        s.synchronize()
        k = int(wcnt.item())
        assert int(cnt.item()) == k and int(err.item()) == 0, (op, c)
        assert torch.equal(out[:k], want[:k]), (op, c)
        assert np.array_equal(out[:k].cpu().numpy(), oracle.filter(a, op, c)), (op, c)
    ctx.close()


def test_noalloc_filter_with_selection_vector(pq):
    rng = np.random.default_rng(7)
    a = rng.integers(-1000, 1000, size=500_003).astype(np.int64)
    x = torch.from_numpy(a).cuda()
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=256 << 20)
    with torch.cuda.stream(s):
        sel, scnt = pq.pq_filter(ctx, x, ">", -200, stream=s)
        s.synchronize()
        n_in = int(scnt.item())
        sel = sel[:n_in].contiguous()
        want, wcnt = pq.pq_filter(ctx, x, "!=", 5, sel_in=sel, stream=s)
    out = torch.empty(n_in, dtype=torch.int64, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _call(pq, s, x, "!=", 5, out, cnt, err, sel=sel, n_in=n_in) == pq.PQ_OK
    s.synchronize()
    k = int(wcnt.item())
    assert int(cnt.item()) == k and int(err.item()) == 0
    assert torch.equal(out[:k], want[:k])
    want_cpu = oracle.filter(a, "!=", 5, sel_in=oracle.filter(a, ">", -200))
    assert np.array_equal(out[:k].cpu().numpy(), want_cpu)
    ctx.close()


def test_noalloc_filter_rejects_inputs_beyond_its_scratch(pq):
    lib = pq.library()
    # 2^30 rows exceeds the static scratch; refused before any GPU work, so the
    # (never dereferenced) column pointer may be anything non-null
    big = pq.pq_col(ctypes.c_void_p(16), 1 << 30, pq.PQ_INT32, 0)
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    st = lib.pq_filter_noalloc(big, pq.CMP["<"], 0, None, 0, out.data_ptr(), cnt.data_ptr(),
                               None, None)
    assert st == pq.PQ_ERR_CAPACITY
