"""Packed columns (frame of reference + bit packing) on the host, no GPU:
pq_pack_column's output is decoded here by a reference reader written from
the layout in pq.h (header, block table, LSB-first bit streams) and must give
back the input exactly; block widths are the fewest bits for each block's
spread; sizes stay within pq_pack_bound; bad arguments and short buffers are
refused."""
import ctypes
import struct

import numpy as np
import pytest

import paper_2512_02862_gb300 as pq

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return pq.library()


CODES = {np.dtype(np.int8): pq.PQ_INT8, np.dtype(np.int32): pq.PQ_INT32,
         np.dtype(np.int64): pq.PQ_INT64}


def pack(lib, a, cap=None):
    a = np.ascontiguousarray(a)
    code = CODES[a.dtype]
    bound = lib.pq_pack_bound(len(a), code)
    cap = bound if cap is None else cap
    buf = np.zeros(max(cap, 1), dtype=np.uint8)
    used = ctypes.c_int64(0)
    st = lib.pq_pack_column(a.ctypes.data if len(a) else None, code, len(a),
                            buf.ctypes.data, cap, ctypes.byref(used))
    return st, buf[:used.value].tobytes(), bound


def read_packed(b: bytes):
    """Reference reader: the layout documented in pq.h."""
    magic, version, typ, block_rows, nrows, nblocks = struct.unpack_from("<IIiIqq", b, 0)
    assert magic == 0x4B505150 and version == 1
    table = [struct.unpack_from("<qIB3x", b, 32 + 16 * i) for i in range(nblocks + 1)]
    pay = (32 + 16 * (nblocks + 1) + 15) // 16 * 16
    words = np.frombuffer(b, dtype="<u4", offset=pay)
    out = []
    for k in range(nblocks):
        base, first, width = table[k]
        rows = min(block_rows, nrows - k * block_rows)
        stream = 0
        nwords = (rows * width + 31) // 32
        for j in range(nwords):          # the block's bits as one integer, LSB first
            stream |= int(words[first + j]) << (32 * j)
        mask = (1 << width) - 1
        for i in range(rows):
            d = (stream >> (i * width)) & mask
            v = (base + d) & ((1 << 64) - 1)
            out.append(v - (1 << 64) if v >= 1 << 63 else v)
    assert table[nblocks][1] == sum((min(block_rows, nrows - k * block_rows) * table[k][2] + 31)
                                    // 32 for k in range(nblocks))
    return typ, nrows, [t[2] for t in table[:nblocks]], out


@pytest.mark.parametrize("dtype", [np.int8, np.int32, np.int64])
@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 4097, 3 * 4096 + 5])
def test_roundtrip_random(lib, dtype, n):
    rng = np.random.default_rng(n + np.dtype(dtype).itemsize)
    info = np.iinfo(dtype)
    a = rng.integers(info.min, info.max, size=n, dtype=dtype, endpoint=True)
    st, b, bound = pack(lib, a)
    assert st == 0 and len(b) <= bound
    typ, nrows, widths, out = read_packed(b)
    assert typ == CODES[np.dtype(dtype)] and nrows == n
    assert out == a.astype(np.int64).tolist()


def test_widths_are_minimal(lib):
    """Each block's width is the bit length of its max - min."""
    rng = np.random.default_rng(3)
    blocks = []
    for w in (0, 1, 7, 12, 31, 33, 63, 64):
        base = int(rng.integers(-2**40, 2**40))
        if w == 0:
            blk = np.full(4096, base, dtype=np.int64)
        elif w == 64:
            blk = rng.integers(-2**63, 2**63 - 1, size=4096, dtype=np.int64, endpoint=True)
            blk[0], blk[1] = -2**63, 2**63 - 1
        else:
            base = -(2**62) if w > 40 else base        # base + 2^w - 1 stays in int64
            blk = base + rng.integers(0, 2**w - 1, size=4096, dtype=np.int64, endpoint=True)
            blk[0], blk[1] = base, base + 2**w - 1       # spread exactly 2^w - 1
        blocks.append(blk)
    a = np.concatenate(blocks)
    st, b, _ = pack(lib, a)
    assert st == 0
    _, _, widths, out = read_packed(b)
    assert widths == [0, 1, 7, 12, 31, 33, 63, 64]
    assert out == a.tolist()


def test_generated_columns_shrink(lib):
    """The plan's columns pack well: dates fit 12 bits, discounts 4 bits."""
    import datagen
    D, M, F = datagen.workload("small")
    st, b, _ = pack(lib, F["date2"])
    _, _, widths, out = read_packed(b)
    assert st == 0 and max(widths) <= 12 and out == F["date2"].tolist()
    st, b, _ = pack(lib, F["disc"])
    _, _, widths, _ = read_packed(b)
    assert max(widths) <= 4


def test_errors(lib):
    a = np.arange(5000, dtype=np.int64) * 1000003
    st, _, bound = pack(lib, a, cap=100)
    assert st == pq.PQ_ERR_CAPACITY
    used = ctypes.c_int64(0)
    buf = np.zeros(bound, dtype=np.uint8)
    assert lib.pq_pack_column(a.ctypes.data, 9, len(a), buf.ctypes.data, bound,
                              ctypes.byref(used)) == pq.PQ_ERR_INVALID_ARG
    assert lib.pq_pack_column(None, pq.PQ_INT64, 10, buf.ctypes.data, bound,
                              ctypes.byref(used)) == pq.PQ_ERR_INVALID_ARG
    assert lib.pq_pack_bound(-1, pq.PQ_INT64) == -1
