"""The C-ABI library builds, loads and exports every entry point that
include/pq.h declares; the ctypes layouts match the C structs.  No compute
call is made (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

import __graft_entry__

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pq():
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    return pq


def test_every_header_symbol_is_exported(pq):
    lib = pq.library()
    syms = pq.header_symbols()
    assert len(syms) >= 25
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", pq.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(syms) <= exported


def test_struct_layouts_match_header(pq, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pq.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(pq_col),sizeof(pq_options),sizeof(pq_source),sizeof(pq_plan),'
                   'sizeof(pq_result),sizeof(pq_stats),sizeof(pq_tuning),'
                   'offsetof(pq_result,status));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(pq.pq_col), ctypes.sizeof(pq.pq_options), ctypes.sizeof(pq.pq_source),
            ctypes.sizeof(pq.pq_plan), ctypes.sizeof(pq.pq_result), ctypes.sizeof(pq.pq_stats),
            ctypes.sizeof(pq.pq_tuning), pq.pq_result.status.offset]
    assert got == want


def test_status_strings_and_defaults(pq):
    lib = pq.library()
    for code, name in pq.STATUS.items():
        assert lib.pq_status_string(code).decode() == name
    opt = pq.pq_options()
    assert lib.pq_default_options(ctypes.byref(opt)) == 0
    assert opt.block_threads == 256 and opt.chunk_bytes == 128 << 20
    assert abs(opt.load_factor - 0.5) < 1e-6 and opt.spin_limit > 0


def test_invalid_arguments_are_rejected_without_a_device(pq):
    lib = pq.library()
    h = ctypes.c_void_p()
    # a NULL arena is refused before any CUDA call
    assert lib.pq_create(None, None, 1 << 30, ctypes.byref(h)) == pq.PQ_ERR_INVALID_ARG
    assert lib.pq_create(None, None, 0, None) == pq.PQ_ERR_INVALID_ARG
    assert lib.pq_sync(None, None) == pq.PQ_ERR_INVALID_ARG
    assert lib.pq_run_plan(None, None, None, None) == pq.PQ_ERR_INVALID_ARG


def test_binding_refuses_to_run_without_library(pq, monkeypatch):
    monkeypatch.setattr(pq, "_lib", None)
    monkeypatch.setattr(pq, "LIB_PATH", "/nonexistent/libpq.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pq.library()
