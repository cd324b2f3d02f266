"""The seeded generator: determinism (also across thread counts), value
ranges and the structure the workloads state."""
import os
import subprocess
import sys

import numpy as np

import datagen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_workload_shape_and_ranges():
    D, M, F = datagen.workload("small")
    assert len(D["key"]) == 15_000 and len(M["key"]) == 150_000 and len(F["mkey"]) == 600_000
    assert np.array_equal(D["key"], np.arange(1, 15_001, dtype=np.int32))
    assert D["seg"].min() == 0 and D["seg"].max() == 4
    r = M["key"] - 4 * np.arange(len(M["key"]))
    assert r.min() == 0 and r.max() == 3                     # key = 4 i + U{0..3}
    assert M["dref"].min() >= 1 and M["dref"].max() <= 15_000
    assert M["date"].min() == 0 and M["date"].max() == 2405
    assert F["price"].min() >= 90_000 and F["price"].max() <= 10_500_000
    assert F["disc"].min() == 0 and F["disc"].max() == 10
    # clustered: F.mkey follows M order in runs of 1..7 (first lap)
    starts = datagen.f_starts(1, len(M["key"]), len(F["mkey"]))
    runs = np.diff(starts)
    assert runs[:-1].min() >= 1 and runs[:-1].max() <= 7
    i = np.searchsorted(starts, np.arange(starts[-1]), side="right") - 1
    assert np.array_equal(F["mkey"][:starts[-1]], M["key"][i])
    delta = F["date2"][:starts[-1]] - M["date"][i]
    assert delta.min() == 1 and delta.max() == 121
    # every F.mkey exists in M
    assert np.isin(F["mkey"], M["key"]).all()


def test_deterministic_across_thread_counts(tmp_path):
    code = ("import datagen,numpy as np,sys;d,m,f=datagen.make(100,3000,12000,seed=9);"
            "np.savez(sys.argv[1],a=f['mkey'],b=f['price'],c=m['key'],d=f['date2'])")
    outs = []
    for nt in ("1", "3"):
        p = str(tmp_path / f"o{nt}.npz")
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        subprocess.run([sys.executable, "-c", code, p], check=True, cwd=ROOT, env=env)
        outs.append(np.load(p))
    for k in "abcd":
        assert np.array_equal(outs[0][k], outs[1][k])


def test_zipf_foreign_keys_are_skewed():
    D, M, F = datagen.make(1000, 20_000, 200_000, seed=4, fk="zipf")
    assert np.isin(F["mkey"], M["key"]).all()
    _, counts = np.unique(F["mkey"], return_counts=True)
    counts = np.sort(counts)[::-1]
    # Zipf(1): frequency of rank r ~ 1/r; rank 1 holds ~1/H_n of the rows
    h = (1.0 / np.arange(1, 20_001)).sum()
    assert abs(counts[0] / 200_000 - 1 / h) < 0.01
    assert 1.6 < counts[0] / counts[1] < 2.5
