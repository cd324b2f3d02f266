"""The benchmark's reference arm (the CPU oracle) on the host, no GPU: one
JSON line with the contract's keys, the oracle's rows per second as `value`,
and an end-to-end figure equal to it with no host-device bytes; ranks other
than 0 print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       env=e, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_reference_line_keeps_the_contract():
    lines = run_bench("--impl", "reference", "--workload", "small", "--steps", "2",
                      "--warmup", "3")
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["unit"] == "rows/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    # the small workload fits the time budget: every step is the whole workload
    assert d["cpu_baseline"]["whole_workload"] and d["cpu_baseline"]["f_rows_per_step"] == 600_000
    assert d["e2e"] == {"value": d["value"], "unit": "rows/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - 1e3 * 600_000 / d["value"]) < 1e-6 * d["ms_per_step"] + 1e-9
    assert set(d["config"]) == {"workload", "query", "l2", "parallelism"}


def test_reference_takes_a_consistent_slice_over_budget():
    """A time budget the whole workload does not fit: each step runs the
    oracle on the first M rows and exactly their F rows (D whole)."""
    d = json.loads(run_bench("--impl", "reference", "--workload", "small", "--steps", "2",
                             "--ref-budget-s", "0.001")[0])
    cb = d["cpu_baseline"]
    assert not cb["whole_workload"] and 0 < cb["f_rows_per_step"] < 600_000
    assert "M rows [0," in cb["sample"]


def test_reference_runs_on_rank_zero_only():
    assert run_bench("--impl", "reference", "--workload", "small", "--steps", "1",
                     env={"RANK": "1"}) == []
