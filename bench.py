"""Benchmark of the three-table plan on GB300 through the C ABI.

Default workload (one GPU): x100 -- D 1.5M, M 15M, F 60M rows resident in
HBM; D.seg == 1, M.date < 1200, F.date2 > 1200; join F-M-D; group by M key
SUM(price * (100 - disc)); top-10.  A step is one pq_run_plan over the whole
workload.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload x100|small|skew] [--mode plan|serve|stream]

--impl reference times the CPU oracle (the plain relational definition,
single-threaded) on the same workload, metric and unit.
--mode serve: batched / served execution of a query stream against the plain
one-query-at-a-time path (queries/s, p50/p99 latency).
--mode stream: the storage-resident plan (x2000 by default) streamed from
pinned host memory, against the measured host-to-device link.
--mode aggfirst: the aggregate-first plan (group F by key, filter on the sum,
semi-join with M', top-k) beside the join-first plan on the same tables.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "plan rows/s and GB/s vs HBM/host-link roofline; p50/p99 latency batched vs plain"
L2_BYTES = 129 * 2**20
WORKLOAD_TEXT = {
    "small": "small: D 15k, M 150k, F 600k rows",
    "x100": "x100: D 1.5M, M 15M, F 60M rows, all columns resident in HBM",
    "x2000": "x2000: D 30M, M 300M, F 1.2B rows in pinned host memory, 128 MiB chunks, "
             "16 GB device budget",
    "skew": "skew: D 4M, M 40M, F 200M rows, Zipf(1.0) foreign keys, pass-all predicates",
}
QUERY_TEXT = ("D.seg == 1, M.date < 1200, F.date2 > 1200; join F-M-D; group by M.key "
              "SUM(price*(100-disc)) int64; top-10")
SKEW_QUERY_TEXT = ("pass-all predicates; join F-M-D; group by M.key SUM(price*(100-disc)) "
                   "int64; top-10")


def table_bytes(n_d, n_m, n_f):
    """Algorithmic bytes of a plan: every referenced column read once."""
    return 5 * n_d + 16 * n_m + 21 * n_f


def moved_bytes(n_d, n_m, n_f, hits):
    """Bytes the plan's kernels load from the tables (an upper bound): the D
    and M columns in full, date2 and mkey of every F row, price and disc
    only for the F rows that joined."""
    return 5 * n_d + 16 * n_m + 12 * n_f + 9 * hits


def bench_config(workload: str, n_gpus: int) -> dict:
    """The `config` both arms print (identical, so the arms are comparable)."""
    import datagen
    w = datagen.WORKLOADS[workload]
    nbytes = table_bytes(w["n_d"], w["n_m"], w["n_f"])
    return {"workload": WORKLOAD_TEXT[workload],
            "query": SKEW_QUERY_TEXT if workload == "skew" else QUERY_TEXT,
            "l2": f"inputs ({nbytes / 1e9:.2f} GB) larger than L2 (129 MB); no flush between "
                  "steps",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU"}


def query(name):
    import datagen
    q = dict(datagen.QUERY)
    if name == "skew":
        return dict(seg=0, m_date_lt=0, f_date_gt=0, k=10, d_op="all", m_op="all", f_op="all")
    return dict(seg=q["seg"], m_date_lt=q["m_date_lt"], f_date_gt=q["f_date_gt"], k=q["k"],
                d_op="==", m_op="<", f_op=">")


# ------------------------------------------------------------------ clocks ----
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.time()  # the timed region starts once sampling has started
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.lines.clear()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers ----
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("pq_plan_kernels.cuh", "pq_dev.cuh", "pq_topk.cuh"):
        with open(os.path.join(ROOT, "paper_2512_02862_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        t = json.load(fh)
    e = t.get(kernel, {}).get(workload)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the job's time is its slowest replica)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, t_max_s: float, world: int) -> float:
    """Whole-job throughput of `world` replicas: all units over the slowest time."""
    return world * units_per_rank * steps / t_max_s


# -------------------------------------------------------------- CPU side ----
def cpu_oracle_rate(D, M, F, q, budget_s=20.0, max_runs=3):
    """Oracle (single-threaded) on the workload: F rows per second, runs,
    seconds, and the result of the last run (for the parity check)."""
    import oracle
    oracle.build()
    runs, t_total = 0, 0.0
    n_f = len(F["mkey"])
    want = None
    while runs < max_runs and t_total < budget_s:
        t0 = time.perf_counter()
        want = oracle.run_plan(D, M, F, **q)
        t_total += time.perf_counter() - t0
        runs += 1
    return n_f * runs / t_total, runs, t_total, want


def same_as_oracle(got: dict, want: dict) -> bool:
    return (got["status"] == want["status"] and got["ngroups"] == want["ngroups"]
            and got["keys"] == [int(x) for x in want["keys"]]
            and got["sums"] == [int(x) for x in want["sums"]])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import datagen
    import oracle
    oracle.build()
    D, M, F = datagen.workload(args.workload)
    q = query(args.workload)
    # Each step runs the oracle on the whole workload when the warm-up and
    # timed steps fit in --ref-budget-s; otherwise on a self-consistent slice
    # of it (the first rows of M and exactly their F rows, F being grouped by
    # M key, with D whole), sized so that they do.
    t0 = time.perf_counter()
    oracle.run_plan(D, M, F, **q)
    t_full = time.perf_counter() - t0
    n_m, n_f = len(M["key"]), len(F["mkey"])
    frac = min(1.0, args.ref_budget_s / max(1e-9, t_full * (args.steps + args.warmup)))
    if frac < 1.0 and args.workload != "skew":
        w = datagen.WORKLOADS[args.workload]
        starts = datagen.f_starts(w["seed"], n_m, n_f)
        m_rows = max(16, int(n_m * frac))
        f_rows = int(starts[m_rows]) if m_rows < n_m else n_f
        Ms = {k: v[:m_rows] for k, v in M.items()}
        Fs = {k: v[:f_rows] for k, v in F.items()}
        sample = (f"M rows [0, {m_rows}) and their F rows [0, {f_rows}) with D whole, per step "
                  f"(the whole workload takes {t_full:.1f} s per run)")
    else:
        Ms, Fs, f_rows = M, F, n_f
        sample = f"the whole workload ({n_f} F rows) per step"
    for _ in range(max(0, args.warmup - 1)):
        oracle.run_plan(D, Ms, Fs, **q)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run_plan(D, Ms, Fs, **q)
    t = time.perf_counter() - t0
    value = f_rows * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": bench_config(args.workload, args.gpus),
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "f_rows_per_step": int(f_rows),
                         "whole_workload": bool(f_rows == n_f)},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU side ----
def _events_ms(torch, s, fn, reps):
    """Mean milliseconds of fn() over reps runs, CUDA events on stream s."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        a.record(s)
        for _ in range(reps):
            fn()
        b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def skew_sub(pq, torch, s, hbm, reps=20):
    """The skewed workload (F 200M rows, Zipf(1.0) foreign keys into M 40M,
    pass-all predicates, ~20M groups) timed at full size, plain and
    partitioned (2^8 buckets), with parity against the oracle checked at
    1/20 scale through the same kernels (the oracle needs minutes at full
    size)."""
    import datagen
    import oracle
    q = query("skew")
    w = datagen.WORKLOADS["skew"]
    out = {"workload": WORKLOAD_TEXT["skew"], "query": SKEW_QUERY_TEXT}

    def tables(ctx, D, M, F):
        dev = {k: {c: torch.from_numpy(v).cuda() for c, v in t.items()}
               for k, t in (("D", D), ("M", M), ("F", F))}
        with torch.cuda.stream(s):
            TD = pq.pq_load_columns(ctx, [dev["D"]["key"], dev["D"]["seg"]], stream=s)
            TM = pq.pq_load_columns(ctx, [dev["M"][c] for c in ("key", "dref", "date")], stream=s)
            TF = pq.pq_load_columns(ctx, [dev["F"][c] for c in ("mkey", "price", "disc", "date2")],
                                    stream=s)
        return TD, TM, TF, dev

    # parity at 1/20 scale
    D, M, F = datagen.make(w["n_d"] // 20, w["n_m"] // 20, w["n_f"] // 20, seed=w["seed"],
                           fk="zipf", zipf_s=w["zipf_s"])
    t0 = time.perf_counter()
    want = oracle.run_plan(D, M, F, **q)
    t_oracle = time.perf_counter() - t0
    ctx = pq.Context(arena_bytes=4 << 30)
    TD, TM, TF, keep = tables(ctx, D, M, F)
    res = pq.pinned_results(1)
    ok = True
    for flags, lp in ((0, 0), (pq.PQ_PLAN_PARTITIONED, 8)):
        with torch.cuda.stream(s):
            pq.pq_run_plan(ctx, pq.make_plan(TD, TM, TF, flags=flags, log2P=lp, **q), res[0],
                           stream=s)
            ctx.sync(s)
        ok = ok and same_as_oracle(res[0].as_dict(), want)
    ctx.close()
    del keep
    out["parity"] = {"oracle": ok, "scale": "1/20 (F 10M rows)", "groups": want["ngroups"],
                     "oracle_s": round(t_oracle, 1)}
    # full size
    D, M, F = datagen.workload("skew")
    n_d, n_m, n_f = w["n_d"], w["n_m"], w["n_f"]
    ctx = pq.Context(arena_bytes=16 << 30)
    TD, TM, TF, keep = tables(ctx, D, M, F)
    nbytes = table_bytes(n_d, n_m, n_f)
    legs, first = {}, None
    for name, flags, lp in (("plain", 0, 0), ("partitioned_2^8", pq.PQ_PLAN_PARTITIONED, 8)):
        plan = pq.make_plan(TD, TM, TF, flags=flags, log2P=lp, **q)
        with torch.cuda.stream(s):
            for _ in range(3):
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
        r = res[0].as_dict()
        first = first or r
        ms = _events_ms(torch, s, lambda: pq.pq_run_plan(ctx, plan, res[0], stream=s), reps)
        ctx.sync(s)
        legs[name] = {"ms_per_plan": round(ms, 4), "rows_per_s": n_f / (ms / 1e3),
                      "gb_per_s": round(nbytes / (ms / 1e3) / 1e9, 1),
                      "frac_of_hbm": round(nbytes / (ms / 1e3) / 1e9 / hbm, 4),
                      "same_result_as_plain": r == first}
    out.update({"legs": legs, "groups": first["ngroups"], "algorithmic_bytes": nbytes,
                "timing": f"CUDA events over {reps} plans after 3 warm-ups (graph replay)"})
    ctx.close()
    return out


def serve_sub(pq, torch, ctx, s, tables, data, n_queries=500, rate=500.0, sample=8):
    """Serving on the resident x100 tables: n_queries queries of the serving
    workload (lognormal F slices, randomised predicates, Poisson arrivals at
    `rate`), plain one-at-a-time vs batched vs served, closed loop, and the
    open-loop p50/p99 latency; results identical across the three paths and
    equal to the oracle's on a sample of the queries."""
    import datagen
    import oracle
    TD, TM, TF = tables
    D, M, F = data
    w = datagen.WORKLOADS["x100"]
    starts = datagen.f_starts(w["seed"], w["n_m"], w["n_f"])
    qs = datagen.query_stream(5, n_queries, w["n_m"], starts, rate_qps=rate)

    def mk(q, flags):
        return pq.make_plan(TD, TM, TF, seg=q["seg"], m_date_lt=q["c"], f_date_gt=q["c"], k=10,
                            rows=dict(m=(q["m_row0"], q["m_rows"]), f=(q["f_row0"], q["f_rows"])),
                            flags=flags)

    plain_plans = [mk(q, pq.PQ_PLAN_NO_GRAPH) for q in qs]
    serve_plans = [mk(q, 0) for q in qs]
    n = len(qs)
    rp, rb = pq.pinned_results(n), pq.pinned_results(n)

    def plain():
        with torch.cuda.stream(s):
            for i, p in enumerate(plain_plans):
                pq.pq_run_plan(ctx, p, rp[i], stream=s)
                ctx.sync(s)

    def batched():
        with torch.cuda.stream(s):
            for a in range(0, n, 512):
                sub = serve_plans[a:a + 512]
                arr = (pq.pq_plan * len(sub))(*sub)
                dst = pq.ctypes.cast(pq.ctypes.addressof(rb) + a * pq.ctypes.sizeof(pq.pq_result),
                                     pq.ctypes.POINTER(pq.pq_result))
                ctx.check(pq.library().pq_run_batch(ctx.h, arr, len(sub), dst, pq._stream(s)))
            ctx.sync(s)

    def served():
        tickets = [pq.pq_submit(ctx, p) for p in serve_plans]
        res = []
        for t in tickets:
            st, r, lat = pq.pq_poll(ctx, t, timeout_ms=60_000)
            assert st == pq.PQ_OK, st
            res.append(r.as_dict())
        return res

    plain(); batched(); served()      # warm-up: code, caches, resident D-sets
    t0 = time.perf_counter(); plain(); t_plain = time.perf_counter() - t0
    t0 = time.perf_counter(); batched(); t_batch = time.perf_counter() - t0
    t0 = time.perf_counter(); sres = served(); t_serve = time.perf_counter() - t0
    pres = [rp[i].as_dict() for i in range(n)]
    bres = [rb[i].as_dict() for i in range(n)]
    identical = pres == bres == sres
    pick = np.linspace(0, n - 1, sample).astype(int)
    cut = lambda t, r0, nn: {c: v[r0:r0 + nn] for c, v in t.items()}
    oracle_ok = all(same_as_oracle(pres[i], oracle.run_plan(
        D, cut(M, qs[i]["m_row0"], qs[i]["m_rows"]), cut(F, qs[i]["f_row0"], qs[i]["f_rows"]),
        seg=qs[i]["seg"], m_date_lt=qs[i]["c"], f_date_gt=qs[i]["c"], k=10)) for i in pick)
    # open loop: arrivals on the Poisson schedule
    arrive = np.array([q["arrive_s"] for q in qs])
    lat_plain = []
    t_start = time.perf_counter()
    with torch.cuda.stream(s):
        for i, p in enumerate(plain_plans):
            now = time.perf_counter() - t_start
            if now < arrive[i]:
                time.sleep(arrive[i] - now)
            pq.pq_run_plan(ctx, p, rp[i], stream=s)
            ctx.sync(s)
            lat_plain.append(time.perf_counter() - t_start - arrive[i])
    tickets = [None] * n

    def feeder():
        t_s = time.perf_counter()
        for i, p in enumerate(serve_plans):
            now = time.perf_counter() - t_s
            if now < arrive[i]:
                time.sleep(arrive[i] - now)
            tickets[i] = pq.pq_submit(ctx, p)

    th = threading.Thread(target=feeder)
    th.start()
    lat_serve = []
    for i in range(n):
        while tickets[i] is None:
            time.sleep(1e-4)
        st, r, lat = pq.pq_poll(ctx, tickets[i], timeout_ms=60_000)
        identical = identical and st == pq.PQ_OK and r.as_dict() == pres[i]
        lat_serve.append(lat / 1e6)
    th.join()
    pct = lambda a, p: round(1e3 * float(np.percentile(a, p)), 3)
    return {"workload": f"{n} queries on slices of x100 (F rows lognormal, median 500k, "
                        f"sigma 1.5), randomised seg and date constants, Poisson {rate} q/s",
            "closed_loop_qps": {"plain": n / t_plain, "batched": n / t_batch,
                                "served": n / t_serve},
            "speedup_vs_plain": {"batched": round(t_plain / t_batch, 2),
                                 "served": round(t_plain / t_serve, 2)},
            "open_loop_latency_ms": {"plain": {"p50": pct(lat_plain, 50),
                                               "p99": pct(lat_plain, 99)},
                                     "served": {"p50": pct(lat_serve, 50),
                                                "p99": pct(lat_serve, 99)}},
            "parity": {"identical_across_paths": bool(identical), "oracle": bool(oracle_ok),
                       "oracle_sample": f"{sample} of the {n} queries"}}


def run_ours(args):
    import torch

    import __graft_entry__
    import datagen
    rank, world, local = dist_setup(args.gpus)
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq

    w = datagen.WORKLOADS[args.workload]
    n_d, n_m, n_f = w["n_d"], w["n_m"], w["n_f"]
    q = query(args.workload)
    # Pinned host copies of the tables (for the end-to-end leg), device copies
    # (resident leg).
    host = {}
    for name, cols, n in (("D", datagen.D_COLS, n_d), ("M", datagen.M_COLS, n_m),
                          ("F", datagen.F_COLS, n_f)):
        host[name] = {c: torch.empty(n, dtype=getattr(torch, np.dtype(dt).name), pin_memory=True)
                      for c, dt in cols}
    out = {k: {c: t.numpy() for c, t in v.items()} for k, v in host.items()}
    D, M, F = datagen.workload(args.workload, out=out)
    dev = {k: {c: t.cuda() for c, t in v.items()} for k, v in host.items()}
    torch.cuda.synchronize()

    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=args.arena_gb << 30, profile=0)
    with torch.cuda.stream(s):
        TD = pq.pq_load_columns(ctx, [dev["D"]["key"], dev["D"]["seg"]], stream=s)
        TM = pq.pq_load_columns(ctx, [dev["M"]["key"], dev["M"]["dref"], dev["M"]["date"]],
                                stream=s)
        TF = pq.pq_load_columns(ctx, [dev["F"][c] for c in ("mkey", "price", "disc", "date2")],
                                stream=s)
    plan = pq.make_plan(TD, TM, TF, **q)
    res = pq.pinned_results(1)

    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
        ctx.sync(s)
    check = res[0].as_dict()
    launches0 = ctx.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(s):
            ev0.record(s)
            evs = []
            for _ in range(args.steps):
                a = torch.cuda.Event(enable_timing=True)
                a.record(s)
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
                evs.append(a)
            ev1.record(s)
        torch.cuda.synchronize()
        barrier(world)
    ctx.sync(s)
    t_ms = ev0.elapsed_time(ev1)
    evs.append(ev1)
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(evs) - 1)]
    t_ms = max_over_ranks(t_ms, world)
    launches = ctx.stats()["kernel_launches"] - launches0
    assert res[0].as_dict() == check, "results changed between steps"

    # Kernel timing: the timed steps above replay the plan's CUDA graph with
    # no per-kernel events; a second pass of the same K steps runs the plan's
    # kernels as separate launches with an event pair around each kernel on
    # the launch stream (the bracket includes the launch, so kernel times are
    # upper bounds).
    ctx.profile_enable(True)
    with torch.cuda.stream(s):
        pq.pq_run_plan(ctx, plan, res[0], stream=s)
        ctx.sync(s)
        ctx.profile_reset()
        for _ in range(args.steps):
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
        ctx.sync(s)
    ctx.profile_enable(False)
    fscan_ms, fscan_n = ctx.profile("plan_fscan")
    per_stage = {}
    for nm in ("plan_dscan", "plan_dfill", "plan_dbuild", "plan_mscan", "plan_mfill",
               "plan_mbuild", "plan_mrank", "plan_mdup", "plan_fscan", "plan_fprobe",
               "plan_topk"):
        try:
            ms, n = ctx.profile(nm)
            per_stage[nm] = round(ms / max(n, 1), 5)
        except pq.PQError:
            pass
    assert res[0].as_dict() == check, "results changed between steps"

    value = job_rate(n_f, args.steps, t_ms / 1e3, world)
    plan_bytes = table_bytes(n_d, n_m, n_f)
    moved = moved_bytes(n_d, n_m, n_f, int(res[0].hits))
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    # Dominant kernel: the F scan.  Algorithmic bytes per launch: date2 and
    # mkey of every F row (12 B/row); price and disc of the ~0.5 % matching
    # rows are read by the probe kernel and not counted.
    fscan_bytes = 12 * n_f
    fscan_avg_s = fscan_ms / max(fscan_n, 1) / 1e3
    achieved = fscan_bytes / fscan_avg_s / 1e9
    roofline = {"kernel": "k_plan_fscan", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": ncu_traffic("k_plan_fscan", args.workload),
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src ==
                "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": fscan_bytes,
                "avg_launch_ms": round(fscan_avg_s * 1e3, 5), "launches": fscan_n,
                "timing": "CUDA events around each launch on its stream, in a second pass of "
                          "the same steps run as separate launches"}

    # End to end through the public API with host buffers: the tables live in
    # pinned host memory and every step moves its inputs over the host link
    # inside the timed region, then reads the result back to pinned host
    # memory.  Two paths: PQ_MAPPED (the plan kernels read the host columns in
    # place, so only the bytes they load cross the link) and PQ_STREAMING (the
    # tables are copied to the device chunk by chunk every step).
    e2e = None
    if not args.no_e2e:
        def host_plan_rate(ctx2, mode, src=None):
            src = src or host
            with torch.cuda.stream(s):
                HD = pq.pq_load_columns(ctx2, [src["D"]["key"], src["D"]["seg"]], mode=mode)
                HM = pq.pq_load_columns(ctx2, [src["M"][c] for c in ("key", "dref", "date")],
                                        mode=mode)
                HF = pq.pq_load_columns(ctx2, [src["F"][c] for c in ("mkey", "price", "disc",
                                                                    "date2")], mode=mode)
                hplan = pq.make_plan(HD, HM, HF, **q)
                hres = pq.pinned_results(1)
                pq.pq_run_plan(ctx2, hplan, hres[0], stream=s)
                ctx2.sync(s)
                st0 = ctx2.stats()
                k_e2e = max(1, min(args.steps, args.e2e_steps))
                barrier(world)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(k_e2e):
                    pq.pq_run_plan(ctx2, hplan, hres[0], stream=s)
                    ctx2.sync(s)
                t_e2e = max_over_ranks(time.perf_counter() - t0, world)
                st1 = ctx2.stats()
            assert hres[0].as_dict() == check, "end-to-end result differs from resident result"
            h2d = (st1["h2d_bytes"] - st0["h2d_bytes"]) // k_e2e
            if mode == pq.PQ_MAPPED:
                # Bytes the kernels load from the host columns (an upper bound:
                # the scanned columns in full, the probe's columns for the F
                # rows that joined).
                h2d = 5 * n_d + 16 * n_m + 12 * n_f + 17 * int(hres[0].hits)
            return {"value": world * n_f * k_e2e / t_e2e, "unit": "rows/s",
                    "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": (st1["d2h_bytes"] - st0["d2h_bytes"]) // k_e2e,
                    "steps": k_e2e, "ms_per_step": 1e3 * t_e2e / k_e2e}

        # The host tables in their packed storage form (frame of reference +
        # bit packing, made once by pq_pack_column, like files written ahead):
        # every step copies the packed bytes and decodes them on the device.
        t0 = time.perf_counter()
        packed = {tn: {c: pq.pq_pack_column(t) for c, t in cols.items()}
                  for tn, cols in host.items()}
        t_pack = time.perf_counter() - t0
        packed_bytes = sum(p.nbytes for cols in packed.values() for p in cols.values())

        def with_link(leg):
            leg["_link"] = True  # filled in after the legs (measure_h2d allocates 2 GiB)
            return leg

        def fill_link(leg, link):
            del leg["_link"]
            gbs = leg["h2d_bytes_per_step"] / (leg["ms_per_step"] / 1e3) / 1e9
            leg["link"] = {"gb_per_s": round(gbs, 1), "peak_gb_per_s": round(link, 1),
                           "frac": round(gbs / link, 4),
                           "peak": "measured here: pinned cudaMemcpyAsync host to device, "
                                   "1 GiB, best of 5"}
        # 256 MB chunks (of plain rows) on three copy streams: measured 2.78 ms
        # per plan against 3.03 ms with the default 128 MB on two.
        ctx2 = pq.Context(arena_bytes=args.arena_gb << 30, chunk_bytes=256 << 20, ring_slots=6,
                          copy_streams=3)
        e2e = with_link(host_plan_rate(ctx2, pq.PQ_STREAMING, packed))
        e2e["path"] = ("pq_run_plan on PQ_STREAMING tables of packed columns in pinned host "
                       "memory: chunked copies of the packed bytes, decoded on the device")
        e2e["packed"] = {"bytes": packed_bytes, "plain_bytes": plan_bytes,
                         "ratio": round(plan_bytes / packed_bytes, 2),
                         "pack_s": round(t_pack, 2), "chunk_bytes": 256 << 20,
                         "ring_slots": 6, "copy_streams": 3}
        ctx2.close()
        ctx3 = pq.Context(arena_bytes=args.arena_gb << 30)
        e2e["mapped"] = with_link(host_plan_rate(ctx3, pq.PQ_MAPPED))
        e2e["mapped"]["path"] = ("pq_run_plan on PQ_MAPPED tables in pinned host memory: the "
                                 "plan kernels read the plain columns in place")
        ctx3.close()
        ctx4 = pq.Context(arena_bytes=args.arena_gb << 30)
        e2e["streaming"] = with_link(host_plan_rate(ctx4, pq.PQ_STREAMING))
        e2e["streaming"]["path"] = ("pq_run_plan on PQ_STREAMING tables of plain columns in "
                                    "pinned host memory (chunked host-to-device copies)")
        ctx4.close()
        del packed
        link = measure_h2d()  # pinned host-to-device copy bandwidth, GB/s
        for leg in (e2e, e2e["mapped"], e2e["streaming"]):
            fill_link(leg, link)

    cpu = None
    parity = None
    if rank == 0 and not args.no_cpu:
        rate, runs, secs, want = cpu_oracle_rate(D, M, F, q,
                                                 max_runs=3 if world == 1 else 1)
        parity = {"oracle": same_as_oracle(check, want),
                  "what": "the timed plan's result (top-k keys and sums, group count, status) "
                          "against the CPU oracle's on the same full workload"}
        if world == 1:
            cpu = {"value": rate, "unit": "rows/s", "cores": 1, "kind": "oracle",
                   "sample": f"{runs} full run(s) of the plan on the same workload "
                             f"({secs:.1f} s, single thread)"}
    subs = {}
    if rank == 0 and world == 1 and args.workload == "x100" and not args.no_subs:
        subs["serve"] = serve_sub(pq, torch, ctx, s, (TD, TM, TF), (D, M, F))
        subs["skew"] = skew_sub(pq, torch, s, hbm)

    line = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": bench_config(args.workload, world),
        "parity": parity,
        "gb_per_s": round(world * plan_bytes * args.steps / (t_ms / 1e3) / 1e9, 1),
        "plan_frac_of_hbm": round(plan_bytes * args.steps / (t_ms / 1e3) / 1e9 / hbm, 4),
        "plan_frac_moved_bytes": round(moved * args.steps / (t_ms / 1e3) / 1e9 / hbm, 4),
        "moved_bytes_per_plan": moved,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "stage_ms": per_stage,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "result": {"ngroups": check["ngroups"], "top_key": check["keys"][:1]},
        "sub_results": subs or None,
    }
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def resident_tables(pq, ctx, host_or_np, stream):
    import torch
    dev = {k: {c: (torch.from_numpy(v) if isinstance(v, np.ndarray) else v).cuda()
               for c, v in t.items()} for k, t in host_or_np.items()}
    TD = pq.pq_load_columns(ctx, [dev["D"]["key"], dev["D"]["seg"]], stream=stream)
    TM = pq.pq_load_columns(ctx, [dev["M"][c] for c in ("key", "dref", "date")], stream=stream)
    TF = pq.pq_load_columns(ctx, [dev["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            stream=stream)
    return TD, TM, TF, dev


def run_serve(args):
    """Batched and served execution of a query stream (serving workload:
    lognormal F sizes, randomised predicates, Poisson arrivals, 32 GB budget)
    against the plain one-query-at-a-time path on the same GPU."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    w = datagen.WORKLOADS["x100"]
    D, M, F = datagen.workload("x100")
    starts = datagen.f_starts(w["seed"], w["n_m"], w["n_f"])
    qs = datagen.query_stream(5, args.queries, w["n_m"], starts, rate_qps=args.rate)
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=32 << 30)
    with torch.cuda.stream(s):
        TD, TM, TF, keep = resident_tables(pq, ctx, {"D": D, "M": M, "F": F}, s)

    def plan(q, flags):
        return pq.make_plan(TD, TM, TF, seg=q["seg"], m_date_lt=q["c"], f_date_gt=q["c"], k=10,
                            rows=dict(m=(q["m_row0"], q["m_rows"]),
                                      f=(q["f_row0"], q["f_rows"])), flags=flags)

    plain_plans = [plan(q, pq.PQ_PLAN_NO_GRAPH) for q in qs]
    serve_plans = [plan(q, 0) for q in qs]
    n = len(qs)
    f_rows = sum(q["f_rows"] for q in qs)
    res_plain = pq.pinned_results(n)
    res_batch = pq.pinned_results(n)

    def plain_closed():
        with torch.cuda.stream(s):
            for i, p in enumerate(plain_plans):
                pq.pq_run_plan(ctx, p, res_plain[i], stream=s)
                ctx.sync(s)      # the plain path waits for every query

    def batched_closed(bs=512):
        with torch.cuda.stream(s):
            for a in range(0, n, bs):
                sub = serve_plans[a:a + bs]
                arr = (pq.pq_plan * len(sub))(*sub)
                dst = pq.ctypes.cast(pq.ctypes.addressof(res_batch) +
                                     a * pq.ctypes.sizeof(pq.pq_result),
                                     pq.ctypes.POINTER(pq.pq_result))
                ctx.check(pq.library().pq_run_batch(ctx.h, arr, len(sub), dst, pq._stream(s)))
            ctx.sync(s)

    def served_closed():
        tickets = [pq.pq_submit(ctx, p) for p in serve_plans]
        out = []
        for t in tickets:
            st, r, lat = pq.pq_poll(ctx, t, timeout_ms=600_000)
            assert st == pq.PQ_OK, st
            out.append(r.as_dict())
        return out

    with torch.cuda.stream(s):          # warm-up: code, caches, resident D-sets
        for p in plain_plans[:args.warmup]:
            pq.pq_run_plan(ctx, p, res_plain[0], stream=s)
            ctx.sync(s)
    batched_closed()
    served_closed()
    t0 = time.perf_counter(); plain_closed(); t_plain = time.perf_counter() - t0
    t0 = time.perf_counter(); batched_closed(); t_batch = time.perf_counter() - t0
    t0 = time.perf_counter(); served = served_closed(); t_serve = time.perf_counter() - t0
    plain = [res_plain[i].as_dict() for i in range(n)]
    batch = [res_batch[i].as_dict() for i in range(n)]
    assert plain == batch == served, "batched / served results differ from the plain path"

    # Open loop: queries arrive on their Poisson schedule.
    arrive = np.array([q["arrive_s"] for q in qs])
    lat_plain = []
    t_start = time.perf_counter()
    with torch.cuda.stream(s):
        for i, p in enumerate(plain_plans):
            now = time.perf_counter() - t_start
            if now < arrive[i]:
                time.sleep(arrive[i] - now)
            pq.pq_run_plan(ctx, p, res_plain[i], stream=s)
            ctx.sync(s)
            lat_plain.append(time.perf_counter() - t_start - arrive[i])
    tickets = [None] * n

    def feeder():
        t_s = time.perf_counter()
        for i, p in enumerate(serve_plans):
            now = time.perf_counter() - t_s
            if now < arrive[i]:
                time.sleep(arrive[i] - now)
            tickets[i] = pq.pq_submit(ctx, p)

    th = threading.Thread(target=feeder)
    th.start()
    lat_serve = []
    for i in range(n):
        while tickets[i] is None:
            time.sleep(1e-4)
        st, r, lat = pq.pq_poll(ctx, tickets[i], timeout_ms=600_000)
        assert st == pq.PQ_OK and r.as_dict() == plain[i]
        lat_serve.append(lat / 1e6)
    th.join()
    pct = lambda a, p: round(1e3 * float(np.percentile(a, p)), 3)

    # The same queries over host-resident tables (pinned host memory, streamed):
    # plain = one query at a time, each streaming its own slices; batched =
    # pq_run_batch, one ingest pass per batch for all its queries (reader
    # combining); served = pq_submit / pq_poll.
    nh = min(n, args.host_queries)
    hctx = pq.Context(arena_bytes=32 << 30)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    HD = pq.pq_load_columns(hctx, [pin(D["key"]), pin(D["seg"])], mode=pq.PQ_STREAMING)
    HM = pq.pq_load_columns(hctx, [pin(M[c]) for c in ("key", "dref", "date")],
                            mode=pq.PQ_STREAMING)
    HF = pq.pq_load_columns(hctx, [pin(F[c]) for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_STREAMING)
    hplans = [pq.make_plan(HD, HM, HF, seg=q["seg"], m_date_lt=q["c"], f_date_gt=q["c"], k=10,
                           rows=dict(m=(q["m_row0"], q["m_rows"]), f=(q["f_row0"], q["f_rows"])))
              for q in qs[:nh]]
    hres_plain = pq.pinned_results(nh)
    hres_batch = pq.pinned_results(nh)
    with torch.cuda.stream(s):
        pq.pq_run_plan(hctx, hplans[0], hres_plain[0], stream=s)     # warm-up
        hctx.sync(s)
        h0 = hctx.stats()["h2d_bytes"]
        t0 = time.perf_counter()
        for i, p in enumerate(hplans):
            pq.pq_run_plan(hctx, p, hres_plain[i], stream=s)
            hctx.sync(s)
        th_plain = time.perf_counter() - t0
        h1 = hctx.stats()["h2d_bytes"]
        t0 = time.perf_counter()
        bs = 256
        for a in range(0, nh, bs):
            sub = hplans[a:a + bs]
            arr = (pq.pq_plan * len(sub))(*sub)
            dst = pq.ctypes.cast(pq.ctypes.addressof(hres_batch) +
                                 a * pq.ctypes.sizeof(pq.pq_result),
                                 pq.ctypes.POINTER(pq.pq_result))
            hctx.check(pq.library().pq_run_batch(hctx.h, arr, len(sub), dst, pq._stream(s)))
        hctx.sync(s)
        th_batch = time.perf_counter() - t0
        h2 = hctx.stats()["h2d_bytes"]
    t0 = time.perf_counter()
    htk = [pq.pq_submit(hctx, p) for p in hplans]
    hserved = []
    for t in htk:
        st, r, lat = pq.pq_poll(hctx, t, timeout_ms=600_000)
        assert st == pq.PQ_OK, st
        hserved.append(r.as_dict())
    th_serve = time.perf_counter() - t0
    assert ([hres_plain[i].as_dict() for i in range(nh)] == plain[:nh] ==
            [hres_batch[i].as_dict() for i in range(nh)] == hserved), "host-resident results differ"
    hctx.close()
    host_line = {
        "queries": nh, "batch_size": bs,
        "closed_loop_qps": {"plain": nh / th_plain, "batched": nh / th_batch,
                            "served": nh / th_serve},
        "speedup_vs_plain": {"batched": th_plain / th_batch, "served": th_plain / th_serve},
        "h2d_gb": {"plain": round((h1 - h0) / 1e9, 2), "batched": round((h2 - h1) / 1e9, 2)},
        "tables": "x100 in pinned host memory, streamed (128 MB chunks)",
        "results_identical": True,
    }

    line = {
        "metric": METRIC, "mode": "serve", "value": n / t_serve, "unit": "queries/s",
        "higher_is_better": True, "n_gpus": 1, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"serving: {n} queries on slices of x100 (F sizes lognormal "
                               "median 500k, sigma 1.5, 10k..30M), randomised seg and date "
                               f"constants, Poisson {args.rate} q/s, 32 GB budget",
                   "f_rows_total": int(f_rows)},
        "closed_loop_qps": {"plain": n / t_plain, "batched": n / t_batch, "served": n / t_serve},
        "speedup_vs_plain": {"batched": t_plain / t_batch, "served": t_plain / t_serve},
        "open_loop_latency_ms": {"rate_qps": args.rate,
                                 "plain": {"p50": pct(lat_plain, 50), "p99": pct(lat_plain, 99)},
                                 "served": {"p50": pct(lat_serve, 50),
                                            "p99": pct(lat_serve, 99)}},
        "results_identical": True,
        "rows_per_s_served": f_rows / t_serve,
        "host_resident": host_line,
    }
    print(json.dumps(line))
    ctx.close()
    return 0


def run_skew(args):
    """The skewed workload at `--scale` of its size (F 200M rows at 1):
    the plain and the partitioned (2^8 buckets) plan, `--steps` timed runs
    each after `--warmup`, and their per-kernel times from a profiled pass."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    w = datagen.WORKLOADS["skew"]
    n_d, n_m, n_f = (int(w[k] * args.scale) for k in ("n_d", "n_m", "n_f"))
    D, M, F = datagen.make(n_d, n_m, n_f, seed=w["seed"], fk="zipf", zipf_s=w["zipf_s"])
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=args.arena_gb << 30)
    with torch.cuda.stream(s):
        TD, TM, TF, keep = resident_tables(pq, ctx, {"D": D, "M": M, "F": F}, s)
    q = query("skew")
    res = pq.pinned_results(1)
    legs = {}
    for name, flags, lp in (("plain", 0, 0), ("partitioned_2^8", pq.PQ_PLAN_PARTITIONED, 8)):
        plan = pq.make_plan(TD, TM, TF, flags=flags | pq.PQ_PLAN_NO_GRAPH, log2P=lp, **q)
        with torch.cuda.stream(s):
            for _ in range(args.warmup):
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
        ms = _events_ms(torch, s, lambda: pq.pq_run_plan(ctx, plan, res[0], stream=s),
                        args.steps)
        ctx.sync(s)
        ctx.profile_enable(True)
        ctx.profile_reset()
        with torch.cuda.stream(s):
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
        ctx.profile_enable(False)
        stages = {}
        for nm in ("plan_dscan", "plan_mscan", "plan_mrank", "plan_mdup", "plan_fscan",
                   "plan_fpart", "plan_fscatter", "plan_fagg", "plan_fprobe", "plan_topk"):
            try:
                t, nl = ctx.profile(nm)
                stages[nm] = round(t / max(nl, 1), 4)
            except pq.PQError:
                pass
        legs[name] = {"ms_per_plan": round(ms, 4), "stage_ms": stages,
                      "result": res[0].as_dict()["ngroups"]}
    print(json.dumps({"metric": METRIC, "mode": "skew", "scale": args.scale,
                      "config": {"workload": f"skew at {args.scale} of F 200M rows",
                                 "rows": {"D": n_d, "M": n_m, "F": n_f}}, "legs": legs}))
    ctx.close()
    return 0


def run_buffering(args):
    """Dynamic buffering of a streamed plan's F hits: the x100 tables in
    pinned host memory streamed in small chunks (--chunk-mb), the query of
    the benchmark (about 0.5 % of F rows join), the probe run after every
    chunk (hit_buffer -1) against hits buffered on the device and probed
    once the buffer could not take another chunk (hit_buffer 16).  CUDA
    events around each plan on its stream; identical results required."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    D, M, F = datagen.workload("x100")
    pin = lambda t, names: [torch.from_numpy(np.ascontiguousarray(t[c])).pin_memory()
                            for c in names]
    host = (pin(D, ("key", "seg")), pin(M, ("key", "dref", "date")),
            pin(F, ("mkey", "price", "disc", "date2")))
    q = query("x100")
    s = torch.cuda.Stream()
    legs, results = {}, []
    for chunk_mb in [int(x) for x in args.chunk_mb.split(",")]:
        for hb in (-1, 16):
            ctx = pq.Context(arena_bytes=16 << 30, chunk_bytes=chunk_mb << 20, ring_slots=6,
                             copy_streams=2, hit_buffer=hb)
            T = [pq.pq_load_columns(ctx, cols, mode=pq.PQ_STREAMING) for cols in host]
            plan = pq.make_plan(*T, **q)
            res = pq.pinned_results(1)
            with torch.cuda.stream(s):
                for _ in range(args.warmup):
                    pq.pq_run_plan(ctx, plan, res[0], stream=s)
                    ctx.sync(s)
                l0 = ctx.stats()["kernel_launches"]
                ms = _events_ms(torch, s, lambda: pq.pq_run_plan(ctx, plan, res[0], stream=s),
                                args.steps)
                ctx.sync(s)
                launches = (ctx.stats()["kernel_launches"] - l0) // args.steps
            results.append(res[0].as_dict())
            legs[f"chunk_{chunk_mb}MB_{'per_chunk' if hb < 0 else 'buffered'}"] = {
                "ms_per_plan": round(ms, 3), "rows_per_s": len(F["mkey"]) / (ms / 1e3),
                "kernel_launches_per_plan": int(launches)}
            ctx.close()
    print(json.dumps({"metric": METRIC, "mode": "buffering", "steps": args.steps,
                      "config": {"workload": "x100 in pinned host memory, streamed",
                                 "query": QUERY_TEXT},
                      "legs": legs,
                      "results_identical": all(r == results[0] for r in results)}))
    return 0


def run_ops(args):
    """Each standalone operator on x100-sized columns, timed with CUDA events
    on its stream (median of args.steps launches after args.warmup), against
    the HBM roofline.  Algorithmic bytes: every input read once and every
    output written once."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    if args.rows:
        w = datagen.WORKLOADS["x100"]
        D, M, F = datagen.make(w["n_d"], max(1, args.rows // 4), args.rows, seed=w["seed"])
    else:
        D, M, F = datagen.workload("x100")
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=16 << 30)
    dev = lambda a: torch.from_numpy(a).cuda()
    date2, mkey, price = dev(F["date2"]), dev(F["mkey"]), dev(F["price"])
    want = lambda name: not args.ops or name in args.ops.split(",")
    m_key = dev(M["key"])
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])

    def timed(fn):
        with torch.cuda.stream(s):
            for _ in range(args.warmup):
                out = fn()
            ctx.sync(s)
            ts = []
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                out = fn()
                b.record(s)
                ts.append((a, b))
            ctx.sync(s)
        return float(np.median([a.elapsed_time(b) for a, b in ts])), out

    rows = []

    def add(name, ms, nbytes, units, note):
        gbs = nbytes / (ms / 1e3) / 1e9
        rows.append({"op": name, "ms": round(ms, 4), "gb_per_s": round(gbs, 1),
                     "frac_hbm": round(gbs / hbm, 3), "units_per_s": units / (ms / 1e3),
                     "bytes": nbytes, "note": note})

    n_f, n_m = len(F["mkey"]), len(M["key"])
    if want("filter"):
        ms, (sel, cnt) = timed(lambda: pq.pq_filter(ctx, date2, ">", 1200, stream=s))
        k = int(cnt.item())
        add("pq_filter", ms, 4 * n_f + 8 * k, n_f,
            f"F.date2 > 1200 over {n_f} int32 rows, {k} ids out")
    for lp in (6, 10) if want("partition") else ():
        ms, _ = timed(lambda: pq.pq_partition(ctx, mkey, [price], log2P=lp, stream=s))
        add(f"pq_partition P={1 << lp}", ms, 2 * 16 * n_f, n_f,
            f"F.mkey + price ({n_f} rows): 16 B in + 16 B out per row")
    if not (want("join") or want("groupby") or want("topk")):
        print(json.dumps({"metric": METRIC, "mode": "ops", "unit": "GB/s", "n_gpus": 1,
                          "steps": args.steps, "warmup": args.warmup, "dtype": "int64",
                          "data": "synthetic", "config": {"rows": n_f, "peak_hbm_gbs": hbm},
                          "ops": rows}))
        ctx.close()
        return 0
    ht_holder = {}

    def build():
        if "ht" in ht_holder:
            ht_holder["ht"].free(s)
        ht_holder["ht"] = pq.pq_join_build(ctx, m_key, None, stream=s)
        return ht_holder["ht"]
    ms, ht = timed(build)
    add("pq_join_build", ms, 8 * n_m, n_m, f"{n_m} int64 M keys, value = row id")
    ms, (r, v, c) = timed(lambda: pq.pq_join_probe(ctx, ht_holder["ht"], mkey, cap=n_f, stream=s))
    hits = int(c.item())
    add("pq_join_probe", ms, 8 * n_f + 16 * hits, n_f, f"{n_f} F.mkey probes, {hits} pairs out")
    ms, (gk, gs, gn) = timed(lambda: pq.pq_groupby_sum(ctx, mkey, price, cap=n_m, stream=s))
    g = int(gn.item())
    add("pq_groupby_sum", ms, 16 * n_f + 16 * g, n_f, f"group {n_f} rows by F.mkey, {g} groups")
    ms, _ = timed(lambda: pq.pq_topk(ctx, gk[:g], gs[:g], 10, stream=s))
    add("pq_topk", ms, 16 * g, g, f"k=10 over {g} groups")
    line = {"metric": METRIC, "mode": "ops", "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["x100"], "peak_hbm_gbs": hbm},
            "ops": rows}
    print(json.dumps(line))
    ctx.close()
    return 0


def measure_h2d(nbytes=1 << 30, reps=5):
    """Host-to-device copy bandwidth from pinned memory (GB/s, best of reps)."""
    import torch
    src = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dst.copy_(src, non_blocking=True)
        b.record()
        b.synchronize()
        best = max(best, nbytes / (a.elapsed_time(b) / 1e3) / 1e9)
    del src, dst
    return best


def run_stream(args):
    """Storage-resident plan: the x2000 tables live in pinned host memory and
    stream through the 128 MiB chunk ring under a 16 GB device budget."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    name = args.workload if args.workload != "x100" else "x2000"
    w = datagen.WORKLOADS[name]
    n_d, n_m, n_f = w["n_d"], w["n_m"], w["n_f"]
    link = measure_h2d()
    host = {}
    for tn, cols, n in (("D", datagen.D_COLS, n_d), ("M", datagen.M_COLS, n_m),
                        ("F", datagen.F_COLS, n_f)):
        host[tn] = {c: torch.empty(n, dtype=getattr(torch, np.dtype(dt).name), pin_memory=True)
                    for c, dt in cols}
    out = {k: {c: t.numpy() for c, t in v.items()} for k, v in host.items()}
    t0 = time.perf_counter()
    D, M, F = datagen.workload(name, out=out)
    t_gen = time.perf_counter() - t0
    q = query(name)
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=16 << 30, chunk_bytes=128 << 20, ring_slots=6, copy_streams=2)
    HD = pq.pq_load_columns(ctx, [host["D"]["key"], host["D"]["seg"]], mode=pq.PQ_STREAMING)
    HM = pq.pq_load_columns(ctx, [host["M"][c] for c in ("key", "dref", "date")],
                            mode=pq.PQ_STREAMING)
    HF = pq.pq_load_columns(ctx, [host["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_STREAMING)
    plan = pq.make_plan(HD, HM, HF, **q)
    res = pq.pinned_results(1)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
        st0 = ctx.stats()
        times = []
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                t0 = time.perf_counter()
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
                ctx.sync(s)
                times.append(time.perf_counter() - t0)
        st1 = ctx.stats()
    got = res[0].as_dict()
    # Sampled check: each reported group's sum recomputed from the rows of F
    # that carry its key (with M's and D's predicates), independently of the GPU.
    keys = np.array(got["keys"], dtype=np.int64)
    sel = np.isin(F["mkey"], keys) & (F["date2"] > q["f_date_gt"]) if name != "skew" else \
        np.isin(F["mkey"], keys)
    rev = F["price"][sel].astype(np.int64) * (100 - F["disc"][sel].astype(np.int64))
    sums = {int(k): 0 for k in keys}
    for k, v in zip(F["mkey"][sel].tolist(), rev.tolist()):
        sums[k] += v
    checked = all(sums[int(k)] == int(sv) for k, sv in zip(got["keys"], got["sums"]))
    t = float(np.median(times))
    bytes_ = (st1["h2d_bytes"] - st0["h2d_bytes"]) / args.steps
    gbps = bytes_ / t / 1e9
    ctx.close()

    # The same tables mapped: the plan kernels read the pinned host columns
    # in place (the D-set and M dictionary still live in the arena).
    ctx = pq.Context(arena_bytes=16 << 30)
    MD = pq.pq_load_columns(ctx, [host["D"]["key"], host["D"]["seg"]], mode=pq.PQ_MAPPED)
    MM = pq.pq_load_columns(ctx, [host["M"][c] for c in ("key", "dref", "date")],
                            mode=pq.PQ_MAPPED)
    MF = pq.pq_load_columns(ctx, [host["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_MAPPED)
    mplan = pq.make_plan(MD, MM, MF, **q)
    mres = pq.pinned_results(1)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pq.pq_run_plan(ctx, mplan, mres[0], stream=s)
            ctx.sync(s)
        mtimes = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pq.pq_run_plan(ctx, mplan, mres[0], stream=s)
            ctx.sync(s)
            mtimes.append(time.perf_counter() - t0)
    mt = float(np.median(mtimes))
    ctx.close()

    # Out of core: the same mapped tables under a device budget too small
    # for the plan's build side; the M side is radix-partitioned by key range
    # and the plan runs in passes (F read over the link once per pass).
    ctx = pq.Context(arena_bytes=int(args.ooc_arena_gb * (1 << 30)))
    OD = pq.pq_load_columns(ctx, [host["D"]["key"], host["D"]["seg"]], mode=pq.PQ_MAPPED)
    OM = pq.pq_load_columns(ctx, [host["M"][c] for c in ("key", "dref", "date")],
                            mode=pq.PQ_MAPPED)
    OF = pq.pq_load_columns(ctx, [host["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_MAPPED)
    oplan = pq.make_plan(OD, OM, OF, **q)
    ores = pq.pinned_results(1)
    with torch.cuda.stream(s):
        pq.pq_run_plan(ctx, oplan, ores[0], stream=s)
        ctx.sync(s)
        p0 = ctx.stats()["out_of_core_passes"]
        otimes = []
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            pq.pq_run_plan(ctx, oplan, ores[0], stream=s)
            ctx.sync(s)
            otimes.append(time.perf_counter() - t0)
        passes = (ctx.stats()["out_of_core_passes"] - p0) // max(1, args.steps)
    ot = float(np.median(otimes))
    out_of_core = {"value": n_f / ot, "unit": "rows/s", "ms_per_step": 1e3 * ot,
                   "arena_gb": args.ooc_arena_gb, "passes": int(passes),
                   "result_matches_streaming": ores[0].as_dict() == res[0].as_dict()}
    ctx.close()

    # The same tables packed (frame of reference + bit packing, made once
    # ahead like files on storage): the ingest ring copies the packed bytes
    # and the device decodes each chunk before its scan.
    t0 = time.perf_counter()
    packed = {tn: {c: pq.pq_pack_column(t) for c, t in cols.items()} for tn, cols in host.items()}
    t_pack = time.perf_counter() - t0
    pk_bytes = sum(p.nbytes for cols in packed.values() for p in cols.values())
    # Chunks of 256 MB of plain rows (about 85 MB packed) on three copy
    # streams: with a third of the bytes per row, the ring needs more rows in
    # flight to keep the link busy (128 MB chunks on two streams: 55.6 ms).
    ctx = pq.Context(arena_bytes=16 << 30, chunk_bytes=256 << 20, ring_slots=6, copy_streams=3)
    PD = pq.pq_load_columns(ctx, [packed["D"]["key"], packed["D"]["seg"]], mode=pq.PQ_STREAMING)
    PM = pq.pq_load_columns(ctx, [packed["M"][c] for c in ("key", "dref", "date")],
                            mode=pq.PQ_STREAMING)
    PF = pq.pq_load_columns(ctx, [packed["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_STREAMING)
    pplan = pq.make_plan(PD, PM, PF, **q)
    pres = pq.pinned_results(1)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pq.pq_run_plan(ctx, pplan, pres[0], stream=s)
            ctx.sync(s)
        pst0 = ctx.stats()
        ptimes = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pq.pq_run_plan(ctx, pplan, pres[0], stream=s)
            ctx.sync(s)
            ptimes.append(time.perf_counter() - t0)
        pst1 = ctx.stats()
    pt = float(np.median(ptimes))
    pbytes = (pst1["h2d_bytes"] - pst0["h2d_bytes"]) / args.steps
    packed_line = {"value": n_f / pt, "unit": "rows/s", "ms_per_step": 1e3 * pt,
                   "h2d_gb_per_step": round(pbytes / 1e9, 3),
                   "gb_per_s": round(pbytes / pt / 1e9, 1),
                   "plain_gb": round(table_bytes(n_d, n_m, n_f) / 1e9, 2),
                   "packed_gb": round(pk_bytes / 1e9, 2), "pack_s": round(t_pack, 1),
                   "chunk_bytes": 256 << 20, "ring_slots": 6, "copy_streams": 3,
                   "result_matches_streaming": pres[0].as_dict() == res[0].as_dict()}
    ctx.close()
    del packed
    mbytes = 5 * n_d + 16 * n_m + 12 * n_f + 17 * int(mres[0].hits)
    mapped = {"value": n_f / mt, "unit": "rows/s", "ms_per_step": 1e3 * mt,
              "link_gb_per_step": round(mbytes / 1e9, 3),
              "link_bytes": "bytes the kernels load from the host columns (upper bound: "
                            "scanned columns in full, probe columns of the joined F rows)",
              "gb_per_s": round(mbytes / mt / 1e9, 1),
              "result_matches_streaming": mres[0].as_dict() == res[0].as_dict()}
    line = {
        "metric": METRIC, "mode": "stream", "value": n_f / t, "unit": "rows/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT.get(name, name), "query": QUERY_TEXT,
                   "source": "pinned host memory (stands in for NVMe)",
                   "chunk_bytes": 128 << 20, "ring_slots": 6, "copy_streams": 2,
                   "arena_gb": 16},
        "h2d_gb_per_step": round(bytes_ / 1e9, 3), "gb_per_s": round(gbps, 1),
        "roofline": {"bound": "host-link", "achieved": round(gbps, 1), "peak": round(link, 1),
                     "unit": "GB/s", "frac": round(gbps / link, 4),
                     "peak_source": "measured here: pinned cudaMemcpyAsync H2D, 1 GiB, best of 5"},
        "arena_high_water_gb": round(st1["arena_high_water"] / 1e9, 2),
        "chunks_per_step": (st1["chunks_ingested"] - st0["chunks_ingested"]) // args.steps,
        "clocks": clk.summary(), "generate_s": round(t_gen, 1),
        "result": {"ngroups": got["ngroups"], "top_keys": got["keys"][:3]},
        "sampled_check": {"groups_checked": len(keys), "sums_match": checked},
        "mapped": mapped,
        "out_of_core": out_of_core,
        "packed": packed_line,
    }
    print(json.dumps(line))
    ok = (checked and mapped["result_matches_streaming"] and
          packed_line["result_matches_streaming"] and out_of_core["result_matches_streaming"])
    return 0 if ok else 1


def run_packed(args):
    """The plan on packed host tables streamed through the ingest ring (the
    end-to-end leg of the plan mode on its own, for profiling): every step
    copies the packed chunks and decodes them on the device."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    name = args.workload
    w = datagen.WORKLOADS[name]
    n_d, n_m, n_f = w["n_d"], w["n_m"], w["n_f"]
    D, M, F = datagen.workload(name)
    q = query(name)
    t0 = time.perf_counter()
    packed = {tn: {c: pq.pq_pack_column(a) for c, a in tab.items()}
              for tn, tab in (("D", D), ("M", M), ("F", F))}
    t_pack = time.perf_counter() - t0
    pk_bytes = sum(p.nbytes for cols in packed.values() for p in cols.values())
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=args.arena_gb << 30, chunk_bytes=256 << 20, ring_slots=6,
                     copy_streams=3)
    PD = pq.pq_load_columns(ctx, [packed["D"]["key"], packed["D"]["seg"]], mode=pq.PQ_STREAMING)
    PM = pq.pq_load_columns(ctx, [packed["M"][c] for c in ("key", "dref", "date")],
                            mode=pq.PQ_STREAMING)
    PF = pq.pq_load_columns(ctx, [packed["F"][c] for c in ("mkey", "price", "disc", "date2")],
                            mode=pq.PQ_STREAMING)
    plan = pq.make_plan(PD, PM, PF, **q)
    res = pq.pinned_results(1)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
        st0 = ctx.stats()
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
            times.append(time.perf_counter() - t0)
        st1 = ctx.stats()
    want = None
    if name in ("small", "x100"):
        import oracle
        want = oracle.run_plan(D, M, F, **q)
    got = res[0].as_dict()
    ok = want is None or (got["keys"] == want["keys"].tolist() and
                          got["sums"] == want["sums"].tolist() and
                          got["ngroups"] == want["ngroups"])
    t = float(np.median(times))
    h2d = (st1["h2d_bytes"] - st0["h2d_bytes"]) / args.steps
    print(json.dumps({
        "metric": METRIC, "mode": "packed", "value": n_f / t, "unit": "rows/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT.get(name, name), "query": QUERY_TEXT,
                   "source": "packed columns in pinned host memory", "chunk_bytes": 256 << 20,
                   "ring_slots": 6, "copy_streams": 3},
        "h2d_bytes_per_step": int(h2d), "packed_bytes": pk_bytes,
        "plain_bytes": table_bytes(n_d, n_m, n_f), "pack_s": round(t_pack, 2),
        "link_gb_per_s": round(h2d / t / 1e9, 1),
        "result_matches_oracle": ok}))
    ctx.close()
    return 0 if ok else 1


def run_aggfirst(args):
    """The aggregate-first plan (F grouped by mkey into a dense array, filtered
    on the group sum, semi-joined with M', top-k) on the resident workload,
    beside the join-first plan on the same tables.  Each step is one
    pq_run_plan, timed with CUDA events on its stream; the inputs (1.5 GB)
    are larger than L2."""
    import torch

    import __graft_entry__
    import datagen
    __graft_entry__.build()
    import paper_2512_02862_gb300 as pq
    torch.cuda.set_device(0)
    name = args.workload
    w = datagen.WORKLOADS[name]
    n_d, n_m, n_f = w["n_d"], w["n_m"], w["n_f"]
    D, M, F = datagen.workload(name)
    q = query(name)
    having = args.having
    s = torch.cuda.Stream()
    ctx = pq.Context(arena_bytes=args.arena_gb << 30)
    with torch.cuda.stream(s):
        TD, TM, TF, keep = resident_tables(pq, ctx, dict(D=D, M=M, F=F), s)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    res = pq.pinned_results(1)

    def timed(plan):
        with torch.cuda.stream(s):
            for _ in range(args.warmup):
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
            ctx.sync(s)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(args.steps):
                pq.pq_run_plan(ctx, plan, res[0], stream=s)
            b.record(s)
            ctx.sync(s)
        return a.elapsed_time(b) / args.steps, dict(res[0].as_dict(), hits=int(res[0].hits))

    ms, got = timed(pq.make_plan(TD, TM, TF, having=having, **q))
    ms_join, _ = timed(pq.make_plan(TD, TM, TF, **q))
    ok, cpu = None, None
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        want = oracle.run_plan_aggfirst(D, M, F, having=having, **q)
        t_cpu = time.perf_counter() - t0
        ok = (got["keys"] == want["keys"].tolist() and got["sums"] == want["sums"].tolist()
              and got["ngroups"] == want["ngroups"] and got["status"] == want["status"])
        cpu = {"value": n_f / t_cpu, "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": f"one run of the whole {name} plan"}
    nbytes = table_bytes(n_d, n_m, n_f)
    gbs = nbytes / (ms / 1e3) / 1e9
    print(json.dumps({
        "metric": METRIC, "mode": "aggfirst", "value": n_f / (ms / 1e3), "unit": "rows/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT.get(name, name),
                   "query": "F.date2 > 1200 grouped by mkey, SUM(price*(100-disc)) > "
                            f"{having}, key in M' (M.date < 1200, dref in D', D.seg == 1), "
                            "top-10", "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(gbs / hbm, 3), "bytes_per_step": nbytes,
                     "peak_source": peak_src, "scope": "whole plan"},
        "join_first_ms": ms_join, "groups": got["ngroups"], "hits": got["hits"],
        "cpu_baseline": cpu, "result_matches_oracle": ok}))
    ctx.close()
    return 0 if ok is not False else 1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # Default steps per mode: plan 2000 (~0.6 s timed, so that the clocks get
    # sampled), reference 20, stream 3, serve and ops 20.
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="plan", choices=["plan", "serve", "stream", "ops", "packed",
                                                        "aggfirst", "skew", "buffering"])
    ap.add_argument("--chunk-mb", default="4,16", help="buffering mode: chunk sizes in MB")
    ap.add_argument("--ops", default="", help="ops mode: comma list of filter, partition, "
                                              "join, groupby, topk (default all)")
    ap.add_argument("--rows", type=int, default=0, help="ops mode: F rows (default x100's)")
    ap.add_argument("--scale", type=float, default=1.0, help="skew mode: fraction of the size")
    ap.add_argument("--ooc-arena-gb", type=float, default=6.0,
                    help="stream mode: device budget of the out-of-core leg")
    ap.add_argument("--workload", default="x100", choices=["small", "x100", "x2000", "skew"])
    ap.add_argument("--arena-gb", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-budget-s", type=float, default=150.0)
    ap.add_argument("--queries", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=500.0)
    ap.add_argument("--host-queries", type=int, default=256)
    ap.add_argument("--having", type=int, default=4_000_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-subs", action="store_true",
                    help="leave out the skew and serving sub-results of the default line")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = (20 if args.impl == "reference" else 3 if args.mode == "stream"
                      else 2000 if args.mode == "plan" else 20)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "stream":
        return run_stream(args)
    if args.mode == "ops":
        return run_ops(args)
    if args.mode == "packed":
        return run_packed(args)
    if args.mode == "aggfirst":
        return run_aggfirst(args)
    if args.mode == "skew":
        return run_skew(args)
    if args.mode == "buffering":
        return run_buffering(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
