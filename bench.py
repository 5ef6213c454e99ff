"""Benchmark: FK-PK plain join at scale through the C-ABI (gj_join, PHJ-TR / GFTR).

Workload: |R| = 2^25 unique int32 keys (a seeded permutation), |S| = 2^27 foreign
keys drawn uniformly from R's keys (match ratio 1), 4 int32 payload columns per
side, all materialised: T has 2^27 rows of 36 bytes. Metric: input tuples per
second, (|R| + |S|) / time (the paper's join throughput, Sec. 5.1.2), in
Gtuples/s. Inputs (3.4 GB) and output (4.8 GB) are far larger than the 129 MB L2,
so no flush is needed between steps.

`--impl reference` times the CPU oracle on a bounded sample of the same workload.
Under torchrun every rank runs an independent replica (the path has no exchange
step on one GPU); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NR, NS, NCOLS = 1 << 25, 1 << 27, 4
METRIC = "join input tuples/s ((|R|+|S|)/time), plain FK-PK join at scale"
ROW_BYTES = 4 + 4 * NCOLS              # key + payloads of one input row
OUT_ROW_BYTES = 4 + 4 * 2 * NCOLS      # T(key, r1..r4, s1..s4)
MIN_BYTES = (NR + NS) * ROW_BYTES + NS * OUT_ROW_BYTES
WORKLOAD = (f"plain FK-PK join, |R|=2^25 unique int32 keys, |S|=2^27 uniform FK (theta=0), match ratio 1.0, "
            f"{NCOLS} int32 payloads per side materialised (GFTR partitioned hash join)")
SEED = 2023


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_digest() -> str:
    h = hashlib.sha256()
    for name in ("radix.cu", "join.cu", "gj_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2312_00720_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_digest") != kernel_source_digest():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock samples taken while the timed region runs."""

    def __init__(self, device: int):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                rows.append(f)
        load = [r for r in rows if r[7].replace(".", "").isdigit() and float(r[7]) > 50] or rows
        sm = [float(r[0]) for r in load if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i in range(4) if r[3 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(load)}


def cpu_baseline(sample_shift: int = 2):
    """The oracle (single-threaded C++) on 1/2^sample_shift of the workload."""
    import oracle
    from paper_2312_00720_gb300 import workloads as wl

    nr, ns = NR >> sample_shift, NS >> sample_shift
    w = wl.join_workload(nr, ns, NCOLS, NCOLS, seed=SEED)
    oracle.build()
    t0 = time.perf_counter()
    t = oracle.join(w["rkey"], w["rcols"], w["skey"], w["scols"])
    dt = time.perf_counter() - t0
    assert len(t) == ns
    return {"value": (nr + ns) / dt / 1e9, "unit": "Gtuples/s", "cores": 1, "kind": "oracle",
            "sample": f"|R|=2^{25 - sample_shift}, |S|=2^{27 - sample_shift} of the same workload "
                      f"(same generator), single-threaded std::unordered_map join incl. materialisation, "
                      f"{dt:.1f} s"}


def _event_ms(fn, steps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def oracle_sample(fn, rows: int, what: str):
    """Times one call of an oracle function (single-threaded, this process) on a
    bounded sample; returns the cpu_baseline object of a line."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    fn(oracle)
    dt = time.perf_counter() - t0
    return {"value": rows / dt / 1e9, "unit": "Gtuples/s", "cores": 1, "kind": "oracle",
            "sample": f"{what}, {dt:.1f} s"}


GB_VARIANTS = ("hgb", "sgb", "pgb", "sgb_ur", "pgb_ur", "sgb_de")


def groupby_alg_bytes(kind: str, variant: str, n: int, k: int, d: int, launches: int) -> float:
    """Algorithmic bytes one call moves in the kernels of `kind` (n rows, k-byte
    keys, three 4-byte value columns, d groups of 10 int64 aggregates):
    radix passes read and write key + what travels with it (values for TR, a
    4-byte tuple id for UR, 4-byte codes + values for SGB-DE); histograms and
    bounds read the key; a group-id, aggregation or reduction pass reads key and
    values and writes each group once."""
    vals, out = 12, k + 80
    moved = {"sgb": k + vals, "pgb": k + vals, "sgb_ur": k + 4, "pgb_ur": k + 4, "sgb_de": 4 + vals}.get(variant, k)
    if kind == "radix_scatter":
        return launches * 2.0 * n * moved
    if kind == "radix_hist":   # key range (SGB), tile histograms (per pass); the offset scans are not counted
        return launches / 2.0 * n * (4 if variant == "sgb_de" else k)
    if kind == "partition_bounds":
        return n * k
    if kind == "hgb_group_id":  # dictionary pass (+ the code pass of SGB-DE)
        return n * k * (2 if variant == "sgb_de" else 1) + (4 * n if variant == "sgb_de" else 0)
    if kind in ("hgb_aggregate", "pgb", "sgb_reduce"):
        key = 4 if variant == "sgb_de" else k
        return n * (key + vals) + d * out + (n * key if kind == "sgb_reduce" else 0)
    if kind == "agg_init":
        return d * 80
    return 0.0


def bench_groupby(gj, wl, peak, steps: int = 5, cpu: bool = True):
    """Plain grouped aggregation over every cell of the workload: n = 2^27 rows,
    int32 or int64 keys over 2^4, 2^12, 2^20 or 2^26 ids, uniform or Zipf 1.0, three
    int32 value columns in [-2^20, 2^20), COUNT + SUM/MIN/MAX per column (10 int64
    aggregates); every variant, with the cell's cardinality as the groups hint."""
    import torch
    n = 1 << 27
    aggs = ["count"] + ["sum", "min", "max"] * 3
    cols = [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    cells = []
    for lg in (4, 12, 20, 26):
        for kdt in (np.int32, np.int64):
            for theta in (0.0, 1.0):
                w = wl.groupby_workload(n, 1 << lg, nvals=3, key_dtype=kdt, theta=theta, seed=77)
                k = np.dtype(kdt).itemsize
                key = torch.from_numpy(w["key"]).cuda()
                vals = [torch.from_numpy(v).cuda() for v in w["vals"]]
                distinct = int(torch.unique(key).numel())
                min_bytes = n * (k + 12) + distinct * (k + 80)
                cell = {"ids": f"2^{lg}", "key_bytes": k, "zipf": theta, "groups": distinct, "min_bytes": min_bytes}
                for v in GB_VARIANTS:
                    call = lambda: gj.groupby(key, vals, aggs, cols, variant=v, sync=False, groups_hint=1 << lg)
                    _, _, ng = gj.groupby(key, vals, aggs, cols, variant=v, sync=True, groups_hint=1 << lg)
                    assert int(ng.item()) == distinct
                    ms = _event_ms(call, steps)
                    gj.profile_read()
                    gj.profile_enable(True)
                    call()
                    prof = gj.profile_read()
                    gj.profile_enable(False)
                    dom = max(prof, key=lambda q: prof[q][0])
                    dms, dl = prof[dom]
                    ab = groupby_alg_bytes(dom, v, n, k, distinct, dl)
                    ach = ab / (dms * 1e-3) / 1e9
                    cell[v] = {"ms": ms, "gtuples_s": n / (ms * 1e-3) / 1e9,
                               "min_bytes_frac": min_bytes / (ms * 1e-3) / 1e9 / peak,
                               "roofline": {"bound": "hbm", "kernel": dom, "launches": dl, "achieved": ach,
                                            "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                                            "alg_bytes_per_launch": ab / dl},
                               "kernels_ms": {q: round(t, 4) for q, (t, c) in prof.items()}}
                cells.append(cell)
                del key, vals
    out = {"workload": "n=2^27, keys int32/int64 over 2^4/2^12/2^20/2^26 ids, uniform or Zipf 1.0, 3 int32 values, "
                       "COUNT+SUM/MIN/MAX per column (10 int64 aggregates), groups hint = ids",
           "cells": cells}
    if cpu:
        m = 1 << 24  # the first 2^24 rows of the 2^20-id uniform int32 input
        w = wl.groupby_workload(n, 1 << 20, nvals=3, seed=77)
        out["cpu_baseline"] = oracle_sample(
            lambda o: o.groupby_hash(w["key"][:m], [c[:m] for c in w["vals"]], aggs, cols), m,
            "first 2^24 rows of the 2^20-id uniform int32 input, std::unordered_map group-by, 10 aggregates")
    return out


def bench_gather(gj, steps: int = 10):
    """The paper's gather calibration (Sec. 4.1.1, Table gather-profile) on this
    GPU: gather 2^27 4-byte elements through a clustered map (the identity) and
    an unclustered one (a seeded random permutation). Both read the map and write
    the output sequentially (8 bytes per element at B_G); the input costs 4 bytes
    at B_G when clustered and at B_R when not, so with r = t_unclustered /
    t_clustered, B_G / B_R = 3 r - 2 (the paper's A100 figure: r = 8.52, 24)."""
    import torch
    n = 1 << 27
    src = torch.randint(-(2**31), 2**31 - 1, (n,), dtype=torch.int32, device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(3))
    ident = torch.arange(n, dtype=torch.int32, device="cuda")
    perm = torch.randperm(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(4)).to(torch.int32)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    tc = _event_ms(lambda: gj.gather(src, ident, sync=False, out=out), steps)
    tu = _event_ms(lambda: gj.gather(src, perm, sync=False, out=out), steps)
    assert gj.device_status() == 0
    r = tu / tc
    return {"workload": "gather of 2^27 int32 elements, identity vs random permutation map",
            "clustered_ms": tc, "unclustered_ms": tu, "ratio": r, "bg_over_br": 3 * r - 2,
            "clustered_gb_s": 12 * n / (tc * 1e-3) / 1e9}


def bench_selector(gj, n_sample: int = 64):
    """Variant selection on held-out queries, timed live: the first n_sample of the
    819 held-out points of the 4096-point grid (grid(4096, seed=2025), the seeded
    80/20 split the shipped network was trained on), every join and group-by
    variant timed (median of 3), and the regret of the shipped network, the cost
    model and the paper's rules against the best of the 5 x 6 pairs."""
    import numpy as np

    from paper_2312_00720_gb300 import selector as sel
    pts = sel.grid(4096, seed=2025)
    _, held = sel.split(pts, 0.8, seed=1)
    sample = held[:n_sample]
    t0 = time.perf_counter()
    recs = [{"point": p, "features": sel.features(p).tolist(), "ms": sel.measure(p, reps=3)} for p in sample]
    z = np.load(sel.TRAINED)
    ev = sel.evaluate(recs, z["theta"], z["mean"], z["std"])
    return {"workload": f"first {len(sample)} of the {len(held)} held-out points of grid(4096, seed=2025), "
                        "11 variants timed live per point",
            "n_points": ev["n"], "network": "selector_gb300.npz (trained on the other 3277 points)",
            **{k: v for k, v in ev.items() if k != "n"}, "seconds": time.perf_counter() - t0}


def bench_one_query(gj, wl, steps: int = 20, cpu: bool = True, peak: float = 6796.5):
    """One query: |R| = 2^20 ⋈ |S| = 2^22, GROUP BY R.pay mod 1024, SUM/COUNT(S.pay), not materialised."""
    import torch
    w = wl.join_groupby_workload()
    d = lambda a: torch.from_numpy(a).cuda()
    rk, rc, sk, sc = d(w["rkey"]), [d(w["rcols"][0])], d(w["skey"]), [d(w["scols"][0])]
    out = {"workload": "|R|=2^20, |S|=2^22, GROUP BY R.pay mod 1024, SUM/COUNT(S.pay); inputs 40 MB (L2-resident)"}
    for v in ("nphj", "phj_tr"):
        args = (rk, rc, sk, sc, (0, 0, 1024), ["sum", "count"], [(1, 0, 0), (1, 0, 0)])
        okeys, outs, ng = gj.join_groupby(*args, variant=v, sync=True)
        assert int(outs[1][: int(ng.item())].sum().item()) == 1 << 22
        ms = _event_ms(lambda: gj.join_groupby(*args, variant=v, sync=False), steps)
        # minimal bytes: R (key + pay) and S (key + pay) read once, 1024 groups x 20 B written
        min_bytes = ((1 << 20) + (1 << 22)) * 8 + 1024 * 20
        out[v] = {"us": ms * 1e3, "gtuples_s": ((1 << 20) + (1 << 22)) / (ms * 1e-3) / 1e9,
                  "min_bytes_frac": min_bytes / (ms * 1e-3) / 1e9 / peak}
    if cpu:
        out["cpu_baseline"] = oracle_sample(
            lambda o: o.join_groupby(w["rkey"], w["rcols"], w["skey"], w["scols"], g_side=0, g_col=0, g_mod=1024,
                                     aggs=["sum", "count"], agg_side=[1, 1], agg_col=[0, 0]),
            (1 << 20) + (1 << 22), "the whole query, std::unordered_map join then group-by")
    return out


def bench_many_to_many(gj, wl, steps: int = 5, peak: float = 6796.5):
    """Many-to-many join (Sec. 5.1.9): |R| = |S| = 2^26, keys uniform from 2^25 keys,
    two int32 payloads per side; every (r, s) pair materialised (about 2^27 rows)."""
    import torch
    n, nk = 1 << 26, 1 << 25
    w = wl.mn_join_workload(n, n, nk, 2, 2, seed=17)
    d = lambda a: torch.from_numpy(a).cuda()
    rk, rc, sk, sc = d(w["rkey"]), [d(c) for c in w["rcols"]], d(w["skey"]), [d(c) for c in w["scols"]]
    cap = int(1.05 * n * n / nk)
    tkey = torch.empty(cap, dtype=torch.int32, device="cuda")
    tcols = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(4)]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = {"workload": "|R| = |S| = 2^26, keys uniform from 2^25 distinct keys, 2 int32 payloads per side; "
                       "nphj_mn: global table with key chains, phj_mn: GFTR partitions with a partition-"
                       "clustered table"}
    for v in ("nphj_mn", "phj_mn"):
        step = lambda: gj.join(rk, rc, sk, sc, variant=v, capacity=cap, sync=False, out=(tkey, tcols), count=cnt)
        step()
        torch.cuda.synchronize()
        assert gj.device_status() == 0
        m = int(cnt.item())
        ms = _event_ms(step, steps)
        out["output_rows"] = m
        out[v] = {"ms": ms, "gtuples_s": 2 * n / (ms * 1e-3) / 1e9, "output_gb_s": m * 20 / (ms * 1e-3) / 1e9,
                  # minimal bytes: both inputs (key + 2 payloads) read once, every output row written once
                  "min_bytes_frac": (2 * n * 12 + m * 20) / (ms * 1e-3) / 1e9 / peak}
    return out


def _seq_variants(gj, ws):
    """How many of the instances each join variant runs under the paper's rules."""
    inv = {v: k for k, v in gj.JOIN.items()}
    out = {}
    for w in ws:
        j, _ = gj.auto_variants(len(w["rkey"]), len(w["skey"]), 4, 2, 2, 4, -1.0, -1.0, 0, selector="heuristic",
                                fused=True)
        out[inv[j]] = out.get(inv[j], 0) + 1
    return out


def bench_batch(gj, wl, steps: int = 5, cpu: bool = True, peak: float = 6796.5):
    """512 join + group-by instances: the batched plan with each query's variant chosen
    by the trained network (the cost model if the package ships none) vs 512 sequential
    gj_join_groupby calls whose AUTO follows the paper's rules."""
    import torch
    from paper_2312_00720_gb300 import selector as sel
    ws = wl.batch_workload(512, seed=7)
    d = lambda a: torch.from_numpy(a).cuda()
    aggs = ["count", "sum", "sum", "sum"]
    refs = [(1, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)]
    qs = [(d(w["rkey"]), [d(c) for c in w["rcols"]], d(w["skey"]), [d(c) for c in w["scols"]],
           (0, 0, w["modulus"]), aggs, refs) for w in ws]
    learned = sel.install_trained()
    t0 = time.perf_counter()
    plan = gj.BatchPlan(qs, selector="mlp" if learned else "cost")
    tune_s = time.perf_counter() - t0
    gj.selector_set(None, None, None)
    inv = {v: k for k, v in gj.JOIN.items()}
    batched_variants = {}
    for v in plan.variants():
        batched_variants[inv[v]] = batched_variants.get(inv[v], 0) + 1
    batched = _event_ms(plan.launch, steps)
    res = plan.results()
    assert gj.device_status() == 0
    assert all(int(r[1][0].sum()) == len(w["skey"]) for r, w in zip(res, ws))

    def sequential():
        for q in qs:
            gj.join_groupby(*q, variant="auto", selector="heuristic", sync=False, capacity=2 * q[4][2] - 1)

    seq = _event_ms(sequential, max(1, steps // 2))
    rows = sum(len(w["rkey"]) + len(w["skey"]) for w in ws)
    cfg = plan.config()
    plan.close()
    out = {}
    if cpu:
        sub = ws[:64]  # the first 64 instances
        out["cpu_baseline"] = oracle_sample(
            lambda o: [o.join_groupby(w["rkey"], w["rcols"], w["skey"], w["scols"], g_side=0, g_col=0,
                                      g_mod=w["modulus"], aggs=aggs, agg_side=[1, 1, 1, 0], agg_col=[0, 0, 1, 1])
                       for w in sub],
            sum(len(w["rkey"]) + len(w["skey"]) for w in sub),
            "the first 64 of the 512 instances, std::unordered_map join then group-by each")
    return {**out, "workload": "512 instances, |R| log-uniform [2^10, 2^20], |S| = 4|R|, 2 int32 payloads per side, "
                        "GROUP BY R.p0 mod G (G log-uniform [2^2, 2^16]), COUNT, SUM(S.p0), SUM(S.p1), SUM(R.p1)",
            "rows": rows, "batched_ms": batched, "sequential_ms": seq, "speedup": seq / batched,
            "batched_gtuples_s": rows / (batched * 1e-3) / 1e9, "sequential_gtuples_s": rows / (seq * 1e-3) / 1e9,
            # minimal bytes: every input row (key + 2 payloads) read once
            "batched_min_bytes_frac": rows * 12 / (batched * 1e-3) / 1e9 / peak,
            "tuned_config": {"build_rows": cfg[0], "probe_rows": cfg[1], "lookahead": cfg[2], "blocks_per_sm": cfg[3]},
            "batched_selector": "trained network (selector_gb300.npz)" if learned else "cost model",
            "batched_variants": batched_variants,
            "sequential_selector": "the paper's rules (Sec. 7)",
            "sequential_variants": _seq_variants(gj, ws),
            "tune_and_capture_s": tune_s}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("GJ_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time: every rank joins one MAX all-reduce (NCCL on the
    GPU, gloo on the host)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gtuples(rows_per_rank: int, ms: float, world: int) -> float:
    """Whole-job throughput: every rank processes rows_per_rank rows per step
    (weak scaling); ms is the slowest rank's time per step."""
    return world * rows_per_rank / (ms * 1e-3) / 1e9


def run_reference(args, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_2312_00720_gb300 import workloads as wl

    # each step joins a sample small enough that all steps end within about two and
    # a half minutes (the oracle runs at roughly 1.5 M tuples/s on one core)
    budget_rows = 150.0 / max(1, args.steps) * 1.5e6
    shift = 3
    while shift < 12 and (NR + NS) >> shift > budget_rows:
        shift += 1
    nr, ns = NR >> shift, NS >> shift
    w = wl.join_workload(nr, ns, NCOLS, NCOLS, seed=SEED)
    oracle.build()
    for _ in range(args.warmup if args.warmup <= 1 else 1):
        oracle.join(w["rkey"][:1024], [c[:1024] for c in w["rcols"]], w["skey"][:4096],
                    [c[:4096] for c in w["scols"]])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.join(w["rkey"], w["rcols"], w["skey"], w["scols"])
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = args.steps * (nr + ns) / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "Gtuples/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"each step joins |R|=2^{25 - shift}, |S|=2^{27 - shift}"},
        "cpu_baseline": {"value": value, "unit": "Gtuples/s", "cores": 1, "kind": "oracle",
                         "sample": f"|R|=2^{25 - shift}, |S|=2^{27 - shift} per step"},
        "e2e": {"value": value, "unit": "Gtuples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def groupby_case(spec: str):
    """One call per listed group-by variant, synchronised, on seeded input: n =
    2^LOG2N int32 keys over 2^LOG2G ids, three int32 values, COUNT + SUM/MIN/MAX
    per column, 2^LOG2G as the groups hint (as the benchmark's cells run it).
    Prints one JSON line; no timing (run under a profiler)."""
    import torch

    from paper_2312_00720_gb300 import gj
    from paper_2312_00720_gb300 import workloads as wl

    parts = spec.split(",")
    lgn, lgg, variants = int(parts[0]), int(parts[1]), parts[2:]
    gj.load()
    w = wl.groupby_workload(1 << lgn, 1 << lgg, nvals=3, seed=77)
    key = torch.from_numpy(w["key"]).cuda()
    vals = [torch.from_numpy(v).cuda() for v in w["vals"]]
    aggs = ["count"] + ["sum", "min", "max"] * 3
    cols = [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    groups = {}
    for v in variants:
        _, _, ng = gj.groupby(key, vals, aggs, cols, variant=v, sync=True, groups_hint=1 << lgg)
        groups[v] = int(ng.item())
    torch.cuda.synchronize()
    if gj.device_status() != 0:
        raise RuntimeError("device error in the group-by case")
    print(json.dumps({"groupby_case": {"n": 1 << lgn, "ids": 1 << lgg, "groups": groups}}))


def kernel_families():
    """One launch of each kernel family on small cases (inputs larger than L2, a few
    GB on the device at most), synchronised, for profiler captures; no timing.
    Joins |R| = 2^22, |S| = 2^24 with 4 + 4 int32 payloads (PHJ-TR, PHJ-UR, NPHJ,
    SMJ-TR); NPHJ-MN on 2^22 x 2^22 rows over 2^21 keys; the one-query fused
    join -> group-by (NPHJ and PHJ-TR plans); group-by of 2^24 rows with 10
    aggregates (HGB over 2^4 and 2^12 ids, PGB over 2^4 (sliced partitions) and 2^20,
    SGB over 2^20); a 64-instance batch;
    one selector training step (loss + gradient, Adam)."""
    import numpy as np
    import torch

    from paper_2312_00720_gb300 import gj, selector
    from paper_2312_00720_gb300 import workloads as wl

    gj.load()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    w = wl.join_workload(1 << 22, 1 << 24, 4, 4, seed=1)
    rk, rc, sk, sc = d(w["rkey"]), [d(c) for c in w["rcols"]], d(w["skey"]), [d(c) for c in w["scols"]]
    for v in ("phj_tr", "phj_ur", "nphj", "smj_tr"):
        gj.join(rk, rc, sk, sc, variant=v)
    del rk, rc, sk, sc
    wm = wl.mn_join_workload(1 << 22, 1 << 22, 1 << 21, 2, 2, seed=2)
    gj.join(d(wm["rkey"]), [d(c) for c in wm["rcols"]], d(wm["skey"]), [d(c) for c in wm["scols"]],
            variant="nphj_mn", capacity=int(1.1 * (1 << 23)))
    wq = wl.join_groupby_workload()
    qargs = (d(wq["rkey"]), [d(wq["rcols"][0])], d(wq["skey"]), [d(wq["scols"][0])], (0, 0, 1024),
             ["sum", "count"], [(1, 0, 0), (1, 0, 0)])
    for v in ("nphj", "phj_tr"):
        gj.join_groupby(*qargs, variant=v)
    aggs = ["count"] + ["sum", "min", "max"] * 3
    cols = [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    for lg, v in ((4, "hgb"), (4, "pgb"), (12, "hgb"), (20, "pgb"), (20, "sgb")):
        g = wl.groupby_workload(1 << 24, 1 << lg, nvals=3, seed=7)
        gj.groupby(d(g["key"]), [d(x) for x in g["vals"]], aggs, cols, variant=v, groups_hint=1 << lg)
    ws = wl.batch_workload(64, seed=7)
    qs = [(d(b["rkey"]), [d(c) for c in b["rcols"]], d(b["skey"]), [d(c) for c in b["scols"]], (0, 0, b["modulus"]),
           ["count", "sum", "sum", "sum"], [(1, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)]) for b in ws]
    plan = gj.BatchPlan(qs, config=(8192, 8192, 4, 3))
    plan.launch()
    torch.cuda.synchronize()
    plan.close()
    th = torch.from_numpy(selector.init_params(0)).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    x = torch.randn(512, 12, device="cuda", generator=gen)
    t = torch.randn(512, 11, device="cuda", generator=gen)
    loss, grad = gj.mlp_loss_grad(th, x, t, torch.ones(512, 11, device="cuda"))
    gj.mlp_adam_step(th, grad, torch.zeros_like(th), torch.zeros_like(th), 1, lr=1e-3)
    torch.cuda.synchronize()
    if gj.device_status() != 0:
        raise RuntimeError("device error in the kernel families")
    print(json.dumps({"kernel_families": "done"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="phj_tr", choices=["phj_tr", "phj_ur", "nphj", "smj_tr", "smj_ur"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the group-by, one-query and batched lines")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--scale", type=int, default=0, help="divide |R| and |S| by 2^scale (profiling captures only)")
    ap.add_argument("--groupby-case", default=None, metavar="LOG2N,LOG2G,VARIANT[,VARIANT..]",
                    help="run each group-by variant once on 2^LOG2N rows over 2^LOG2G ids and exit "
                         "(the small case the group-by kernel captures are taken on)")
    ap.add_argument("--kernel-families", action="store_true",
                    help="run one launch of each kernel family on small cases and exit (profiler captures)")
    args = ap.parse_args()
    if args.groupby_case:
        groupby_case(args.groupby_case)
        return
    if args.kernel_families:
        kernel_families()
        return
    global NR, NS, MIN_BYTES
    NR, NS = NR >> args.scale, NS >> args.scale
    MIN_BYTES = (NR + NS) * ROW_BYTES + NS * OUT_ROW_BYTES
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    from paper_2312_00720_gb300 import gj
    from paper_2312_00720_gb300 import workloads as wl

    torch.cuda.set_device(local)
    gj.load()
    w = wl.join_workload(NR, NS, NCOLS, NCOLS, seed=SEED)
    dev = lambda a: torch.from_numpy(a).cuda()
    rkey, skey = dev(w["rkey"]), dev(w["skey"])
    rcols, scols = [dev(c) for c in w["rcols"]], [dev(c) for c in w["scols"]]
    tkey = torch.empty(NS, dtype=torch.int32, device="cuda")
    tcols = [torch.empty(NS, dtype=torch.int32, device="cuda") for _ in range(2 * NCOLS)]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    step = lambda: gj.join(rkey, rcols, skey, scols, variant=args.variant, sync=False, out=(tkey, tcols), count=cnt)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(torch.cuda.current_device())
    time.sleep(0.5)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    assert gj.device_status() == 0
    assert int(cnt.item()) == NS, "join count differs from |S| x match ratio"
    barrier()
    torch.cuda.synchronize()
    launches0 = gj.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    launches = gj.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(ms, world)
    assert gj.device_status() == 0
    ms_step = ms / args.steps
    value = whole_job_gtuples(NR + NS, ms_step, world)

    # ---- per-kernel times on the launching stream (CUDA events around each launch)
    gj.profile_enable(True)
    for _ in range(args.steps):
        step()
    prof = gj.profile_read()
    gj.profile_enable(False)
    # partition passes per side, from the scatter launches (one per pass and side)
    passes = prof.get("radix_scatter", (0.0, 2 * args.steps))[1] / (2 * args.steps)
    alg_bytes_per_step = {
        # every pass over R and over S reads and writes key + payloads
        "radix_scatter": passes * 2 * (NR + NS) * ROW_BYTES,
        # per pass, one read of every key for the tile histograms (the per-digit
        # scans of the tile counts are not counted)
        "radix_hist": passes * 4 * (NR + NS),
        # read S' and R' once, write T
        "phj_probe": (NR + NS) * ROW_BYTES + NS * OUT_ROW_BYTES,
        "partition_bounds": 4 * NR,
        # L2-sized partitions: read the build keys and write the tables once (two
        # 8-byte slots per build row, rounded up per partition; counted as 2)
        "nphj_build": 4 * NR + 2 * 8 * NR,
    }
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    per_launch_bytes = alg_bytes_per_step.get(dom, 0) * args.steps / dom_launches
    per_launch_s = dom_ms / dom_launches * 1e-3
    peak, peak_src = load_peaks()
    achieved = per_launch_bytes / per_launch_s / 1e9
    total_ms = sum(v[0] for v in prof.values())
    kernel_split = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                        "share": v[0] / total_ms} for k, v in prof.items()}

    # ---- end to end: pinned host inputs in, result rows out, every step. Steps are
    # pipelined the way a streaming caller would run them: step i's input copies
    # (one copy stream) and step i-1's result copies (another) overlap step i's
    # join, through two sets of device input and output buffers; every step still
    # copies all its inputs in and all its result rows out inside the timed region.
    h_in = [torch.from_numpy(a).pin_memory() for a in [w["rkey"], *w["rcols"], w["skey"], *w["scols"]]]
    h_out = [torch.empty(NS, dtype=torch.int32).pin_memory() for _ in range(1 + 2 * NCOLS)]
    h_cnt = torch.empty(1, dtype=torch.int64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in h_out) + 8
    d_in = [[rkey, *rcols, skey, *scols], [torch.empty_like(t) for t in (rkey, *rcols, skey, *scols)]]
    d_out = [(tkey, tcols, cnt), (torch.empty_like(tkey), [torch.empty_like(c) for c in tcols],
                                  torch.zeros_like(cnt))]
    comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]     # inputs of buffer b copied
    ev_comp = [torch.cuda.Event(), torch.cuda.Event()]   # join on buffer b done
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]    # results of buffer b copied out
    for b in range(2):
        ev_comp[b].record(comp)
        ev_out[b].record(comp)

    def e2e_step(i):
        b = i & 1
        di, (ok, oc, ocnt) = d_in[b], d_out[b]
        with torch.cuda.stream(s_in):
            s_in.wait_event(ev_comp[b])  # the join two steps back has read buffer b
            for h, d in zip(h_in, di):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(s_in)
        comp.wait_event(ev_in[b])
        comp.wait_event(ev_out[b])  # the results two steps back have left buffer b
        gj.join(di[0], di[1:1 + NCOLS], di[1 + NCOLS], di[2 + NCOLS:], variant=args.variant, sync=False,
                out=(ok, oc), count=ocnt)
        ev_comp[b].record(comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[b])
            for h, d in zip(h_out, [ok, *oc]):
                h.copy_(d, non_blocking=True)
            h_cnt.copy_(ocnt, non_blocking=True)
            ev_out[b].record(s_out)

    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize()
    barrier()
    e0.record(comp)
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    for i in range(args.e2e_steps):
        e2e_step(i)
    comp.wait_stream(s_in)
    comp.wait_stream(s_out)
    e1.record(comp)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world)
    assert int(h_cnt.item()) == NS
    e2e_value = whole_job_gtuples(NR + NS, e2e_ms, world)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value, "unit": "Gtuples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "variant": args.variant.upper().replace("_", "-"),
                       "l2": "inputs 3.4 GB and output 4.8 GB exceed the 129 MB L2; no flush",
                       "parallelism": f"{world} independent replica(s)", "seed": SEED},
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "Gtuples/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_source": f"{peak_src} hbm_gbs", "unit": "GB/s", "frac": achieved / peak,
                         "traffic": ncu_traffic(dom),
                         "alg_bytes_per_launch": per_launch_bytes},
            # whole step against the minimal bytes (read R and S once, write T once)
            "min_bytes_roofline": {
                "bytes_per_step": MIN_BYTES,
                "frac": MIN_BYTES / (ms_step * 1e-3) / 1e9 / peak},
            "kernels": kernel_split,
        }
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline()
        if not args.no_extras and world == 1:
            # the other hot-path rows, measured live on the same GPU
            del h_in, h_out
            cpu = not args.no_cpu_baseline
            out["groupby"] = bench_groupby(gj, wl, peak, cpu=cpu)
            out["one_query"] = bench_one_query(gj, wl, cpu=cpu, peak=peak)
            out["batched"] = bench_batch(gj, wl, cpu=cpu, peak=peak)
            out["many_to_many"] = bench_many_to_many(gj, wl, peak=peak)
            out["gather_calibration"] = bench_gather(gj)
            out["selector"] = bench_selector(gj)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
