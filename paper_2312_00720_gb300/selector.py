"""Learned variant selector: timing sweep, training and regret evaluation.

The network (12 features -> 64 -> 64 -> 11) predicts the log run time of the five
join variants (PHJ-TR, PHJ-UR, NPHJ, SMJ-TR, SMJ-UR) and the six group-by variants
(HGB, SGB, PGB, SGB-UR, PGB-UR, SGB-DE) of a query; the selector takes the argmin
within each family. Training data are timings the library itself produces on a
seeded grid of synthetic queries; training runs on the GPU through the library's
own forward, backward and Adam kernels (gj_mlp_*). The paper's rules
(gj_heuristic_choose) are the fallback and the comparison point; exhaustive
timing of every variant is the yardstick (regret).

Inputs of the sweep are generated on the device with torch's random generators:
they only need the workload's shape (sizes, key width, skew, match ratio, group
cardinality), and the timings are never compared against the oracle.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import gj

JOIN_VARIANTS = ["phj_tr", "phj_ur", "nphj", "smj_tr", "smj_ur"]
GB_VARIANTS = ["hgb", "sgb", "pgb", "sgb_ur", "pgb_ur", "sgb_de"]
ALL_VARIANTS = JOIN_VARIANTS + GB_VARIANTS
GB_AGGS = ["count", "sum", "min", "max"]
GB_COLS = [0, 0, 0, 0]


def grid(n_points: int, seed: int = 12345, log_s=(16.0, 27.0), log_g=(2.0, 26.0)):
    """Seeded query shapes, uniform in log space over the workload space of the
    selector: |S| rows in 2^log_s, |R| = |S| / 2^U[0, 4] (at least 16), 4- or
    8-byte keys, 1-8 payload columns in all (the result holds at most eight, so
    R carries ceil(p/2) and S floor(p/2)), Zipf factor in [0, 1.25], match ratio
    in [0.1, 1], group cardinality 2^log_g capped at |S|; the group-by runs over
    |S| rows."""
    rng = np.random.default_rng(seed)
    pts = []
    for i in range(n_points):
        ls = rng.uniform(*log_s)
        lr = ls + rng.uniform(-4.0, 0.0)
        ns, nr = int(2 ** ls), max(16, int(2 ** lr))
        lg = min(rng.uniform(*log_g), ls)
        ncols = int(rng.integers(1, 9))
        pts.append({"id": i, "nr": nr, "ns": ns, "key_bytes": int(rng.choice([4, 8])),
                    "ncols_r": (ncols + 1) // 2, "ncols_s": ncols // 2, "theta": float(rng.uniform(0.0, 1.25)),
                    "mr": float(rng.uniform(0.1, 1.0)), "groups": max(4, int(2 ** lg))})
    return pts


def _zipf_ranks(m, n, theta, gen):
    if theta == 0.0:
        return torch.randint(0, n, (m,), device="cuda", generator=gen)
    w = torch.arange(1, n + 1, device="cuda", dtype=torch.float64).pow(-theta)
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    u = torch.rand(m, device="cuda", dtype=torch.float64, generator=gen)
    return torch.searchsorted(cdf, u).clamp_(max=n - 1)


def make_inputs(p, seed: int = 0):
    """Device tensors for one grid point: join inputs and a group-by input of |S| rows."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed * 1000003 + p["id"])
    nr, ns = p["nr"], p["ns"]
    rkey = torch.randperm(nr, device="cuda", generator=gen)
    skey = rkey[_zipf_ranks(ns, nr, p["theta"], gen)]
    miss = torch.rand(ns, device="cuda", generator=gen) >= p["mr"]
    skey = torch.where(miss, nr + torch.randint(0, 2**30, (ns,), device="cuda", generator=gen), skey)
    if p["key_bytes"] == 8:
        k = 0x9E3779B97F4A7C15 - (1 << 64)  # odd constant: a bijection on 64-bit words
        rkey, skey = rkey.to(torch.int64) * k, skey.to(torch.int64) * k
    else:
        rkey, skey = rkey.to(torch.int32), skey.to(torch.int32)
    col = lambda n: torch.randint(0, 2**31 - 1, (n,), device="cuda", dtype=torch.int32, generator=gen)
    rcols = [col(nr) for _ in range(p["ncols_r"])]
    scols = [col(ns) for _ in range(p["ncols_s"])]
    gk = _zipf_ranks(ns, p["groups"], p["theta"], gen)
    gkey = gk.to(torch.int64) * (0x9E3779B97F4A7C15 - (1 << 64)) if p["key_bytes"] == 8 else gk.to(torch.int32)
    gval = [torch.randint(-(2**20), 2**20, (ns,), device="cuda", dtype=torch.int32, generator=gen)]
    return rkey, rcols, skey, scols, gkey, gval


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _shape(p):
    return (p["nr"], p["ns"], p["key_bytes"], p["ncols_r"], p["ncols_s"], len(GB_AGGS), p["theta"], p["mr"],
            p["groups"])


def features(p) -> np.ndarray:
    return gj.query_features(*_shape(p))


def measure(p, reps: int = 3) -> dict:
    """Median milliseconds of every join and group-by variant on grid point p (the
    group-by with the point's cardinality as its groups hint, as AUTO runs it)."""
    rkey, rcols, skey, scols, gkey, gval = make_inputs(p)
    ms = {}
    out_k = torch.empty(p["ns"], dtype=rkey.dtype, device="cuda")
    out_c = [torch.empty(p["ns"], dtype=torch.int32, device="cuda") for _ in range(p["ncols_r"] + p["ncols_s"])]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for v in JOIN_VARIANTS:
        ms[v] = _time(lambda: gj.join(rkey, rcols, skey, scols, variant=v, sync=False, out=(out_k, out_c),
                                      count=cnt), reps)
    for v in GB_VARIANTS:
        ms[v] = _time(lambda: gj.groupby(gkey, gval, GB_AGGS, GB_COLS, variant=v, sync=False,
                                         groups_hint=p["groups"]), reps)
    if gj.device_status() != 0:
        raise RuntimeError(f"device error while timing point {p['id']}")
    return ms


def sweep(path: str, points, reps: int = 3, log=None) -> list:
    """Times every point not yet in `path` (JSON lines) and appends it: a killed
    sweep resumes from the last completed point."""
    done = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                try:
                    r = json.loads(line)
                    done[r["point"]["id"]] = r
                except (ValueError, KeyError):
                    continue
    with open(path, "a+") as f:
        # a sweep killed mid-write leaves a partial last line: start on a fresh one
        if f.tell() > 0:
            f.seek(f.tell() - 1)
            if f.read(1) != "\n":
                f.write("\n")
        for p in points:
            if p["id"] in done:
                continue
            r = {"point": p, "features": features(p).tolist(), "ms": measure(p, reps)}
            f.write(json.dumps(r) + "\n")
            f.flush()
            done[p["id"]] = r
            if log:
                log(r)
    return [done[p["id"]] for p in points if p["id"] in done]


def split(records, frac: float = 0.8, seed: int = 0):
    """Seeded train / held-out split."""
    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(records))
    k = int(round(frac * len(records)))
    return [records[i] for i in idx[:k]], [records[i] for i in idx[k:]]


def _arrays(records):
    x = np.array([r["features"] for r in records], dtype=np.float64)
    y = np.array([[math.log(max(r["ms"][v], 1e-4)) for v in ALL_VARIANTS] for r in records], dtype=np.float64)
    return x, y


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 11)):
        parts.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == gj.MLP_PARAMS
    return th


def train(records, steps: int = 3000, lr: float = 3e-3, seed: int = 0):
    """Adam on the GPU with the library's kernels. Returns (theta, mean, std, losses)."""
    x, y = _arrays(records)
    mean = x.mean(0)
    std = x.std(0)
    std[std < 1e-6] = 1.0
    xd = torch.from_numpy(((x - mean) / std).astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    md = torch.ones_like(yd)
    th = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    losses = []
    for step in range(1, steps + 1):
        loss, grad = gj.mlp_loss_grad(th, xd, yd, md)
        gj.mlp_adam_step(th, grad, m, v, step, lr=lr)
        if step == 1 or step % 100 == 0:
            losses.append(float(loss.item()))
    return th.cpu().numpy(), mean.astype(np.float32), std.astype(np.float32), losses


def evaluate(records, theta, mean, std) -> dict:
    """Regret of the network, of the paper's rules and of the GB300 cost model on
    `records`: per query, (t_selected - t_best) / t_best on the combined join +
    group-by time, t_best over all 5 x 6 variant pairs."""
    x, _ = _arrays(records)
    xd = torch.from_numpy(((x - mean) / std).astype(np.float32)).cuda()
    jv, gv = gj.mlp_select(torch.from_numpy(np.asarray(theta, np.float32)).cuda(), xd)
    jv, gv = jv.cpu().numpy(), gv.cpu().numpy()
    jname = {gj.JOIN[v]: v for v in JOIN_VARIANTS}
    gname = {gj.GROUPBY[v]: v for v in GB_VARIANTS}
    reg_m, reg_h, reg_c = [], [], []
    for r, a, b in zip(records, jv, gv):
        best = min(r["ms"][v] for v in JOIN_VARIANTS) + min(r["ms"][v] for v in GB_VARIANTS)
        reg_m.append((r["ms"][jname[int(a)]] + r["ms"][gname[int(b)]]) / best - 1.0)
        hj, hg = gj.heuristic_choose(*_shape(r["point"]))
        reg_h.append((r["ms"][jname[hj]] + r["ms"][gname[hg]]) / best - 1.0)
        cj, cg = gj.auto_variants(*_shape(r["point"]), selector="cost", ops=GB_AGGS)
        reg_c.append((r["ms"][jname[cj]] + r["ms"][gname[cg]]) / best - 1.0)
    reg_m, reg_h, reg_c = np.array(reg_m), np.array(reg_h), np.array(reg_c)
    return {"n": len(records), "mlp_mean_regret": float(reg_m.mean()), "mlp_p90_regret": float(np.quantile(reg_m, 0.9)),
            "heuristic_mean_regret": float(reg_h.mean()),
            "heuristic_p90_regret": float(np.quantile(reg_h, 0.9)),
            "cost_model_mean_regret": float(reg_c.mean()),
            "cost_model_p90_regret": float(np.quantile(reg_c, 0.9))}


def summarize(records) -> dict:
    """Per-variant win counts and the spread of the timings of a sweep."""
    wins_j = {v: 0 for v in JOIN_VARIANTS}
    wins_g = {v: 0 for v in GB_VARIANTS}
    for r in records:
        wins_j[min(JOIN_VARIANTS, key=lambda v: r["ms"][v])] += 1
        wins_g[min(GB_VARIANTS, key=lambda v: r["ms"][v])] += 1
    ms = np.array([[r["ms"][v] for v in ALL_VARIANTS] for r in records])
    return {"points": len(records), "join_wins": wins_j, "groupby_wins": wins_g,
            "median_ms": {v: float(np.median(ms[:, i])) for i, v in enumerate(ALL_VARIANTS)}}


def main(argv=None):
    """python -m paper_2312_00720_gb300.selector --sweep PATH [--points N]: time
    the grid into PATH (resumable); --evaluate PATH: train on 80 % of PATH's
    points and print the held-out regrets as one JSON line."""
    import argparse
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweep", metavar="PATH")
    ap.add_argument("--evaluate", metavar="PATH")
    ap.add_argument("--points", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=2025)
    ap.add_argument("--budget-s", type=float, default=0.0, help="stop sweeping after this many seconds (0 = none)")
    ap.add_argument("--save", metavar="NPZ", help="with --evaluate: write the trained network (theta, mean, std)")
    args = ap.parse_args(argv)
    gj.load()
    if args.sweep:
        pts = grid(args.points, seed=args.seed)
        t0 = time.time()

        def log(r):
            # every record is on disk before this runs: stopping here loses nothing
            if args.budget_s > 0 and time.time() - t0 > args.budget_s:
                raise TimeoutError
        try:
            sweep(args.sweep, pts, reps=3, log=log)
        except TimeoutError:
            pass
        with open(args.sweep) as f:
            n_done = sum(1 for line in f if line.strip().endswith("}"))
        print(json.dumps({"swept": args.sweep, "points_done": n_done, "of": len(pts),
                          "seconds": round(time.time() - t0, 1)}))
    if args.evaluate:
        recs = []
        with open(args.evaluate) as f:
            for line in f:
                try:
                    recs.append(json.loads(line))
                except ValueError:
                    pass
        train_r, held = split(recs, 0.8, seed=1)
        theta, mean, std, losses = train(train_r, steps=6000)
        ev = evaluate(held, theta, mean, std)
        if args.save:
            np.savez(args.save, theta=np.asarray(theta, np.float32), mean=np.asarray(mean, np.float64),
                     std=np.asarray(std, np.float64))
        print(json.dumps({"evaluation": ev, "train_points": len(train_r), "loss_first_last": [losses[0], losses[-1]],
                          "summary": summarize(recs)}))


# The network trained on 80 % of the 4096-point GB300 sweep (grid(4096, seed=2025)),
# shipped with the package: install_trained() makes it the GJ_SELECT_MLP selector.
TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_gb300.npz")


def install_trained(path: str = TRAINED) -> bool:
    """Install the shipped network (gj_selector_set); False if the file is absent."""
    if not os.path.exists(path):
        return False
    z = np.load(path)
    gj.selector_set(z["theta"], z["mean"], z["std"])
    return True


if __name__ == "__main__":
    main()
