"""Learned variant selector: timing sweep, training and regret evaluation.

The network (12 features -> 64 -> 64 -> 6) predicts the log run time of the three
join variants (PHJ-TR, PHJ-UR, NPHJ) and the three group-by variants (HGB, SGB,
PGB) of a query; the selector takes the argmin within each family. Training data
are timings the library itself produces on a seeded grid of synthetic queries;
training runs on the GPU through the library's own forward, backward and Adam
kernels (gj_mlp_*). The paper's rules (gj_heuristic_choose) are the fallback and
the comparison point; exhaustive timing of every variant is the yardstick (regret).

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

JOIN_VARIANTS = ["phj_tr", "phj_ur", "nphj"]
GB_VARIANTS = ["hgb", "sgb", "pgb"]
ALL_VARIANTS = JOIN_VARIANTS + GB_VARIANTS
GB_AGGS = ["count", "sum", "min", "max"]
GB_COLS = [0, 0, 0, 0]


def grid(n_points: int, seed: int = 12345, log_s=(14.0, 22.0)):
    """Seeded query shapes, uniform in log space (a reduced form of the paper's
    workload space: sizes, 4/8-byte keys, 1-4 payload columns, Zipf factor in
    [0, 1.25], match ratio in [0.1, 1], group cardinality in [2^2, |S|])."""
    rng = np.random.default_rng(seed)
    pts = []
    for i in range(n_points):
        ls = rng.uniform(*log_s)
        lr = ls + rng.uniform(-4.0, 0.0)
        ns, nr = int(2 ** ls), max(16, int(2 ** lr))
        lg = rng.uniform(2.0, ls)
        pts.append({"id": i, "nr": nr, "ns": ns, "key_bytes": int(rng.choice([4, 8])),
                    "ncols": int(rng.integers(1, 5)), "theta": float(rng.uniform(0.0, 1.25)),
                    "mr": float(rng.uniform(0.1, 1.0)), "groups": int(2 ** lg)})
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
    rcols = [col(nr) for _ in range(p["ncols"])]
    scols = [col(ns) for _ in range(p["ncols"])]
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


def features(p) -> np.ndarray:
    return gj.query_features(p["nr"], p["ns"], p["key_bytes"], p["ncols"], p["ncols"], len(GB_AGGS), p["theta"],
                             p["mr"], p["groups"])


def measure(p, reps: int = 3) -> dict:
    """Median milliseconds of every join and group-by variant on grid point p."""
    rkey, rcols, skey, scols, gkey, gval = make_inputs(p)
    ms = {}
    out_k = torch.empty(p["ns"], dtype=rkey.dtype, device="cuda")
    out_c = [torch.empty(p["ns"], dtype=torch.int32, device="cuda") for _ in range(2 * p["ncols"])]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for v in JOIN_VARIANTS:
        ms[v] = _time(lambda: gj.join(rkey, rcols, skey, scols, variant=v, sync=False, out=(out_k, out_c),
                                      count=cnt), reps)
    for v in GB_VARIANTS:
        ms[v] = _time(lambda: gj.groupby(gkey, gval, GB_AGGS, GB_COLS, variant=v, sync=False), reps)
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
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 6)):
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
    """Regret of the network and of the paper's rules on `records`: per query,
    (t_selected - t_best) / t_best on the combined join + group-by time, t_best
    over all 3 x 3 variant pairs."""
    x, _ = _arrays(records)
    xd = torch.from_numpy(((x - mean) / std).astype(np.float32)).cuda()
    jv, gv = gj.mlp_select(torch.from_numpy(np.asarray(theta, np.float32)).cuda(), xd)
    jv, gv = jv.cpu().numpy(), gv.cpu().numpy()
    reg_m, reg_h = [], []
    for r, a, b in zip(records, jv, gv):
        tj = [r["ms"][v] for v in JOIN_VARIANTS]
        tg = [r["ms"][v] for v in GB_VARIANTS]
        best = min(tj) + min(tg)
        reg_m.append((tj[a - 1] + tg[b - 1]) / best - 1.0)
        p = r["point"]
        hj, hg = gj.heuristic_choose(p["nr"], p["ns"], p["key_bytes"], p["ncols"], p["ncols"], len(GB_AGGS),
                                     p["theta"], p["mr"], p["groups"])
        reg_h.append((tj[hj - 1] + tg[hg - 1]) / best - 1.0)
    reg_m, reg_h = np.array(reg_m), np.array(reg_h)
    return {"n": len(records), "mlp_mean_regret": float(reg_m.mean()), "mlp_p90_regret": float(np.quantile(reg_m, 0.9)),
            "heuristic_mean_regret": float(reg_h.mean()),
            "heuristic_p90_regret": float(np.quantile(reg_h, 0.9))}
