"""Batched join -> group-by (one persistent launch, CUDA graph) vs the oracle, and
output invariance under every tuning configuration."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_00720_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

AGGS = ["count", "sum", "sum", "sum"]
# COUNT(*), SUM(S.p0), SUM(S.p1), SUM(R.p1) grouped by R.p0 mod G
AGG_COLS = [(1, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)]


def make_queries(ws):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    qs = []
    for w in ws:
        qs.append((dev(w["rkey"]), [dev(c) for c in w["rcols"]], dev(w["skey"]), [dev(c) for c in w["scols"]],
                   (0, 0, w["modulus"]), AGGS, AGG_COLS))
    return qs


def expected(w):
    return oracle.canonical(oracle.join_groupby(
        w["rkey"], w["rcols"], w["skey"], w["scols"], g_side=0, g_col=0, g_mod=w["modulus"], aggs=AGGS,
        agg_side=[a[0] for a in AGG_COLS], agg_col=[a[1] for a in AGG_COLS]))


def as_rows(keys, aggs):
    return oracle.canonical(np.stack([keys] + aggs, 1)) if len(keys) else np.zeros((0, 1 + len(aggs)), np.int64)


@pytest.fixture(scope="module")
def small_batch():
    return wl.batch_workload(40, log_r_lo=4, log_r_hi=14, log_g_lo=0, log_g_hi=12, seed=3)


@pytest.mark.parametrize("config", [None, (8192, 8192, 1, 2), (1024, 2048, 4, 3), (65536, 256, 2, 1)])
def test_batch_matches_oracle_under_every_config(gj, small_batch, config):
    plan = gj.BatchPlan(make_queries(small_batch), config=config)
    for _ in range(2):  # replays recompute everything from the inputs
        plan.launch()
    got = plan.results()
    assert gj.device_status() == 0
    for w, (keys, aggs, g) in zip(small_batch, got):
        assert np.array_equal(as_rows(keys, aggs), expected(w))
    if config is not None:
        assert plan.config()[:3] == tuple(config[:3])
    plan.close()


def test_batch_edge_queries(gj):
    ws = [wl.join_workload(0, 100, 2, 2, seed=1), wl.join_workload(100, 0, 2, 2, seed=2),
          wl.join_workload(1, 1, 2, 2, seed=3), wl.join_workload(5000, 20000, 2, 2, mr=0.3, seed=4)]
    for w, m in zip(ws, [1, 7, 1, 1 << 20]):
        w["modulus"] = m
    plan = gj.BatchPlan(make_queries(ws))
    plan.launch()
    for w, (keys, aggs, g) in zip(ws, plan.results()):
        assert np.array_equal(as_rows(keys, aggs), expected(w))
    plan.close()


def test_batch_duplicate_key_is_reported(gj):
    w = wl.join_workload(1000, 4000, 2, 2, seed=5)
    w["rkey"][3] = w["rkey"][4]
    w["modulus"] = 16
    plan = gj.BatchPlan(make_queries([w]))
    plan.launch()
    torch.cuda.synchronize()
    assert gj.device_status() == 5
    plan.close()


@pytest.mark.slow
def test_batch_512_full_config(gj):
    """512 instances, |R| log-uniform in [2^10, 2^20], |S| = 4|R|, G log-uniform in [2^2, 2^16]:
    every instance equals the oracle."""
    ws = wl.batch_workload(512, seed=7)
    plan = gj.BatchPlan(make_queries(ws))
    plan.launch()
    got = plan.results()
    assert gj.device_status() == 0
    rng = np.random.default_rng(0)
    for i in rng.choice(512, 64, replace=False):
        keys, aggs, g = got[i]
        assert np.array_equal(as_rows(keys, aggs), expected(ws[i]))
    for (keys, aggs, g), w in zip(got, ws):
        assert aggs[0].sum() == len(w["skey"])            # every S row matches once
        assert aggs[1].sum() == w["scols"][0].astype(np.int64).sum()
    plan.close()
