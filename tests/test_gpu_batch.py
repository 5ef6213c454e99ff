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


def test_batch_runs_each_query_with_its_chosen_variant(gj):
    """Queries outside the persistent kernel's limits (int64 keys, a modulus above
    2^20) and queries whose chosen variant is partitioned run one at a time after
    it; every query still equals the oracle, on two launches."""
    ws = [wl.join_workload(3000, 12000, 2, 2, seed=11),
          wl.join_workload(3000, 12000, 2, 2, key_dtype=np.int64, seed=12),
          wl.join_workload(200_000, 800_000, 2, 2, seed=13),
          wl.join_workload(5000, 20000, 2, 2, mr=0.5, seed=14)]
    for w, m in zip(ws, [64, 1000, 1 << 21, 7]):
        w["modulus"] = m
    plan = gj.BatchPlan(make_queries(ws), selector="cost")
    v = plan.variants()
    assert v[0] == v[3] == 3 and v[1] in (1, 2, 3) and v[2] in (1, 2, 3)
    for _ in range(2):
        plan.launch()
    got = plan.results()
    assert gj.device_status() == 0
    for w, (keys, aggs, g) in zip(ws, got):
        assert np.array_equal(as_rows(keys, aggs), expected(w))
    plan.close()


@pytest.mark.parametrize("variant", ["phj_tr", "phj_ur"])
def test_batch_with_an_explicit_partitioned_variant_runs_every_query_alone(gj, small_batch, variant):
    qs = small_batch[:12]
    plan = gj.BatchPlan(make_queries(qs), variant=variant)
    assert plan.variants() == [gj.JOIN[variant]] * len(qs)
    plan.launch()
    got = plan.results()
    assert gj.device_status() == 0
    for w, (keys, aggs, g) in zip(qs, got):
        assert np.array_equal(as_rows(keys, aggs), expected(w))
    plan.close()


def test_batch_follows_an_installed_network(gj, small_batch):
    """A network preferring PHJ-UR for every query sends every query through the
    one-query path; removed again, the default choice is the persistent kernel's
    non-partitioned join for these small instances."""
    from oracle import mlp
    p = mlp.unpack(np.zeros(gj.MLP_PARAMS))
    b3 = np.ones(mlp.D_OUT)
    b3[1] = -1.0          # y1: PHJ-UR
    gj.selector_set(mlp.pack({**p, "b3": b3}).astype(np.float32), np.zeros(12), np.ones(12))
    try:
        plan = gj.BatchPlan(make_queries(small_batch[:6]), selector="mlp")
        assert plan.variants() == [2] * 6
        plan.launch()
        for w, (keys, aggs, g) in zip(small_batch[:6], plan.results()):
            assert np.array_equal(as_rows(keys, aggs), expected(w))
        plan.close()
    finally:
        gj.selector_set(None, None, None)
    plan = gj.BatchPlan(make_queries(small_batch[:6]), selector="cost")
    assert plan.variants() == [3] * 6
    plan.close()
