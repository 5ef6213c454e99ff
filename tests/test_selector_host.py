"""Host-side logic of the learned selector (no GPU): the seeded query grid, the
resumable timing sweep, the train / held-out split and the parameter layout."""
import json

import numpy as np
import pytest

from paper_2312_00720_gb300 import build, selector


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_grid_is_seeded_and_within_its_ranges():
    a, b = selector.grid(4096, seed=5), selector.grid(4096, seed=5)
    assert a == b and selector.grid(300, seed=6) != a[:300]
    for p in a:
        assert 2**16 <= p["ns"] <= 2**27 and 16 <= p["nr"] <= p["ns"]
        assert p["key_bytes"] in (4, 8)
        assert 1 <= p["ncols_r"] + p["ncols_s"] <= 8 and 0 <= p["ncols_r"] - p["ncols_s"] <= 1
        assert 0.0 <= p["theta"] <= 1.25 and 0.1 <= p["mr"] <= 1.0 and 4 <= p["groups"] <= p["ns"]
    # the grid spans the workload space: both ends of every range are reached
    ls = np.log2([p["ns"] for p in a])
    lg = np.log2([p["groups"] for p in a])
    assert ls.min() < 16.1 and ls.max() > 26.9 and lg.min() < 2.1 and lg.max() > 25.0
    assert {p["ncols_r"] + p["ncols_s"] for p in a} == set(range(1, 9))


def test_sweep_resumes_after_the_last_completed_point(tmp_path, monkeypatch):
    timed = []

    def fake_measure(p, reps=3):
        timed.append(p["id"])
        return {v: float(p["id"] + k + 1) for k, v in enumerate(selector.ALL_VARIANTS)}

    monkeypatch.setattr(selector, "measure", fake_measure)
    path = str(tmp_path / "sweep.jsonl")
    pts = selector.grid(7, seed=1)
    first = selector.sweep(path, pts[:4])
    assert timed == [0, 1, 2, 3] and [r["point"]["id"] for r in first] == [0, 1, 2, 3]
    with open(path, "a") as f:
        f.write('{"point": {"id": 5}, "truncated')   # a line cut off by a killed sweep
    f_before = open(path).read()
    recs = selector.sweep(path, pts)
    assert timed == [0, 1, 2, 3, 4, 5, 6]           # only the missing points were timed
    assert [r["point"]["id"] for r in recs] == list(range(7))
    assert open(path).read().startswith(f_before)
    assert selector.sweep(path, pts) == recs and len(timed) == 7   # nothing left to time
    for r in recs:
        assert len(r["features"]) == 12 and r["features"][1] == pytest.approx(np.log2(r["point"]["ns"] + 1), rel=1e-6)
    x, y = selector._arrays(recs)
    assert x.shape == (7, 12) and y.shape == (7, 11) and y[2, 0] == pytest.approx(np.log(3.0))


def test_split_is_a_seeded_partition():
    recs = [{"i": i} for i in range(50)]
    tr, te = selector.split(recs, 0.8, seed=3)
    assert len(tr) == 40 and len(te) == 10
    assert sorted(r["i"] for r in tr + te) == list(range(50))
    assert selector.split(recs, 0.8, seed=3) == (tr, te)


def test_initial_parameters_follow_the_network_layout():
    from oracle import mlp
    th = selector.init_params(seed=0).astype(np.float64)
    assert th.size == mlp.N_PARAMS
    p = mlp.unpack(th)
    for b in ("b1", "b2", "b3"):
        assert np.all(p[b] == 0.0)
    for w, fan_in in (("w1", 12), ("w2", 64), ("w3", 64)):
        assert abs(p[w].std() - np.sqrt(2.0 / fan_in)) < 0.25 * np.sqrt(2.0 / fan_in)


def _network_preferring(join_idx: int, gb_idx: int):
    # all weights zero, output biases alone: y = b3, so the argmins are fixed
    from oracle import mlp
    th = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(th)
    b3 = np.ones(mlp.D_OUT)
    b3[join_idx] = -1.0
    b3[5 + gb_idx] = -1.0
    return mlp.pack({**p, "b3": b3}).astype(np.float32)


@pytest.mark.parametrize("join_idx", [0, 1, 2])
def test_fused_call_resolves_auto_like_the_join_under_the_network(join_idx):
    from paper_2312_00720_gb300 import gj
    gj.selector_set(_network_preferring(join_idx, 2), np.zeros(12), np.ones(12))
    try:
        for shape in ((1 << 20, 1 << 22, 4, 1, 1, 2, 0.0, 1.0, 1024), (1 << 12, 1 << 16, 8, 2, 2, 4, 1.0, 0.1, 16)):
            j_plain, g_plain = gj.auto_variants(*shape, selector=1)
            j_fused, _ = gj.auto_variants(*shape, selector=1, fused=True)
            assert j_plain == j_fused == 1 + join_idx     # PHJ-TR, PHJ-UR, NPHJ
            assert g_plain == 3                            # PGB
            # an explicit variant is never overridden
            assert gj.auto_variants(*shape, selector=1, fused=True, join="nphj")[0] == 3
    finally:
        gj.selector_set(None, None, None)


def test_fused_call_follows_the_paper_rule_without_a_network():
    from paper_2312_00720_gb300 import gj
    gj.selector_set(None, None, None)
    for mr, z, kb in ((1.0, 0.0, 4), (0.1, 0.0, 4), (0.1, 0.7, 4), (0.1, 0.0, 8)):
        shape = (1 << 16, 1 << 18, kb, 2, 2, 2, z, mr, 64)
        rule = gj.heuristic_choose(*shape)
        for sel in (0, 1):   # the MLP mode without a network falls back to the rules
            assert gj.auto_variants(*shape, selector=sel)[0] == rule[0]
            assert gj.auto_variants(*shape, selector=sel, fused=True)[0] == rule[0]
