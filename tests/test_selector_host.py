"""Host-side logic of variant selection (no GPU): the learned selector's seeded
query grid, resumable timing sweep, train / held-out split and parameter layout;
how AUTO resolves under each selector; and the GB300 cost model's choices."""
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


def test_fused_call_follows_the_paper_rule_under_the_heuristic_selector():
    from paper_2312_00720_gb300 import gj
    gj.selector_set(None, None, None)
    for mr, z, kb in ((1.0, 0.0, 4), (0.1, 0.0, 4), (0.1, 0.7, 4), (0.1, 0.0, 8)):
        shape = (1 << 16, 1 << 18, kb, 2, 2, 2, z, mr, 64)
        rule = gj.heuristic_choose(*shape)
        assert gj.auto_variants(*shape, selector="heuristic")[0] == rule[0]
        assert gj.auto_variants(*shape, selector="heuristic", fused=True)[0] == rule[0]


JOIN_ORDER = [1, 2, 3, 5, 6]   # PHJ-TR, PHJ-UR, NPHJ, SMJ-TR, SMJ-UR


@pytest.mark.parametrize("sel", ["cost", "mlp"])   # the MLP mode without a network takes the cost model
def test_auto_takes_the_cost_models_argmin(sel):
    from paper_2312_00720_gb300 import gj
    gj.selector_set(None, None, None)
    rng = np.random.default_rng(4)
    for _ in range(60):
        ns = int(2 ** rng.uniform(12, 28))
        nr = max(1, ns >> int(rng.integers(0, 5)))
        shape = (nr, ns, int(rng.choice([4, 8])), int(rng.integers(1, 5)), int(rng.integers(1, 5)), 4,
                 float(rng.uniform(0, 1.3)), float(rng.uniform(0.05, 1)), int(2 ** rng.uniform(1, 26)))
        ops = ["count", "sum", "min", "max"]
        jc, gc = gj.cost_estimate(*shape, ops=ops)
        j, g = gj.auto_variants(*shape, selector=sel, ops=ops)
        assert j == JOIN_ORDER[int(np.argmin(jc))]
        assert g == 1 + int(np.argmin(gc))
        jf, _ = gj.auto_variants(*shape, selector=sel, ops=ops, fused=True)
        assert jf == JOIN_ORDER[int(np.argmin(jc[:3]))]   # the fused call runs PHJ-TR, PHJ-UR, NPHJ


def test_default_selector_is_the_cost_model():
    from paper_2312_00720_gb300 import gj
    o = gj.options()
    assert o.selector == gj.SELECT["cost"]


def test_cost_model_picks_the_regimes_the_models_predict():
    from paper_2312_00720_gb300 import gj
    ops = ["count", "sum", "min", "max"]
    J = lambda *a: JOIN_ORDER[int(np.argmin(gj.cost_estimate(*a, ops=ops)[0]))]
    G = lambda *a: 1 + int(np.argmin(gj.cost_estimate(*a, ops=ops)[1]))
    # a build side whose global table fits in L2: the non-partitioned join
    assert J(1 << 14, 1 << 18, 4, 2, 2, 4, 0.0, 1.0, 64) == 3
    # a build side far beyond L2 with every row matching: the GFTR partitioned join
    assert J(1 << 26, 1 << 27, 4, 2, 2, 4, 0.0, 1.0, 64) == 1
    # few groups: the hash group-by aggregates in shared memory
    assert G(1 << 20, 1 << 24, 4, 1, 1, 4, 0.0, 1.0, 16) == 1
    # many groups under heavy skew: the hottest PGB partition dominates, a sort-based variant wins
    assert G(1 << 20, 1 << 26, 4, 1, 1, 4, 1.25, 1.0, 1 << 22) in (2, 4, 6)
    # the same groups without skew: the partition-based group-by
    assert G(1 << 20, 1 << 26, 4, 1, 1, 4, 0.0, 1.0, 1 << 22) == 3


def test_cost_model_gftr_gains_with_the_match_ratio_and_the_random_access_penalty():
    """M3's reading (Sec. 4.1.4): GFUR's unclustered gathers scale with the matches
    and with B_G / B_R, GFTR's extra partitioning does not; so Cost(PHJ-UR) -
    Cost(PHJ-TR) rises with the match ratio, and the break-even match ratio falls
    as B_G / B_R grows."""
    from paper_2312_00720_gb300 import gj

    def gap(mr):
        jc, _ = gj.cost_estimate(1 << 28, 1 << 28, 4, 3, 3, 1, 0.0, mr, 64)
        return jc[1] - jc[0]

    def break_even():
        lo, hi = 0.0, 1.0
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if gap(mid) < 0 else (lo, mid)
        return hi

    try:
        gaps = [gap(m) for m in np.linspace(0.02, 1.0, 25)]
        assert all(b > a for a, b in zip(gaps, gaps[1:]))
        be = []
        for rho in (8.0, 16.0, 27.5, 48.0):
            gj.set_cost_params({"bg_over_br": rho, "bg_over_bl2": rho / 4.5})
            be.append(break_even())
        assert all(b < a for a, b in zip(be, be[1:])) and 0.0 < be[-1] < be[0] < 1.0
    finally:
        gj.set_cost_params(None)


def test_cost_model_zipf_share_of_the_hottest_partition():
    """The PGB skew term is share(g, z) x n x SMs x hot_row_bytes with share =
    1 / H(g, z): its growth from z = 0 to z = 1 at g = 2 is (2/3 - 1/2) of that
    product (H(2, 1) = 3/2), and at g = 10^6 the share matches 1 / sum i^-z."""
    from paper_2312_00720_gb300 import gj
    n, sms, hot = 1 << 20, 152, 20.0
    try:
        gj.set_cost_params({"num_sms": sms, "hot_row_bytes": hot})
        pgb = lambda g, z: gj.cost_estimate(None, n, 4, 0, 1, 1, z, 1.0, g, ops=["count"])[1][2]
        assert pgb(2, 1.0) - pgb(2, 0.0) == pytest.approx((2 / 3 - 1 / 2) * n * sms * hot, rel=1e-9)
        g = 10 ** 6
        for z in (0.5, 1.0, 1.25):
            exact = 1.0 / np.sum(np.arange(1, g + 1, dtype=np.float64) ** -z)
            got = (pgb(g, z) - pgb(g, 0.0)) / (n * sms * hot) + 1.0 / g
            assert got == pytest.approx(exact, rel=1e-4)
    finally:
        gj.set_cost_params(None)


def test_cost_params_defaults_and_validation():
    from paper_2312_00720_gb300 import gj
    d = gj.cost_params_default()
    assert d["bg_over_br"] == pytest.approx(27.5) and d["bg_over_bl2"] == pytest.approx(27.5 / 4.5)
    for bad in ({"bg_over_br": 0.5}, {"bg_over_bl2": 0.0}, {"l2_bytes": -1.0}, {"num_sms": -2}):
        with pytest.raises(gj.GjError) as e:
            gj.set_cost_params(bad)
        assert e.value.code == 1
    gj.set_cost_params({"bg_over_br": 40.0})
    gj.set_cost_params(None)
    a = gj.cost_estimate(1 << 20, 1 << 22, 4, 2, 2, 4, 0.0, 1.0, 64)
    gj.set_cost_params({"bg_over_br": 27.5})
    b = gj.cost_estimate(1 << 20, 1 << 22, 4, 2, 2, 4, 0.0, 1.0, 64)
    gj.set_cost_params(None)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_shipped_network_installs_and_picks_the_clear_cases():
    """The package's trained network (80 % of the 4096-point GB300 sweep) loads with
    the parameter layout of the selector and, installed, picks the non-partitioned
    join for a build side far inside L2 and a partitioned join for one far beyond
    it, and the hash group-by for a handful of groups."""
    from paper_2312_00720_gb300 import gj
    z = np.load(selector.TRAINED)
    assert z["theta"].shape == (gj.MLP_PARAMS,) and z["theta"].dtype == np.float32
    assert z["mean"].shape == z["std"].shape == (12,) and (z["std"] > 0).all()
    assert np.isfinite(z["theta"]).all()
    assert selector.install_trained()
    try:
        small = gj.auto_variants(1 << 14, 1 << 17, 4, 2, 2, 4, 0.0, 1.0, 16, selector="mlp", ops=selector.GB_AGGS)
        big = gj.auto_variants(1 << 26, 1 << 27, 4, 2, 2, 4, 0.0, 1.0, 16, selector="mlp", ops=selector.GB_AGGS)
        assert small[0] == 3 and big[0] in (1, 2)
        assert big[1] == 1
    finally:
        gj.selector_set(None, None, None)
