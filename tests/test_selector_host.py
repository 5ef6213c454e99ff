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
    a, b = selector.grid(300, seed=5), selector.grid(300, seed=5)
    assert a == b and selector.grid(300, seed=6) != a
    for p in a:
        assert 2**14 <= p["ns"] <= 2**22 and 16 <= p["nr"] <= p["ns"]
        assert p["key_bytes"] in (4, 8) and 1 <= p["ncols"] <= 4
        assert 0.0 <= p["theta"] <= 1.25 and 0.1 <= p["mr"] <= 1.0 and 4 <= p["groups"] <= p["ns"]


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
    assert x.shape == (7, 12) and y.shape == (7, 6) and y[2, 0] == pytest.approx(np.log(3.0))


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
