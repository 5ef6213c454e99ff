"""Pins of the CPU oracle against facts that do not come from the oracle itself:
nested-loop brute force on tiny inputs, invariants, closed forms, special cases
that reduce to library routines, and values printed in the paper."""
import math

import numpy as np
import pytest

import oracle
from oracle import cost_models as cm
from oracle import heuristics as hz
from paper_2312_00720_gb300 import workloads as wl

from conftest import read_golden


# ------------------------------------------------------------------ brute force
def brute_join(rkey, rcols, skey, scols):
    rows = []
    for j in range(len(skey)):
        for i in range(len(rkey)):
            if int(rkey[i]) == int(skey[j]):
                rows.append([int(rkey[i])] + [int(c[i]) for c in rcols] + [int(c[j]) for c in scols])
    return np.array(rows, dtype=np.int64).reshape(-1, 1 + len(rcols) + len(scols))


def brute_groupby(key, cols, aggs, agg_cols):
    out = []
    for k in sorted(set(int(x) for x in key)):
        idx = [i for i in range(len(key)) if int(key[i]) == k]
        row = [k]
        for a, c in zip(aggs, agg_cols):
            vals = [int(cols[c][i]) for i in idx]
            row.append({"sum": sum(vals), "count": len(idx), "min": min(vals), "max": max(vals)}[a])
        out.append(row)
    return np.array(out, dtype=np.int64).reshape(-1, 1 + len(aggs))


AGGS = ["count", "sum", "min", "max", "sum", "min", "max"]
AGG_COLS = [0, 0, 0, 0, 1, 1, 1]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("nr,ns,kdom", [(0, 5, 4), (5, 0, 4), (1, 1, 1), (17, 40, 8), (64, 200, 300), (50, 50, 3)])
def test_join_vs_nested_loop(seed, nr, ns, kdom):
    # keys drawn with replacement: covers many-to-many, all-equal keys (kdom = 1) and no-match
    rng = np.random.default_rng(seed)
    rkey = rng.integers(-kdom, kdom, nr)
    skey = rng.integers(-kdom, kdom, ns)
    rcols = [rng.integers(-100, 100, nr) for _ in range(2)]
    scols = [rng.integers(-100, 100, ns) for _ in range(3)]
    got = oracle.canonical(oracle.join(rkey, rcols, skey, scols))
    want = oracle.canonical(brute_join(rkey, rcols, skey, scols))
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_join_fk_pk_cardinality_is_ns_times_mr():
    for mr in (1.0, 0.5, 0.1):
        w = wl.join_workload(1000, 5000, 2, 2, mr=mr, seed=11)
        t = oracle.join(w["rkey"], w["rcols"], w["skey"], w["scols"])
        assert len(t) == int(round(5000 * mr)) == w["n_match"]
        # every row's R part is the R row holding its key (R.key is a permutation of 0..|R|-1)
        pos = np.empty(1000, dtype=np.int64)
        pos[w["rkey"]] = np.arange(1000)
        for c in range(2):
            assert np.array_equal(t[:, 1 + c], w["rcols"][c][pos[t[:, 0]]])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n,kdom", [(0, 3), (1, 1), (37, 1), (100, 7), (300, 1000), (257, 256)])
def test_groupby_vs_brute_force(seed, n, kdom):
    rng = np.random.default_rng(100 + seed)
    key = rng.integers(-kdom, kdom + 1, n)
    cols = [rng.integers(-(2**20), 2**20, n), rng.integers(-(2**31), 2**31, n)]
    want = brute_groupby(key, cols, AGGS, AGG_COLS)
    for fn in (oracle.groupby_hash, oracle.groupby_sort):
        got = oracle.canonical(fn(key, cols, AGGS, AGG_COLS))
        assert np.array_equal(got, oracle.canonical(want))


def test_groupby_hash_and_sort_agree_and_invariants():
    w = wl.groupby_workload(20000, 4096, nvals=3, seed=5)
    aggs = ["count"] + ["sum", "min", "max"] * 3
    cols = [0] + [0, 0, 0, 1, 1, 1, 2, 2, 2]
    a = oracle.canonical(oracle.groupby_hash(w["key"], w["vals"], aggs, cols))
    b = oracle.canonical(oracle.groupby_sort(w["key"], w["vals"], aggs, cols))
    assert np.array_equal(a, b)
    assert a[:, 1].sum() == 20000                       # sum of COUNT = n
    for c in range(3):
        assert a[:, 2 + 3 * c].sum() == w["vals"][c].astype(np.int64).sum()   # sum of SUM = column sum
        assert np.all(a[:, 3 + 3 * c] <= a[:, 4 + 3 * c])                     # MIN <= MAX
    assert len(a) == len(np.unique(w["key"]))


def test_groupby_special_cases_reduce_to_numpy():
    rng = np.random.default_rng(9)
    v = rng.integers(-1000, 1000, 500)
    # one group: the aggregates are numpy's reductions of the column
    g = oracle.groupby_sort(np.full(500, 42), [v], ["count", "sum", "min", "max"], [0, 0, 0, 0])
    assert g.tolist() == [[42, 500, int(v.sum()), int(v.min()), int(v.max())]]
    # all keys distinct: every group is its own row
    k = rng.permutation(500)
    g = oracle.canonical(oracle.groupby_hash(k, [v], ["count", "sum", "min", "max"], [0, 0, 0, 0]))
    assert np.array_equal(g[:, 0], np.arange(500))
    assert np.array_equal(g[:, 2], v[np.argsort(k)])
    assert np.all(g[:, 1] == 1)


def test_sum_wraps_in_two_complement():
    big = np.array([2**62, 2**62, 2**62, 2**62], dtype=np.int64)
    g = oracle.groupby_hash(np.zeros(4), [big], ["sum"], [0])
    assert g[0, 1] == 0  # 2^64 wraps to 0 exactly


@pytest.mark.parametrize("seed", range(4))
def test_join_groupby_is_join_then_groupby(seed):
    rng = np.random.default_rng(seed)
    nr, ns = 40, 120
    rkey = rng.integers(0, 30, nr)
    skey = rng.integers(0, 30, ns)
    rcols = [rng.integers(0, 2**31, nr), rng.integers(-50, 50, nr)]
    scols = [rng.integers(0, 2**31, ns)]
    got = oracle.join_groupby(rkey, rcols, skey, scols, g_side=0, g_col=0, g_mod=7,
                              aggs=["count", "sum", "max"], agg_side=[0, 1, 0], agg_col=[0, 0, 1])
    t = brute_join(rkey, rcols, skey, scols)
    gk = t[:, 1] % 7
    want = brute_groupby(gk, [t[:, 3], t[:, 2]], ["count", "sum", "max"], [0, 0, 1])
    assert np.array_equal(oracle.canonical(got), oracle.canonical(want))


def test_join_groupby_one_query_closed_forms():
    # the one-query shape at 1/16 scale: every S row matches once, so COUNTs total |S|
    # and SUMs total the S payload column
    w = wl.join_workload(1 << 16, 1 << 18, 1, 1, seed=5)
    a = oracle.join_groupby(w["rkey"], w["rcols"], w["skey"], w["scols"], g_side=0, g_col=0, g_mod=1024,
                            aggs=["sum", "count"], agg_side=[1, 1], agg_col=[0, 0])
    assert a[:, 2].sum() == 1 << 18
    assert a[:, 1].sum() == w["scols"][0].astype(np.int64).sum()
    assert len(a) <= 1024 and a[:, 0].min() >= 0 and a[:, 0].max() < 1024


@pytest.mark.parametrize("transform", [0, 1, 2])
@pytest.mark.parametrize("key_bytes", [4, 8])
@pytest.mark.parametrize("lo,hi", [(0, 4), (3, 11), (0, 1)])
def test_radix_partition_is_python_stable_sort(transform, key_bytes, lo, hi):
    rng = np.random.default_rng(lo * 31 + hi + key_bytes + transform)
    n = 777
    if key_bytes == 4:
        key = rng.integers(-(2**31), 2**31, n).astype(np.int64)
    else:
        key = rng.integers(-(2**63), 2**63 - 1, n, dtype=np.int64)
    key[::5] = key[0]  # duplicates make stability observable
    perm, offs = oracle.radix_partition(key, key_bytes, lo, hi, transform)

    mask = (1 << (8 * key_bytes)) - 1

    def fmix32(h):
        h ^= h >> 16; h = (h * 0x85EBCA6B) & 0xFFFFFFFF; h ^= h >> 13
        h = (h * 0xC2B2AE35) & 0xFFFFFFFF; h ^= h >> 16
        return h

    def fmix64(k):
        m = 0xFFFFFFFFFFFFFFFF
        k ^= k >> 33; k = (k * 0xFF51AFD7ED558CCD) & m; k ^= k >> 33
        k = (k * 0xC4CEB9FE1A85EC53) & m; k ^= k >> 33
        return k

    def digit(x):
        u = int(x) & mask
        if transform == 1:
            u ^= 1 << (8 * key_bytes - 1)
        if transform == 2:
            u = fmix32(u) if key_bytes == 4 else fmix64(u)
        return (u >> lo) & ((1 << (hi - lo)) - 1)

    want = sorted(range(n), key=lambda i: digit(key[i]))  # Python's sort is stable
    assert perm.tolist() == want
    counts = np.bincount([digit(x) for x in key], minlength=1 << (hi - lo))
    assert offs.tolist() == [0] + np.cumsum(counts).tolist()


def test_radix_partition_full_width_signed_is_a_sort():
    rng = np.random.default_rng(3)
    key = rng.integers(-(2**31), 2**31, 1000)
    perm, _ = oracle.radix_partition(key, 4, 0, 32, 1)
    assert np.array_equal(key[perm], np.sort(key, kind="stable"))


# ------------------------------------------------------------------ cost models
def test_fig_phj_mr_estimates():
    for mr, want in read_golden("fig_phj_mr_estimated.txt"):
        assert cm.fig_phj_mr_estimate_ms(float(mr)) == pytest.approx(float(want), rel=1e-9)


def test_fig_sgb_model1_estimates():
    for lg, want in read_golden("fig_sgb_model1_estimated.txt"):
        assert cm.fig_sgb_model1_estimate_ms(2.0 ** int(lg)) == pytest.approx(float(want), rel=1e-9)


def test_fig_sgb_model2_estimates():
    for k, lg, want in read_golden("fig_sgb_model2_estimated.txt"):
        got = cm.fig_sgb_model2_estimate_ms(2.0 ** int(lg), int(k))
        assert got == pytest.approx(float(want), rel=1e-6, abs=1e-6)


def test_printed_thresholds():
    # Sec. 4.1.3: at least 16 groups for sorting to beat the permutation
    assert not cm.m2_gftr_wins(15) and cm.m2_gftr_wins(16)
    # Sec. 4.1.4: mr > 0.39 for one column, > 0.2 for two
    assert round(cm.m3_threshold_mr(1), 2) == 0.39
    assert round(cm.m3_threshold_mr(2), 1) == 0.2


def test_table_de_opt():
    for k, lo, hi, p in read_golden("table_de_opt.txt"):
        k, lo, hi, p = int(k), int(lo), int(hi), int(p)
        got = max(cm.m4_min_payloads(2.0**e, k) for e in range(lo, hi + 1))
        if k == 4 and lo in (15, 17):
            # the model with the figure's constants gives 2 and 4 where the table prints
            # 3 and 5; the model is pinned by Fig. sgb-model2, the mismatch is recorded
            assert got == p - 1
        else:
            assert got == p


def test_gather_profile_gives_bg_over_24():
    rows = {r[0]: (int(r[1]), int(r[2])) for r in read_golden("table_gather_profile.txt")}
    ratio = rows["unclustered"][0] / rows["clustered"][0]
    assert round(ratio, 2) == 8.52
    # both gathers read the map and write the output at B_G (8 bytes/item) and read
    # the input at B_G (clustered) or B_R (unclustered): ratio = (8 + 4 r) / 12, r = B_G / B_R
    r = (ratio * 12 - 8) / 4
    assert round(r) == 24
    assert rows["unclustered"][1] == rows["clustered"][1]


# ------------------------------------------------------------------ heuristics
def test_join_heuristic_follows_conclusion():
    assert hz.choose_join(1.0, 0.0, 4) == hz.JOIN_PHJ_TR
    assert hz.choose_join(0.25, 0.0, 4) == hz.JOIN_PHJ_TR
    assert hz.choose_join(0.2, 0.0, 4) == hz.JOIN_PHJ_UR
    assert hz.choose_join(0.1, 1.0, 4) == hz.JOIN_PHJ_TR
    assert hz.choose_join(0.1, 0.0, 8) == hz.JOIN_PHJ_TR


def test_groupby_decision_tree():
    smem = 200 * 1024
    assert hz.choose_groupby(2**10, 52, smem, 0.0, 4) == hz.GB_HGB
    assert hz.choose_groupby(2**20, 52, smem, 0.0, 4) == hz.GB_PGB
    assert hz.choose_groupby(2**20, 52, smem, 1.0, 4) == hz.GB_SGB
    assert hz.choose_groupby(2**10, 52, smem, 0.0, 4, must_sort=True) == hz.GB_SGB
    assert hz.choose_groupby(2**10, 52, smem, 0.0, 8, must_sort=True, have_dictionary=True) == hz.GB_SGB_DE


# ------------------------------------------------------------------ generators
def test_generator_shapes_and_determinism():
    a = wl.join_workload(4096, 16384, 4, 4, theta=0.5, mr=0.5, seed=3)
    b = wl.join_workload(4096, 16384, 4, 4, theta=0.5, mr=0.5, seed=3)
    assert np.array_equal(a["skey"], b["skey"]) and np.array_equal(a["rcols"][3], b["rcols"][3])
    assert sorted(a["rkey"].tolist()) == list(range(4096))
    assert int(np.sum(a["skey"] >= 4096)) == 8192
    assert all(c.dtype == np.int32 and c.min() >= 0 for c in a["scols"])


def test_zipf_rank_frequencies():
    n, m, theta = 64, 400000, 1.0
    r = wl.zipf_ranks(m, n, theta, seed=1, stream=1)
    p = np.arange(1, n + 1, dtype=np.float64) ** -theta
    p /= p.sum()
    counts = np.bincount(r, minlength=n)
    chi2 = float(np.sum((counts - m * p) ** 2 / (m * p)))
    # 63 degrees of freedom: the 0.999 quantile is about 103
    assert chi2 < 103.0


# ------------------------------------------------------------------ MLP reference
def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, mlp.N_PARAMS)
    x = rng.normal(0, 1, (7, mlp.D_IN))
    t = rng.normal(0, 1, (7, mlp.D_OUT))
    mask = (rng.random((7, mlp.D_OUT)) < 0.8).astype(np.float64)
    _, g = mlp.grad(theta, x, t, mask)
    assert mlp.N_PARAMS == 5707
    h = 1e-6
    for i in rng.choice(mlp.N_PARAMS, 200, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, x, t, mask) - mlp.loss(theta - e, x, t, mask)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_mlp_linear_special_case():
    # with all pre-activations positive the network is affine: y = W3 W2 W1 x + const
    from oracle import mlp
    rng = np.random.default_rng(1)
    p = {"w1": rng.random((64, 12)), "b1": np.ones(64), "w2": rng.random((64, 64)), "b2": np.ones(64),
         "w3": rng.normal(0, 1, (11, 64)), "b3": rng.normal(0, 1, 11)}
    x = rng.random((5, 12))
    y, _ = mlp.forward(mlp.pack(p), x)
    want = ((x @ p["w1"].T + 1) @ p["w2"].T + 1) @ p["w3"].T + p["b3"]
    assert np.allclose(y, want, rtol=1e-12)


def test_sgd_step_on_a_hand_computed_vector():
    from oracle import mlp
    theta = np.array([1.0, -2.0, 0.5, 0.0])
    g = np.array([0.5, 4.0, -1.0, 3.0])
    # theta - 0.25 * g, worked out by hand
    assert np.array_equal(mlp.sgd_step(theta, g, 0.25), np.array([0.875, -3.0, 0.75, -0.75]))


def test_adam_first_step_moves_by_lr_times_sign():
    # from m = v = 0 the bias-corrected moments are g and g^2, so step 1 moves every
    # parameter by lr * g / (|g| + eps) (Kingma & Ba 2015, Algorithm 1), whatever the betas
    from oracle import mlp
    rng = np.random.default_rng(5)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50) * 10.0 ** rng.integers(-3, 3, 50)
    for b1, b2 in ((0.9, 0.999), (0.5, 0.9)):
        new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, 0.01, b1, b2, 1e-8)
        assert np.allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
        assert np.allclose(m, (1 - b1) * g) and np.allclose(v, (1 - b2) * g * g)


def test_adam_constant_gradient_takes_the_same_step_every_time():
    # with a constant gradient m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2: the bias
    # corrections cancel exactly, so steps 1, 2 and 3 are equal
    from oracle import mlp
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    steps = []
    for t in (1, 2, 3):
        new, m, v = mlp.adam_step(th, g, m, v, t, 0.1)
        steps.append(new - th)
        th = new
    want = -0.1 * g / (np.abs(g) + 1e-8)
    for s in steps:
        assert np.allclose(s, want, rtol=1e-12, atol=0)


def test_adam_eps_is_added_after_the_square_root():
    # a gradient far below eps: the step is lr * g / (|g| + eps), not lr * g / sqrt(g^2 + eps)
    from oracle import mlp
    g = np.array([1e-12, -3e-12])
    new, _, _ = mlp.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, 1.0, eps=1e-8)
    assert np.allclose(new, -g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert abs(new[0]) < 1.1e-4 and abs(new[0]) > 0.9e-4


def test_many_to_many_generator_draws_from_nk_keys():
    a = wl.mn_join_workload(5000, 7000, 300, 2, 1, seed=4)
    b = wl.mn_join_workload(5000, 7000, 300, 2, 1, seed=4)
    for k in ("rkey", "skey"):
        assert np.array_equal(a[k], b[k])
    keys = np.union1d(a["rkey"], a["skey"])
    assert keys.size <= 300 and np.unique(a["rkey"]).size > 250
    assert len(a["rcols"]) == 2 and len(a["scols"]) == 1 and a["scols"][0].shape == (7000,)
    # |T| = sum over keys of (R rows with it) x (S rows with it)
    t = oracle.join(a["rkey"], a["rcols"], a["skey"], a["scols"])
    rk, rc = np.unique(a["rkey"], return_counts=True)
    sk, sc = np.unique(a["skey"], return_counts=True)
    common, ri, si = np.intersect1d(rk, sk, return_indices=True)
    assert len(t) == int((rc[ri].astype(np.int64) * sc[si]).sum())


@pytest.mark.parametrize("n,g,theta", [(1 << 20, 1 << 20, 0.0), (1 << 21, 1 << 12, 0.0), (1 << 20, 1 << 22, 0.0),
                                       (1 << 20, 1 << 18, 1.0)])
def test_groupby_generator_distinct_count(n, g, theta):
    # n draws over g ids: E[distinct] = sum_r 1 - (1 - p_r)^n, which for the uniform law
    # is g (1 - (1 - 1/g)^n) ~ g (1 - e^{-n/g}); occupancy indicators are negatively
    # associated, so Var[distinct] <= sum_r q_r (1 - q_r) with q_r = 1 - (1 - p_r)^n
    w = wl.groupby_workload(n, g, nvals=1, theta=theta, seed=21)
    p = np.arange(1, g + 1, dtype=np.float64) ** -theta
    p /= p.sum()
    q = -np.expm1(n * np.log1p(-p))
    mean, sd = q.sum(), math.sqrt(float(np.sum(q * (1.0 - q))))
    got = np.unique(w["key"]).size
    assert abs(got - mean) <= 6.0 * sd + 1.0
    if theta == 0.0:
        assert mean == pytest.approx(g * (1.0 - math.exp(-n / g)), rel=1e-5)
        assert w["key"].min() >= 0 and w["key"].max() < g
    # 8-byte keys come from a bijection of the same ids: the same groups, the same sizes
    w8 = wl.groupby_workload(n, g, nvals=1, theta=theta, seed=21, key_dtype=np.int64)
    _, c4 = np.unique(w["key"], return_counts=True)
    _, c8 = np.unique(w8["key"], return_counts=True)
    assert np.array_equal(np.sort(c4), np.sort(c8))
    assert np.array_equal(w["vals"][0], w8["vals"][0])
    assert w["vals"][0].min() >= -(2**20) and w["vals"][0].max() < 2**20


def test_batch_generator_sizes_follow_the_log_uniform_law():
    # log2 |R| ~ U[10, 20] and log2 G ~ U[2, 16] over 512 instances: a Kolmogorov-Smirnov
    # bound on each, and the mean |R| against E[2^U] = (2^20 - 2^10) / (10 ln 2)
    sizes = wl.batch_sizes(512)
    nr = np.array([a for a, _ in sizes], dtype=np.float64)
    g = np.array([b for _, b in sizes], dtype=np.float64)
    assert nr.min() >= 2**10 and nr.max() <= 2**20 and g.min() >= 4 and g.max() <= 2**16
    for x, lo, hi in ((np.log2(nr), 10.0, 20.0), (np.log2(g), 2.0, 16.0)):
        u = np.sort((x - lo) / (hi - lo))
        k = np.arange(1, len(u) + 1) / len(u)
        d = max(np.max(k - u), np.max(u - (k - 1.0 / len(u))))
        assert d < 1.95 / math.sqrt(len(u)) + 0.5 / len(u)   # 99.9 % quantile, plus rounding to integers
    mean = (2.0**20 - 2.0**10) / (10 * math.log(2))
    var = (4.0**20 - 4.0**10) / (10 * math.log(4)) - mean**2
    assert abs(nr.mean() - mean) < 5 * math.sqrt(var / len(nr))
    assert round(mean, -3) == 151000   # E[|R|] of the batched configuration, about 1.51e5


def test_zipf_foreign_keys_follow_the_primary_key_order():
    # S.key takes rank r to R.key[r] (R is a seeded permutation): R.key[0] is the
    # hottest key with probability 1 / H_n, R.key[1] half of that, ...
    nr, ns = 1000, 400000
    w = wl.join_workload(nr, ns, 1, 1, theta=1.0, mr=1.0, seed=9)
    p = 1.0 / np.arange(1, nr + 1)
    p /= p.sum()
    counts = {int(k): c for k, c in zip(*np.unique(w["skey"], return_counts=True))}
    for r in (0, 1, 2, 9, 99):
        want = ns * p[r]
        assert abs(counts.get(int(w["rkey"][r]), 0) - want) < 5 * math.sqrt(want * (1 - p[r]))
    assert set(counts) <= set(int(x) for x in w["rkey"])


def test_join_groupby_modulus_truncates_toward_zero():
    # reading R9: the group key modulus is C's %, so negative values keep their sign
    # (residues in (-m, m)); np.fmod is the same truncating remainder
    rng = np.random.default_rng(17)
    nr, ns = 60, 300
    rkey = rng.permutation(nr)
    skey = rng.integers(0, nr, ns)
    rcols = [rng.integers(-1000, 1000, nr)]
    scols = [rng.integers(-50, 50, ns)]
    got = oracle.join_groupby(rkey, rcols, skey, scols, g_side=0, g_col=0, g_mod=7,
                              aggs=["count", "sum", "min"], agg_side=[1, 1, 1], agg_col=[0, 0, 0])
    t = brute_join(rkey, rcols, skey, scols)
    gk = np.fmod(t[:, 1], 7)
    assert gk.min() < 0                      # the case the reading is about occurs
    want = brute_groupby(gk, [t[:, 2]], ["count", "sum", "min"], [0, 0, 0])
    assert np.array_equal(oracle.canonical(got), oracle.canonical(want))
    assert got[:, 0].min() > -7 and got[:, 0].max() < 7


def test_gather_is_indexing_and_a_permutation_round_trips():
    rng = np.random.default_rng(6)
    src = rng.integers(-(2**31), 2**31, 50).astype(np.int32)
    idx = rng.integers(0, 50, 80)
    assert np.array_equal(oracle.gather(src, idx), src[idx])
    perm = rng.permutation(50)
    inv = np.argsort(perm)
    assert np.array_equal(oracle.gather(oracle.gather(src, perm), inv), src)
