"""Group-by variants (HGB Alg. 1, SGB-TR, PGB-TR, their GFUR halves SGB-UR, PGB-UR,
and SGB-DE on dictionary codes) through the C-ABI vs the oracle: canonically
sorted (key, aggregates) rows must be identical."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_00720_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VARIANTS = ["hgb", "sgb", "pgb", "sgb_ur", "pgb_ur", "sgb_de"]
AGGS = ["count", "sum", "min", "max", "sum", "min", "max", "sum", "min", "max"]
COLS = [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]


def run_gb(gj, key, vals, aggs, cols, variant, **kw):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    okeys, outs, ng = gj.groupby(dev(key), [dev(v) for v in vals], aggs, cols, variant=variant, **kw)
    g = int(ng.item())
    return np.stack([okeys[:g].cpu().numpy().astype(np.int64)] + [o[:g].cpu().numpy() for o in outs], 1) \
        if g else np.zeros((0, 1 + len(aggs)), dtype=np.int64)


def want_rows(key, vals, aggs, cols):
    return oracle.canonical(oracle.groupby_sort(key, vals, aggs, cols))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,g,kdt,theta", [
    (0, 4, np.int32, 0.0), (1, 1, np.int32, 0.0), (31, 3, np.int32, 0.0), (511, 7, np.int64, 0.0),
    (512, 512, np.int32, 0.0), (513, 10, np.int32, 0.0), (100000, 1, np.int32, 0.0),
    (100000, 16, np.int32, 0.0), (100000, 4096, np.int64, 0.0), (200003, 1 << 17, np.int32, 0.0),
    (300000, 1000, np.int32, 1.0), (300000, 1 << 20, np.int64, 1.0), (1 << 20, 1 << 22, np.int32, 0.0)])
def test_groupby_matches_oracle(gj, variant, n, g, kdt, theta):
    w = wl.groupby_workload(n, g, nvals=3, key_dtype=kdt, theta=theta, seed=n + g)
    got = oracle.canonical(run_gb(gj, w["key"], w["vals"], AGGS, COLS, variant))
    want = want_rows(w["key"], w["vals"], AGGS, COLS)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", VARIANTS)
def test_int64_values_and_negative_keys(gj, variant):
    rng = np.random.default_rng(11)
    n = 50000
    key = rng.integers(-300, 300, n).astype(np.int32)
    vals = [rng.integers(-(2**62), 2**62, n, dtype=np.int64), rng.integers(-(2**31), 2**31, n).astype(np.int32)]
    aggs = ["sum", "min", "max", "count", "max", "min"]
    cols = [0, 0, 0, 0, 1, 1]
    got = oracle.canonical(run_gb(gj, key, vals, aggs, cols, variant))
    assert np.array_equal(got, want_rows(key, vals, aggs, cols))


@pytest.mark.parametrize("variant", ["sgb", "sgb_ur"])
def test_sgb_output_is_sorted_and_deterministic(gj, variant):
    w = wl.groupby_workload(200000, 5000, nvals=2, seed=2)
    a = run_gb(gj, w["key"], w["vals"], ["sum", "max"], [0, 1], variant)
    b = run_gb(gj, w["key"], w["vals"], ["sum", "max"], [0, 1], variant)
    assert np.array_equal(a, b)
    assert np.all(np.diff(a[:, 0]) > 0)


@pytest.mark.parametrize("variant", ["pgb", "pgb_ur"])
def test_pgb_sub_rounds_when_partition_overflows(gj, variant):
    # one hashed bit gives partitions of ~100K distinct keys, far above one table
    w = wl.groupby_workload(400000, 200000, nvals=1, seed=9)
    got = oracle.canonical(run_gb(gj, w["key"], w["vals"], ["count", "sum"], [0, 0], variant, radix_bits=1))
    assert np.array_equal(got, want_rows(w["key"], w["vals"], ["count", "sum"], [0, 0]))


def test_sgb_de_groups_follow_the_dictionary(gj):
    # SGB-DE writes group i at the dictionary code i: its keys are distinct and
    # the aggregates sit beside their own key
    w = wl.groupby_workload(250000, 1 << 14, nvals=1, seed=31)
    rows = run_gb(gj, w["key"], w["vals"], ["count", "sum"], [0, 0], "sgb_de")
    assert np.unique(rows[:, 0]).size == rows.shape[0]
    assert np.array_equal(oracle.canonical(rows), want_rows(w["key"], w["vals"], ["count", "sum"], [0, 0]))


def test_sgb_ur_and_tr_give_identical_rows(gj):
    # both sort the keys the same way; only how the values travel differs
    w = wl.groupby_workload(300000, 3000, nvals=3, seed=21)
    a = run_gb(gj, w["key"], w["vals"], AGGS, COLS, "sgb")
    b = run_gb(gj, w["key"], w["vals"], AGGS, COLS, "sgb_ur")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("variant", VARIANTS)
def test_capacity_overflow_is_reported(gj, variant):
    w = wl.groupby_workload(10000, 1000, nvals=1, seed=3)
    with pytest.raises(gj.GjError) as e:
        run_gb(gj, w["key"], w["vals"], ["count"], [0], variant, capacity=10)
    assert e.value.code == 4


def test_auto_variant(gj):
    w = wl.groupby_workload(100000, 64, nvals=1, seed=4)
    got = oracle.canonical(run_gb(gj, w["key"], w["vals"], ["sum"], [0], "auto"))
    assert np.array_equal(got, want_rows(w["key"], w["vals"], ["sum"], [0]))


@pytest.mark.slow
@pytest.mark.parametrize("g,kdt,theta", [(1 << 4, np.int32, 0.0), (1 << 12, np.int32, 0.0),
                                          (1 << 20, np.int64, 0.0), (1 << 26, np.int32, 1.0)])
def test_full_size_plain_groupby(gj, g, kdt, theta):
    """2^27 rows, 3 int32 value columns in [-2^20, 2^20), COUNT + SUM/MIN/MAX per column;
    all three variants equal the oracle's sort-based group-by exactly."""
    n = 1 << 27
    w = wl.groupby_workload(n, g, nvals=3, key_dtype=kdt, theta=theta, seed=77)
    want = want_rows(w["key"], w["vals"], AGGS, COLS)
    assert want[:, 1].sum() == n
    for v in VARIANTS:
        got = oracle.canonical(run_gb(gj, w["key"], w["vals"], AGGS, COLS, v))
        assert np.array_equal(got, want), v


@pytest.mark.parametrize("variant", VARIANTS)
def test_extreme_int32_values(gj, variant):
    # groups whose values all sit at INT32_MAX / INT32_MIN: the 32-bit identities of
    # MIN / MAX are real values here and must come out as such
    rng = np.random.default_rng(17)
    n = 40000
    key = rng.integers(0, 64, n).astype(np.int32)
    v = rng.integers(-5, 5, n).astype(np.int32)
    v[key < 8] = np.iinfo(np.int32).max
    v[(key >= 8) & (key < 16)] = np.iinfo(np.int32).min
    aggs = ["min", "max", "sum", "count"]
    cols = [0, 0, 0, 0]
    got = oracle.canonical(run_gb(gj, key, [v], aggs, cols, variant))
    assert np.array_equal(got, want_rows(key, [v], aggs, cols))


@pytest.mark.parametrize("variant", ["hgb", "pgb", "pgb_ur", "sgb_de"])
@pytest.mark.parametrize("n,g,kdt,theta", [
    (1 << 20, 16, np.int32, 0.0), (1 << 20, 4096, np.int64, 1.0), (1 << 21, 1 << 16, np.int32, 0.0),
    (500001, 1 << 12, np.int32, 1.2), (77777, 3, np.int64, 0.0)])
def test_groupby_with_groups_hint(gj, variant, n, g, kdt, theta):
    # the hint sizes HGB's dictionary and sets PGB's partition bits (few, large
    # partitions for few groups): results are unchanged
    w = wl.groupby_workload(n, g, nvals=3, key_dtype=kdt, theta=theta, seed=n ^ g)
    got = oracle.canonical(run_gb(gj, w["key"], w["vals"], AGGS, COLS, variant, groups_hint=g))
    assert np.array_equal(got, want_rows(w["key"], w["vals"], AGGS, COLS))


@pytest.mark.parametrize("variant", ["hgb", "pgb"])
def test_one_hot_key_per_warp(gj, variant):
    # every row has the same key: each warp's 32 rows are combined before one atomic
    n = 300001
    key = np.full(n, -7, dtype=np.int32)
    rng = np.random.default_rng(4)
    vals = [rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32) for _ in range(3)]
    got = run_gb(gj, key, vals, AGGS, COLS, variant, groups_hint=1)
    assert np.array_equal(oracle.canonical(got), want_rows(key, vals, AGGS, COLS))


@pytest.mark.parametrize("n,g,kdt,theta,hint", [
    (1, 1, np.int32, 0.0, 1), (1000, 16, np.int32, 0.0, 16), (300001, 16, np.int64, 1.0, 16),
    (1 << 20, 32, np.int32, 0.0, 32), (777777, 7, np.int32, 1.2, 8),
    (500000, 48, np.int32, 0.0, 32),     # more groups than the few-groups pass takes: the general path runs
    (200000, 33, np.int64, 0.0, 32)])
def test_hgb_few_groups_pass(gj, n, g, kdt, theta, hint):
    w = wl.groupby_workload(n, g, nvals=3, key_dtype=kdt, theta=theta, seed=n + g)
    got = oracle.canonical(run_gb(gj, w["key"], w["vals"], AGGS, COLS, "hgb", groups_hint=hint))
    assert np.array_equal(got, want_rows(w["key"], w["vals"], AGGS, COLS))


@pytest.mark.parametrize("case", ["count_only", "one_column", "two_columns_int64", "ragged_large",
                                  "seventeen_keys", "int64_min_key", "sums_past_32_bits"])
def test_hgb_sorted_tiles_pass(gj, case):
    """Hints of at most 16 groups take the pass that sorts tiles by group in shared
    memory: every cached-column count (0 to 3), ragged tails over many tiles, a
    17th key or the reserved 8-byte key (the general path takes over, with bulk
    copies still in flight), sums past 32 bits."""
    rng = np.random.default_rng(len(case))
    aggs, cols, hint = AGGS, COLS, 16
    if case == "count_only":
        n = (1 << 20) + 3
        key = rng.integers(-8, 8, n).astype(np.int32)
        vals, aggs, cols = [rng.integers(-5, 5, n).astype(np.int32)], ["count"], [0]
    elif case == "one_column":
        w = wl.groupby_workload((1 << 22) + 5, 12, nvals=1, theta=1.0, seed=3)
        key, vals, hint = w["key"], w["vals"], 12
        aggs, cols = ["max", "count", "sum", "min"], [0, 0, 0, 0]
    elif case == "two_columns_int64":
        w = wl.groupby_workload(999999, 16, nvals=2, key_dtype=np.int64, seed=4)
        key, vals = w["key"], w["vals"]
        aggs, cols = ["sum", "min", "max", "sum", "count"], [0, 0, 1, 1, 0]
    elif case == "ragged_large":
        w = wl.groupby_workload((1 << 24) + 777, 16, nvals=3, seed=5)
        key, vals = w["key"], w["vals"]
    elif case == "seventeen_keys":
        w = wl.groupby_workload(1 << 20, 17, nvals=3, seed=6)
        key, vals = w["key"], w["vals"]
        assert len(np.unique(key)) == 17
    elif case == "int64_min_key":
        n = 300000
        key = rng.integers(0, 4, n).astype(np.int64)
        key[rng.random(n) < 0.25] = np.iinfo(np.int64).min
        vals = [rng.integers(-1000, 1000, n).astype(np.int32) for _ in range(3)]
        hint = 5
    else:
        n = 1 << 21
        key = rng.integers(0, 3, n).astype(np.int32)
        vals = [np.full(n, np.iinfo(np.int32).max, np.int32), np.full(n, np.iinfo(np.int32).min, np.int32),
                rng.integers(2**30, 2**31, n).astype(np.int32)]
    got = oracle.canonical(run_gb(gj, key, vals, aggs, cols, "hgb", groups_hint=hint))
    assert np.array_equal(got, want_rows(key, vals, aggs, cols))


@pytest.mark.parametrize("kdt", [np.int32, np.int64])
def test_hgb_sorted_tiles_unaligned_columns(gj, kdt):
    """Columns that do not start on 16 bytes are read with plain loads instead of
    bulk copies: views one row into their buffers."""
    w = wl.groupby_workload((1 << 21) + 1, 16, nvals=3, key_dtype=kdt, theta=0.5, seed=9)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    key, vals = dev(w["key"])[1:], [dev(v)[1:] for v in w["vals"]]
    assert key.data_ptr() % 16 != 0
    okeys, outs, ng = gj.groupby(key, vals, AGGS, COLS, variant="hgb", groups_hint=16)
    g = int(ng.item())
    got = np.stack([okeys[:g].cpu().numpy().astype(np.int64)] + [o[:g].cpu().numpy() for o in outs], 1)
    want = want_rows(w["key"][1:], [v[1:] for v in w["vals"]], AGGS, COLS)
    assert np.array_equal(oracle.canonical(got), want)


def test_hgb_few_groups_pass_extreme_values_and_wide_columns(gj):
    rng = np.random.default_rng(23)
    n = 100000
    key = rng.integers(0, 20, n).astype(np.int32)
    v = rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32)
    v[key == 3] = np.iinfo(np.int32).max
    v[key == 4] = np.iinfo(np.int32).min
    aggs, cols = ["sum", "min", "max", "count"], [0, 0, 0, 0]
    got = oracle.canonical(run_gb(gj, key, [v], aggs, cols, "hgb", groups_hint=20))
    assert np.array_equal(got, want_rows(key, [v], aggs, cols))
    # an 8-byte value column is outside the few-groups pass: the general path runs
    wide = rng.integers(-(2**62), 2**62, n, dtype=np.int64)
    got = oracle.canonical(run_gb(gj, key, [wide], aggs, cols, "hgb", groups_hint=20))
    assert np.array_equal(got, want_rows(key, [wide], aggs, cols))


def _hot_mix(n, hot_frac, n_other, seed):
    """Keys: a hot_frac share of the rows on one key, the rest uniform over n_other keys."""
    rng = np.random.default_rng(seed)
    key = rng.integers(-(2**31), 2**31, n_other, dtype=np.int64).astype(np.int32)[rng.integers(0, n_other, n)]
    key[rng.random(n) < hot_frac] = 123456789
    vals = [rng.integers(-(2**20), 2**20, n).astype(np.int32) for _ in range(3)]
    return key, vals


@pytest.mark.parametrize("variant", ["pgb", "pgb_ur"])
@pytest.mark.parametrize("case", ["few_groups", "zipf", "hot_key_many_groups", "hot_key_wrong_hint"])
def test_pgb_slices_large_partitions(gj, variant, case):
    """Partitions far larger than the average are cut into slices aggregated by
    several blocks into partial rows, then merged: few groups (every non-empty
    partition sliced), Zipf skew, and a hot key whose partition also holds more
    distinct keys than one block can (sub-rounds in the slices and in the merge)."""
    n = 1 << 22
    if case == "few_groups":
        w = wl.groupby_workload(n, 16, nvals=3, seed=5)
        key, vals, hint = w["key"], w["vals"], 16
    elif case == "zipf":
        w = wl.groupby_workload(n, 1 << 12, nvals=3, theta=1.2, seed=6)
        key, vals, hint = w["key"], w["vals"], 1 << 12
    elif case == "hot_key_many_groups":
        key, vals = _hot_mix(n, 0.5, 1 << 20, seed=7)
        hint = 1 << 10  # too small: partitions hold several rounds' worth of keys
    else:
        key, vals = _hot_mix(n, 0.3, 1 << 16, seed=8)
        hint = 0
    got = oracle.canonical(run_gb(gj, key, vals, AGGS, COLS, variant, groups_hint=hint))
    assert np.array_equal(got, want_rows(key, vals, AGGS, COLS))
