"""Join variants through the C-ABI vs the oracle (Sec. 2.2): canonically sorted
result multisets must be identical; at full size, properties that pin every row."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_00720_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VARIANTS = ["phj_tr", "phj_ur", "nphj", "smj_tr", "smj_ur"]


def run_join(gj, w, variant, **kw):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    tkey, tcols, cnt = gj.join(dev(w["rkey"]), [dev(c) for c in w["rcols"]], dev(w["skey"]),
                               [dev(c) for c in w["scols"]], variant=variant, **kw)
    m = int(cnt.item())
    rows = np.stack([tkey[:m].cpu().numpy().astype(np.int64)] +
                    [c[:m].cpu().numpy().astype(np.int64) for c in tcols], axis=1) if m else \
        np.zeros((0, 1 + len(tcols)), dtype=np.int64)
    return rows


def oracle_rows(w):
    return oracle.join(w["rkey"], w["rcols"], w["skey"], w["scols"])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nr,ns,ncr,ncs,theta,mr", [
    (0, 1000, 2, 2, 0.0, 1.0), (1000, 0, 2, 2, 0.0, 1.0), (1, 1, 1, 1, 0.0, 1.0),
    (5000, 20000, 4, 4, 0.0, 1.0), (5000, 20011, 4, 4, 0.0, 0.5), (3000, 50000, 2, 3, 1.0, 1.0),
    (70000, 300007, 1, 1, 0.5, 0.5), (20000, 9000, 0, 0, 0.0, 0.9), (300000, 1000000, 4, 4, 0.0, 1.0)])
def test_join_matches_oracle(gj, variant, nr, ns, ncr, ncs, theta, mr):
    w = wl.join_workload(nr, ns, ncr, ncs, theta=theta, mr=mr, seed=nr + ns)
    got = oracle.canonical(run_join(gj, w, variant))
    want = oracle.canonical(oracle_rows(w))
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", VARIANTS)
def test_int64_keys_and_mixed_columns(gj, variant):
    rng = np.random.default_rng(3)
    nr, ns = 40000, 120000
    rkey = rng.permutation(np.unique(rng.integers(-(2**62), 2**62, nr + 100, dtype=np.int64)))[:nr]
    skey = np.where(rng.random(ns) < 0.7, rkey[rng.integers(0, nr, ns)], rng.integers(-(2**63), 2**63 - 1, ns))
    w = {"rkey": rkey, "skey": skey.astype(np.int64),
         "rcols": [rng.integers(-(2**40), 2**40, nr), rng.integers(0, 100, nr).astype(np.int32)],
         "scols": [rng.integers(0, 2**31, ns).astype(np.int32), rng.integers(-(2**60), 2**60, ns)]}
    got = oracle.canonical(run_join(gj, w, variant))
    assert np.array_equal(got, oracle.canonical(oracle_rows(w)))


@pytest.mark.parametrize("bits,bpp", [(0, 0), (1, 0), (7, 0), (12, 4), (16, 0), (16, 5)])
def test_radix_bits_do_not_change_result(gj, bits, bpp):
    w = wl.join_workload(30000, 90000, 2, 2, theta=0.5, mr=0.8, seed=5)
    want = oracle.canonical(oracle_rows(w))
    for v in ("phj_tr", "phj_ur"):
        got = oracle.canonical(run_join(gj, w, v, radix_bits=bits, bits_per_pass=bpp))
        assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", ["smj_tr", "smj_ur"])
def test_sort_merge_with_a_large_build_range_per_tile(gj, variant):
    # |R| >> |S|: a tile's keys span far more R rows than the shared-memory stage
    # holds, so the merge searches R in global memory
    w = wl.join_workload(1 << 20, 5000, 2, 2, mr=0.9, seed=12)
    assert np.array_equal(oracle.canonical(run_join(gj, w, variant)), oracle.canonical(oracle_rows(w)))


def test_build_partition_larger_than_shared_memory_table(gj):
    # radix_bits = 1 puts ~16K build rows in a partition: chunked builds
    w = wl.join_workload(1 << 15, 1 << 17, 2, 1, seed=8)
    got = oracle.canonical(run_join(gj, w, "phj_tr", radix_bits=1))
    assert np.array_equal(got, oracle.canonical(oracle_rows(w)))


@pytest.mark.parametrize("variant", VARIANTS)
def test_duplicate_primary_key_is_reported(gj, variant):
    w = wl.join_workload(1000, 4000, 1, 1, seed=2)
    w["rkey"][10] = w["rkey"][20]
    with pytest.raises(gj.GjError) as e:
        run_join(gj, w, variant)
    assert e.value.code == 5


@pytest.mark.parametrize("variant", ["phj_tr", "phj_ur"])
@pytest.mark.parametrize("nr,ns,kdt,theta,mr", [
    (1 << 18, 1 << 20, np.int32, 1.0, 0.7), (200003, 600011, np.int64, 0.0, 1.0),
    (131073, 131073, np.int32, 0.5, 0.3), (1 << 20, 3 << 20, np.int32, 0.0, 1.0)])
def test_l2_sized_build_partitions_match_oracle(gj, variant, nr, ns, kdt, theta, mr):
    # build sides above 2^17 rows take one 8-bit pass per side and L2-resident tables;
    # the result equals the oracle's and the two-pass shared-memory path's
    w = wl.join_workload(nr, ns, 2, 2, theta=theta, mr=mr, key_dtype=kdt, seed=nr ^ ns)
    want = oracle.canonical(oracle_rows(w))
    got = oracle.canonical(run_join(gj, w, variant))
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.canonical(run_join(gj, w, variant, radix_bits=16)), want)


@pytest.mark.parametrize("variant", ["phj_tr", "phj_ur"])
def test_duplicate_primary_key_in_an_l2_sized_build(gj, variant):
    w = wl.join_workload(300000, 400000, 1, 1, seed=4)
    w["rkey"][123456] = w["rkey"][7]
    with pytest.raises(gj.GjError) as e:
        run_join(gj, w, variant)
    assert e.value.code == 5


@pytest.mark.parametrize("variant", VARIANTS)
def test_capacity_overflow_is_reported(gj, variant):
    w = wl.join_workload(1000, 4000, 1, 1, seed=2)
    with pytest.raises(gj.GjError) as e:
        run_join(gj, w, variant, capacity=100)
    assert e.value.code == 4


def test_phj_output_is_deterministic(gj):
    w = wl.join_workload(100000, 400000, 2, 2, theta=1.0, mr=0.7, seed=4)
    a = run_join(gj, w, "phj_tr")
    b = run_join(gj, w, "phj_tr")
    assert np.array_equal(a, b)


def _fingerprint(mat):
    h = np.zeros(mat.shape[0], dtype=np.uint64)
    with np.errstate(over="ignore"):
        for c in range(mat.shape[1]):
            h = wl.mix64(h ^ mat[:, c].astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15 + 2 * c))
    return np.sort(h)


@pytest.mark.slow
@pytest.mark.parametrize("theta,mr", [(0.0, 1.0), (0.0, 0.5), (0.5, 1.0), (1.0, 1.0), (1.0, 0.5), (0.5, 0.5)])
@pytest.mark.parametrize("variant", ["phj_tr", "phj_ur"])
def test_full_size_plain_join(gj, theta, mr, variant):
    """|R| = 2^25, |S| = 2^27, 4 int32 payloads per side, the benchmark's launch configuration.
    Pins every output row: |T| = |S| mr exactly; each row's R part is the R row of its key;
    the (key, S part) multiset equals that of the matching S rows (64-bit row fingerprints)."""
    nr, ns = 1 << 25, 1 << 27
    w = wl.join_workload(nr, ns, 4, 4, theta=theta, mr=mr, seed=2023)
    dev = lambda a: torch.from_numpy(a).cuda()
    tkey, tcols, cnt = gj.join(dev(w["rkey"]), [dev(c) for c in w["rcols"]], dev(w["skey"]),
                               [dev(c) for c in w["scols"]], variant=variant)
    m = int(cnt.item())
    assert m == w["n_match"] == int(round(ns * mr))
    tk = tkey[:m].cpu().numpy()
    pos = np.empty(nr, dtype=np.int64)
    pos[w["rkey"]] = np.arange(nr)
    assert tk.min() >= 0 and tk.max() < nr
    rp = pos[tk]
    for c in range(4):
        assert np.array_equal(tcols[c][:m].cpu().numpy(), w["rcols"][c][rp])
    matched = w["skey"] < nr
    s_side = np.stack([w["skey"][matched]] + [c[matched] for c in w["scols"]], axis=1)
    t_side = np.stack([tk] + [tcols[4 + c][:m].cpu().numpy() for c in range(4)], axis=1)
    assert np.array_equal(_fingerprint(t_side), _fingerprint(s_side))


# ---- many-to-many (Sec. 5.1.9): R and S keys from a set of nk keys, every pair out
@pytest.mark.parametrize("nr,ns,nk,ncr,ncs", [
    (1, 1, 1, 1, 1), (100, 100, 1, 2, 2), (1000, 3000, 50, 2, 2), (20011, 30011, 5000, 2, 2),
    (65536, 65536, 1 << 13, 2, 2), (100000, 70000, 100000, 3, 1), (5000, 4000, 4000, 0, 0)])
@pytest.mark.parametrize("variant", ["nphj_mn", "phj_mn"])
def test_many_to_many_matches_oracle(gj, variant, nr, ns, nk, ncr, ncs):
    w = wl.mn_join_workload(nr, ns, nk, ncr, ncs, seed=nr + nk)
    want = oracle.canonical(oracle_rows(w))
    got = oracle.canonical(run_join(gj, w, variant, capacity=max(1, want.shape[0])))
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", ["nphj_mn", "phj_mn"])
def test_many_to_many_int64_keys_and_pk_fk_input(gj, variant):
    # 8-byte keys; and on a key-foreign-key input the pairs equal the FK-PK join's
    w = wl.mn_join_workload(30000, 40000, 7000, 2, 2, key_dtype=np.int64, seed=5)
    want = oracle.canonical(oracle_rows(w))
    assert np.array_equal(oracle.canonical(run_join(gj, w, variant, capacity=want.shape[0])), want)
    w = wl.join_workload(5000, 20011, 2, 2, mr=0.5, seed=3)
    assert np.array_equal(oracle.canonical(run_join(gj, w, variant)),
                          oracle.canonical(run_join(gj, w, "nphj")))


def test_partitioned_many_to_many_with_few_partitions_or_hot_keys(gj):
    # radix_bits 1: two partitions; nk = 3: three keys, each with thousands of rows
    w = wl.mn_join_workload(20000, 300, 3, 1, 1, seed=6)
    want = oracle.canonical(oracle_rows(w))
    for bits in (1, 0):
        got = oracle.canonical(run_join(gj, w, "phj_mn", capacity=want.shape[0], radix_bits=bits))
        assert np.array_equal(got, want)


@pytest.mark.parametrize("variant", ["nphj_mn", "phj_mn"])
def test_many_to_many_capacity_overflow_is_reported(gj, variant):
    w = wl.mn_join_workload(2000, 2000, 10, 1, 1, seed=8)  # about 4e5 pairs
    with pytest.raises(gj.GjError) as e:
        run_join(gj, w, variant, capacity=1000)
    assert e.value.code == 4
