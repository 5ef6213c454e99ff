"""Join -> group-by without materialising the join (gj_join_groupby) vs the oracle,
which computes the join first and groups its rows."""
import numpy as np
import pytest
import torch

import oracle
from paper_2312_00720_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VARIANTS = ["nphj", "phj_tr", "phj_ur"]


def run_jg(gj, w, gk, aggs, agg_cols, variant, **kw):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    okeys, outs, ng = gj.join_groupby(dev(w["rkey"]), [dev(c) for c in w["rcols"]], dev(w["skey"]),
                                      [dev(c) for c in w["scols"]], gk, aggs, agg_cols, variant=variant, **kw)
    g = int(ng.item())
    return np.stack([okeys[:g].cpu().numpy()] + [o[:g].cpu().numpy() for o in outs], 1) if g else \
        np.zeros((0, 1 + len(aggs)), dtype=np.int64)


def want(w, gk, aggs, agg_cols):
    return oracle.canonical(oracle.join_groupby(
        w["rkey"], w["rcols"], w["skey"], w["scols"], g_side=gk[0], g_col=gk[1], g_mod=gk[2], aggs=aggs,
        agg_side=[a[0] for a in agg_cols], agg_col=[a[1] for a in agg_cols]))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nr,ns,mr,theta", [(1, 1, 1.0, 0.0), (1000, 0, 1.0, 0.0), (0, 1000, 1.0, 0.0),
                                            (5000, 20000, 1.0, 0.0), (20000, 80000, 0.6, 1.0),
                                            (100000, 400003, 1.0, 0.5)])
@pytest.mark.parametrize("gk", [(0, 0, 1024), (1, 1, 37), (0, -1, 0), (1, 0, 0), (0, 1, 3)])
def test_join_groupby_matches_oracle(gj, variant, nr, ns, mr, theta, gk):
    w = wl.join_workload(nr, ns, 2, 2, theta=theta, mr=mr, seed=nr + 7 * ns)
    aggs = ["sum", "count", "min", "max"]
    agg_cols = [(1, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)]
    got = oracle.canonical(run_jg(gj, w, gk, aggs, agg_cols, variant))
    exp = want(w, gk, aggs, agg_cols)
    assert got.shape == exp.shape
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("variant", VARIANTS)
def test_int64_keys_negative_group_values(gj, variant):
    rng = np.random.default_rng(5)
    nr, ns = 3000, 9000
    rkey = rng.permutation(np.unique(rng.integers(-(2**60), 2**60, nr + 50, dtype=np.int64)))[:nr]
    skey = rkey[rng.integers(0, nr, ns)]
    w = {"rkey": rkey, "skey": skey, "rcols": [rng.integers(-1000, 1000, nr).astype(np.int32)],
         "scols": [rng.integers(-(2**40), 2**40, ns, dtype=np.int64)]}
    gk = (0, 0, 17)   # residues of negative values are negative: keys in (-17, 17)
    aggs = ["sum", "max", "count"]
    agg_cols = [(1, 0, 0), (1, 0, 0), (0, 0, 0)]
    got = oracle.canonical(run_jg(gj, w, gk, aggs, agg_cols, variant))
    assert np.array_equal(got, want(w, gk, aggs, agg_cols))


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_query_full_size(gj, variant):
    """|R| = 2^20, |S| = 2^22, GROUP BY R.pay mod 1024, SUM/COUNT(S.pay) in int64."""
    w = wl.join_groupby_workload()
    gk = (0, 0, 1024)
    aggs = ["sum", "count"]
    agg_cols = [(1, 0, 0), (1, 0, 0)]
    got = oracle.canonical(run_jg(gj, w, gk, aggs, agg_cols, variant))
    exp = want(w, gk, aggs, agg_cols)
    assert np.array_equal(got, exp)
    assert got[:, 2].sum() == 1 << 22
    assert got[:, 1].sum() == w["scols"][0].astype(np.int64).sum()
