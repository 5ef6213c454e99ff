"""Seeded synthetic workloads for the join and group-by operators.

This module only draws inputs. It holds none of the operators' arithmetic, so the
CUDA library and the CPU oracle can both be fed from it without sharing any
computation. Every generator is deterministic in its seed.

Workload shapes follow the paper's experimental setup:

* join keys: R.key is a seeded permutation of 0..|R|-1 (Sec. 5.1.1); S.key is
  drawn from R's keys uniformly or with a Zipf law (Sec. 5.1.7, P(rank r) ~ r^-theta);
  a match ratio below one replaces exactly round((1-mr)|S|) foreign keys by
  values outside R's key range (Sec. 5.1.6, "Match Ratio");
* group keys: uniform over the domain {0..g-1} (Sec. 5.2.1) or Zipf over it
  (Sec. 5.2.7); 8-byte keys are a bijective 64-bit mix of the 4-byte domain id so
  that every key bit is live;
* payload / value columns: uniform integers.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed & 0xFFFFFFFF, seed >> 32, stream])))


def mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finalizer (Steele, Lea, Flood 2014): a bijection on 64-bit words."""
    z = x.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def zipf_ranks(m: int, n: int, theta: float, seed: int, stream: int) -> np.ndarray:
    """m samples of ranks in [0, n) with P(rank r) proportional to (r+1)^-theta.

    Inverse-CDF sampling with a guide table (Chen & Asau 1974): bucket j of the
    unit interval points at the first rank whose CDF exceeds j/n, and a short
    forward walk finishes the search. theta = 0 is the uniform law.
    """
    rng = _rng(seed, stream)
    if m == 0:
        return np.zeros(0, dtype=np.int64)
    if theta == 0.0:
        return rng.integers(0, n, size=m, dtype=np.int64)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-float(theta))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    guide = np.searchsorted(cdf, np.arange(n, dtype=np.float64) / n, side="right")
    u = rng.random(m)
    idx = guide[np.minimum((u * n).astype(np.int64), n - 1)]
    pending = np.nonzero(cdf[idx] <= u)[0]
    while pending.size:
        idx[pending] += 1
        pending = pending[cdf[idx[pending]] <= u[pending]]
    return idx


def join_workload(nr: int, ns: int, ncols_r: int, ncols_s: int, *, theta: float = 0.0,
                  mr: float = 1.0, key_dtype=np.int32, col_dtype=np.int32, seed: int = 1):
    """FK-PK join inputs R(key, r1..), S(key, s1..) as numpy columns.

    R.key: seeded permutation of 0..nr-1. S.key: R.key[rank] with rank uniform
    (theta = 0) or Zipf(theta); exactly round((1-mr)*ns) seeded S rows get keys
    uniform in [nr, 2^31) so they match nothing and |T| = ns - that count.
    Payloads are uniform in [0, 2^31).
    """
    rng = _rng(seed, 0)
    rkey = rng.permutation(nr).astype(key_dtype)
    if nr:
        ranks = zipf_ranks(ns, nr, theta, seed, 1)
        skey = rkey[ranks].astype(key_dtype)
    else:
        skey = np.zeros(ns, dtype=key_dtype)
    n_miss = int(round((1.0 - mr) * ns)) if nr else ns
    if n_miss:
        r2 = _rng(seed, 2)
        miss = np.argpartition(r2.random(ns), n_miss - 1)[:n_miss] if n_miss < ns else np.arange(ns)
        skey[miss] = r2.integers(max(nr, 0), 2**31, size=n_miss).astype(key_dtype)
    rcols = [_rng(seed, 10 + c).integers(0, 2**31, size=nr, dtype=np.int64).astype(col_dtype)
             for c in range(ncols_r)]
    scols = [_rng(seed, 20 + c).integers(0, 2**31, size=ns, dtype=np.int64).astype(col_dtype)
             for c in range(ncols_s)]
    return {"rkey": rkey, "rcols": rcols, "skey": skey, "scols": scols, "n_match": ns - n_miss}


def mn_join_workload(nr: int, ns: int, nk: int, ncols_r: int = 2, ncols_s: int = 2, *, key_dtype=np.int32,
                     col_dtype=np.int32, seed: int = 13):
    """Many-to-many join inputs: R.key and S.key drawn uniformly from a seeded set
    of nk distinct keys (Sec. 5.1.9, many-to-many joins); payloads uniform in [0, 2^31)."""
    keys = _rng(seed, 0).permutation(max(nk, 1) * 4)[:max(nk, 1)].astype(key_dtype)
    rkey = keys[_rng(seed, 1).integers(0, max(nk, 1), size=nr)]
    skey = keys[_rng(seed, 2).integers(0, max(nk, 1), size=ns)]
    rcols = [_rng(seed, 10 + c).integers(0, 2**31, size=nr, dtype=np.int64).astype(col_dtype)
             for c in range(ncols_r)]
    scols = [_rng(seed, 20 + c).integers(0, 2**31, size=ns, dtype=np.int64).astype(col_dtype)
             for c in range(ncols_s)]
    return {"rkey": rkey, "rcols": rcols, "skey": skey, "scols": scols}


def groupby_workload(n: int, g: int, *, nvals: int = 3, key_dtype=np.int32, theta: float = 0.0,
                     seed: int = 3, lo: int = -(2**20), hi: int = 2**20):
    """Group-by input R(k, r1..r_nvals): keys from a domain of g ids, values uniform in [lo, hi).

    Uniform keys are the domain id itself; Zipf keys map rank -> a seeded
    permutation of the domain so hot keys are not adjacent. 8-byte keys are
    mix64(id), which keeps the group structure but makes all 64 bits live.
    """
    ids = zipf_ranks(n, g, theta, seed, 1)
    if theta != 0.0:
        ids = _rng(seed, 2).permutation(g)[ids]
    if np.dtype(key_dtype) == np.int64:
        keys = mix64(ids.astype(np.uint64)).view(np.int64)
    else:
        keys = ids.astype(np.int32)
    vals = [_rng(seed, 10 + c).integers(lo, hi, size=n, dtype=np.int64).astype(np.int32) for c in range(nvals)]
    return {"key": keys, "vals": vals}


def join_groupby_workload(nr: int = 1 << 20, ns: int = 1 << 22, seed: int = 5):
    """One query: FK-PK join with one int32 payload per side, every S row matching once."""
    return join_workload(nr, ns, 1, 1, theta=0.0, mr=1.0, seed=seed)


def batch_sizes(nq: int = 512, *, log_r_lo: float = 10.0, log_r_hi: float = 20.0,
                log_g_lo: float = 2.0, log_g_hi: float = 16.0, seed: int = 7):
    """(|R|, group modulus) of each batched instance: both log-uniform."""
    rng = _rng(seed, 0)
    lr = rng.uniform(log_r_lo, log_r_hi, size=nq)
    lg = rng.uniform(log_g_lo, log_g_hi, size=nq)
    return [(int(round(2.0 ** a)), int(round(2.0 ** b))) for a, b in zip(lr, lg)]


def batch_workload(nq: int = 512, *, log_r_lo: float = 10.0, log_r_hi: float = 20.0,
                   log_g_lo: float = 2.0, log_g_hi: float = 16.0, s_factor: int = 4, seed: int = 7):
    """Instances for the batched path: |R| log-uniform, |S| = s_factor |R|, uniform FK,
    two int32 payloads per side, group cardinality log-uniform (returned as the modulus)."""
    out = []
    sizes = batch_sizes(nq, log_r_lo=log_r_lo, log_r_hi=log_r_hi, log_g_lo=log_g_lo, log_g_hi=log_g_hi, seed=seed)
    for i, (nr, modulus) in enumerate(sizes):
        w = join_workload(nr, s_factor * nr, 2, 2, seed=seed * 100003 + i)
        w["modulus"] = modulus
        out.append(w)
    return out
