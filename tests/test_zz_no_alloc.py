"""The allocation-free radix-partition entry point (for callers that must not
allocate device memory) against the oracle's stable partition and against
gj_radix_partition, on two calls in a row, whether this file runs alone or after
every other test.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run everything else."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _case(n, seed, key_dtype):
    rng = np.random.default_rng(seed)
    if key_dtype == np.int32:
        key = rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32)
    else:
        key = rng.integers(-(2**63), 2**63 - 1, n, dtype=np.int64)
    if n > 3:
        key[::7] = key[3]  # repeated keys make stability observable
    cols = [rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32),
            rng.integers(-(2**62), 2**62, n, dtype=np.int64)]
    return key, cols


@pytest.mark.parametrize("key_dtype", [np.int32, np.int64])
def test_noalloc_matches_oracle_and_allocating_entry_point_twice(gj, key_dtype):
    # the first call covers many tiles and digits; the smaller second call finds the
    # first call's offsets and totals in the shared array and must clear what it uses
    kb = 4 if key_dtype == np.int32 else 8
    for n, lo, hi, tr in ((1_000_003, 0, 8, 2), (70_001, 3, 9, 1)):
        key, cols = _case(n, n, key_dtype)
        perm, offs = oracle.radix_partition(key, kb, lo, hi, tr)
        d = lambda a: torch.from_numpy(a).cuda()
        got_k, got_c, got_off = gj.radix_partition_noalloc(d(key), [d(c) for c in cols], lo, hi, tr, offsets=True)
        assert np.array_equal(got_k.cpu().numpy(), key[perm])
        for g, c in zip(got_c, cols):
            assert np.array_equal(g.cpu().numpy(), c[perm])
        assert np.array_equal(got_off.cpu().numpy(), offs)
        want_k, want_c, want_off = gj.radix_partition(d(key), [d(c) for c in cols], lo, hi, tr, offsets=True)
        assert torch.equal(got_k, want_k) and torch.equal(got_off, want_off)
        assert all(torch.equal(a, b) for a, b in zip(got_c, want_c))


def test_noalloc_empty_input_synchronises_and_reports(gj):
    # a sync = 1 call with no rows takes the same status path as any other call
    key, cols = _case(200_000, 3, np.int32)
    d = lambda a: torch.from_numpy(a).cuda()
    gj.radix_partition_noalloc(d(key), [d(c) for c in cols], 0, 8, 2, sync=False)
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    _, _, off = gj.radix_partition_noalloc(empty, [], 0, 6, 0, offsets=True, sync=True)
    assert np.array_equal(off.cpu().numpy(), np.zeros(65, dtype=np.int64))


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(gj):
    key, cols = _case(1000, 1, np.int32)
    d = lambda a: torch.from_numpy(a).cuda()
    with pytest.raises(gj.GjError) as e:
        gj.radix_partition_noalloc(d(key), [d(c) for c in cols], 0, 9, 0)     # two passes would be needed
    assert e.value.code == 2
    big = torch.zeros((1 << 21) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(gj.GjError) as e:
        gj.radix_partition_noalloc(big, [], 0, 8, 0)
    assert e.value.code == 2
    # the largest accepted input: 2^21 rows
    key, cols = _case(1 << 21, 5, np.int32)
    perm, offs = oracle.radix_partition(key, 4, 0, 8, 2)
    got_k, _, got_off = gj.radix_partition_noalloc(d(key), [], 0, 8, 2, offsets=True)
    assert np.array_equal(got_k.cpu().numpy(), key[perm])
    assert np.array_equal(got_off.cpu().numpy(), offs)
