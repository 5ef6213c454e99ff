"""The allocation-free radix-partition entry point (for callers that must not
allocate device memory) gives exactly what gj_radix_partition gives, on two calls
in a row, whether this file runs alone or after every other test.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run everything else."""
import numpy as np
import pytest
import torch

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
    d = lambda a: torch.from_numpy(a).cuda()
    return d(key), [d(c) for c in cols]


@pytest.mark.parametrize("key_dtype", [np.int32, np.int64])
def test_noalloc_matches_allocating_entry_point_twice(gj, key_dtype):
    # a large call leaves look-back words behind; the smaller second call must
    # clear what it uses and still match
    for n, lo, hi, tr in ((1_000_003, 0, 8, 2), (70_001, 3, 9, 1)):
        key, cols = _case(n, n, key_dtype)
        want_k, want_c, want_off = gj.radix_partition(key, cols, lo, hi, tr, offsets=True)
        got_k, got_c, got_off = gj.radix_partition_noalloc(key, cols, lo, hi, tr, offsets=True)
        assert torch.equal(got_k, want_k)
        assert all(torch.equal(a, b) for a, b in zip(got_c, want_c))
        assert torch.equal(got_off, want_off)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(gj):
    key, cols = _case(1000, 1, np.int32)
    with pytest.raises(gj.GjError) as e:
        gj.radix_partition_noalloc(key, cols, 0, 9, 0)     # two passes would be needed
    assert e.value.code == 2
    big = torch.zeros((1 << 21) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(gj.GjError) as e:
        gj.radix_partition_noalloc(big, [], 0, 8, 0)
    assert e.value.code == 2
