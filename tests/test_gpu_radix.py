"""radix-partition (Sec. 2.3) through the C-ABI vs the oracle's stable sort by digit:
bit-exact keys, payload columns and partition offsets."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

TILE = 4096


def _keys(n, key_bytes, seed, dup=True):
    rng = np.random.default_rng(seed)
    if key_bytes == 4:
        k = rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32)
    else:
        k = rng.integers(-(2**63), 2**63 - 1, n, dtype=np.int64)
    if dup and n > 3:
        k[::3] = k[1]
    return k


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 100003])
@pytest.mark.parametrize("lo,hi,transform", [(0, 8, 0), (0, 16, 2), (3, 14, 1), (0, 5, 2)])
def test_partition_matches_stable_sort(gj, n, lo, hi, transform):
    k = _keys(n, 4, seed=n + lo + hi)
    rng = np.random.default_rng(7)
    c32 = rng.integers(-(2**31), 2**31, n, dtype=np.int64).astype(np.int32)
    c64 = rng.integers(-(2**62), 2**62, n, dtype=np.int64)
    perm, offs = oracle.radix_partition(k, 4, lo, hi, transform)
    dk = torch.from_numpy(k).cuda()
    ko, co, off = gj.radix_partition(dk, [torch.from_numpy(c32).cuda(), torch.from_numpy(c64).cuda()],
                                     lo, hi, transform, offsets=True)
    assert np.array_equal(ko.cpu().numpy(), k[perm])
    assert np.array_equal(co[0].cpu().numpy(), c32[perm])
    assert np.array_equal(co[1].cpu().numpy(), c64[perm])
    assert np.array_equal(off.cpu().numpy(), offs)


@pytest.mark.parametrize("n", [1, 5000, 70001])
def test_full_width_signed_sort_int64(gj, n):
    k = _keys(n, 8, seed=n)
    perm, _ = oracle.radix_partition(k, 8, 0, 64, 1)
    ko, co, _ = gj.radix_partition(torch.from_numpy(k).cuda(), [torch.arange(n, dtype=torch.int32).cuda()], 0, 64, 1)
    assert np.array_equal(ko.cpu().numpy(), k[perm])
    assert np.array_equal(ko.cpu().numpy(), np.sort(k, kind="stable"))
    assert np.array_equal(co[0].cpu().numpy(), perm.astype(np.int32))


@pytest.mark.parametrize("bpp", [1, 3, 7, 8])
def test_bits_per_pass_do_not_change_result(gj, bpp):
    n = 20000
    k = _keys(n, 4, seed=bpp)
    perm, offs = oracle.radix_partition(k, 4, 2, 13, 2)
    ko, co, off = gj.radix_partition(torch.from_numpy(k).cuda(), [], 2, 13, 2, offsets=True, bits_per_pass=bpp)
    assert np.array_equal(ko.cpu().numpy(), k[perm])
    assert np.array_equal(off.cpu().numpy(), offs)


def test_all_equal_keys_and_determinism(gj):
    n = 50000
    k = np.full(n, 12345, dtype=np.int32)
    v = np.arange(n, dtype=np.int32)
    outs = [gj.radix_partition(torch.from_numpy(k).cuda(), [torch.from_numpy(v).cuda()], 0, 16, 2) for _ in range(2)]
    assert np.array_equal(outs[0][1][0].cpu().numpy(), v)   # stability: input order kept
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1][0], outs[1][1][0])


def test_large_multi_tile_two_passes(gj):
    n = (1 << 22) + 12345
    k = _keys(n, 4, seed=99, dup=False)
    perm, offs = oracle.radix_partition(k, 4, 0, 16, 2)
    ko, co, off = gj.radix_partition(torch.from_numpy(k).cuda(), [torch.arange(n, dtype=torch.int32).cuda()],
                                     0, 16, 2, offsets=True)
    assert np.array_equal(co[0].cpu().numpy(), perm.astype(np.int32))
    assert np.array_equal(off.cpu().numpy(), offs)
