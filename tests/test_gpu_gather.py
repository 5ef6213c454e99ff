"""The gather primitive (Sec. 2.3) through the C-ABI vs the oracle's gather:
clustered and unclustered maps, 4- and 8-byte elements, ragged sizes, and an
out-of-range index reported as an argument error on the device."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [0, 1, 1023, 4097, 300001])
@pytest.mark.parametrize("dtype", [np.int32, np.int64])
@pytest.mark.parametrize("clustered", [True, False])
def test_gather_matches_oracle(gj, n, dtype, clustered):
    rng = np.random.default_rng(n)
    n_in = max(1, n + 17)
    src = rng.integers(-(2**31), 2**31, n_in).astype(dtype)
    idx = (np.sort(rng.integers(0, n_in, n)) if clustered else rng.integers(0, n_in, n)).astype(np.int32)
    got = gj.gather(torch.from_numpy(src).cuda(), torch.from_numpy(idx).cuda())
    assert np.array_equal(got.cpu().numpy(), oracle.gather(src, idx))


def test_out_of_range_index_is_an_argument_error(gj):
    src = torch.arange(100, dtype=torch.int32, device="cuda")
    idx = torch.tensor([3, 100, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(gj.GjError) as e:
        gj.gather(src, idx)
    assert e.value.code == 1
