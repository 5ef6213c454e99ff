"""Failure paths without a GPU fault: bounded device-side waits that run out
(flags that nothing sets, and a product kernel run with a tiny wait limit) return
GJ_ERR_TIMEOUT and leave the context usable; an allocator hook that refuses an
allocation makes the call return GJ_ERR_OOM with nothing left allocated."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2312_00720_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TIMEOUT, OOM = 6, 3


def _small_join_is_exact(gj, variant="phj_tr"):
    w = wl.join_workload(3000, 12000, 2, 1, theta=0.5, mr=0.8, seed=11)
    d = lambda a: torch.from_numpy(a).cuda()
    tk, tc, cnt = gj.join(d(w["rkey"]), [d(c) for c in w["rcols"]], d(w["skey"]), [d(c) for c in w["scols"]],
                          variant=variant)
    m = int(cnt.item())
    got = np.stack([tk[:m].cpu().numpy()] + [c[:m].cpu().numpy() for c in tc], 1).astype(np.int64)
    want = oracle.join(w["rkey"], w["rcols"], w["skey"], w["scols"])
    return np.array_equal(oracle.canonical(got), oracle.canonical(want))


@pytest.mark.parametrize("kind", [0, 2])
def test_wait_on_other_blocks_times_out_at_the_set_limit(gj, kind):
    # kind 0: the warp-wide look-back, kind 2: the batched mode's task counter
    gj.set_wait_limit(20_000_000)  # 20 ms
    try:
        t0 = time.perf_counter()
        st = gj.check_bounded_wait(kind)
        dt = time.perf_counter() - t0
    finally:
        gj.set_wait_limit(0)
    assert st == TIMEOUT
    assert dt < 1.5, f"a 20 ms wait limit took {dt:.2f} s"
    assert gj.device_status() == 0          # the status was returned and cleared
    assert _small_join_is_exact(gj)         # the context is still usable


def test_bulk_copy_wait_keeps_its_fixed_limit(gj):
    # kind 1: an mbarrier nothing arrives at; a block's wait for its own copies keeps
    # the 2 s default whatever limit is set
    gj.set_wait_limit(1_000_000)
    try:
        t0 = time.perf_counter()
        st = gj.check_bounded_wait(1)
        dt = time.perf_counter() - t0
    finally:
        gj.set_wait_limit(0)
    assert st == TIMEOUT
    assert 1.5 < dt < 10.0
    assert _small_join_is_exact(gj)


def test_default_limit_is_about_two_seconds(gj):
    t0 = time.perf_counter()
    st = gj.check_bounded_wait(0)
    dt = time.perf_counter() - t0
    assert st == TIMEOUT and 1.5 < dt < 10.0


@pytest.mark.parametrize("variant", ["phj_tr", "nphj"])
def test_product_kernels_finish_under_a_tiny_wait_limit(gj, variant):
    # a multi-unit probe whose look-back waits give up after a nanosecond: the kernel
    # returns (writes stay inside the output buffers), the status is OK or TIMEOUT,
    # and with the default limit restored the same join is exact again
    w = wl.join_workload(1 << 18, 1 << 22, 1, 1, seed=5)
    d = lambda a: torch.from_numpy(a).cuda()
    args = (d(w["rkey"]), [d(w["rcols"][0])], d(w["skey"]), [d(w["scols"][0])])
    gj.set_wait_limit(1)
    try:
        gj.join(*args, variant=variant, sync=False)
        torch.cuda.synchronize()
        st = gj.device_status()
    finally:
        gj.set_wait_limit(0)
    print(f"{variant} under a 1 ns wait limit: status {st}")
    assert st in (0, TIMEOUT)
    tk, tc, cnt = gj.join(*args, variant=variant)
    assert int(cnt.item()) == len(w["skey"])
    assert _small_join_is_exact(gj, variant)


class _Hook:
    """Scratch allocator through torch's caching allocator that refuses the n-th
    allocation and tracks what is still outstanding."""

    def __init__(self):
        self.calls = 0
        self.fail_at = None
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes)
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "freed an address the hook never gave out"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


@pytest.mark.parametrize("op", ["join_phj_tr", "join_smj_tr", "groupby_sgb", "groupby_pgb", "join_groupby"])
def test_refused_allocation_returns_oom_and_frees_the_rest(gj, op):
    w = wl.join_workload(5000, 20000, 2, 2, seed=3)
    d = lambda a: torch.from_numpy(a).cuda()
    rk, rc, sk, sc = d(w["rkey"]), [d(c) for c in w["rcols"]], d(w["skey"]), [d(c) for c in w["scols"]]

    def call():
        if op.startswith("join_groupby"):
            return gj.join_groupby(rk, rc, sk, sc, (0, 0, 64), ["sum", "count"], [(1, 0, 0), (1, 0, 0)],
                                   variant="phj_tr")
        if op.startswith("join_"):
            return gj.join(rk, rc, sk, sc, variant=op[5:])
        return gj.groupby(sk, sc, ["count", "sum", "max"], [0, 0, 1], variant=op[8:])

    hook = _Hook()
    gj.set_allocator(hook.alloc, hook.free)
    try:
        call()
        torch.cuda.synchronize()
        n = hook.calls
        assert n >= 2 and not hook.live
        for k in range(1, n + 1):
            hook.calls, hook.fail_at = 0, k
            with pytest.raises(gj.GjError) as e:
                call()
            assert e.value.code == OOM
            torch.cuda.synchronize()
            assert not hook.live, f"allocation {k} refused: {len(hook.live)} blocks not freed"
    finally:
        gj.set_allocator()
    assert gj.device_status() == 0
    assert _small_join_is_exact(gj)
