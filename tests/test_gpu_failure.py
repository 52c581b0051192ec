"""Failure detection without a GPU fault: the partition sort's look-back waits
are bounded.  A tile that never publishes its state (a flag that nothing sets)
makes the next tiles' waits run out after a few polls; the kernel records a
timeout, finishes, and the call returns TIMEOUT.  The context must stay usable:
the same sort without the muted tile, and a full build, still give exact
results afterwards."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


def test_lookback_wait_runs_out_and_context_survives(ph, orc):
    from paper_2404_18497_b300 import workloads

    n, P = 2_000_000, 2500  # 326 sort tiles of 6144 keys: every muted tile below exists
    np_ = (n + P - 1) // P
    keys = workloads.distinct_u64(n, 61)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    hk = ph.phobic_hash_u64(dk, 0)
    ref_sorted, ref_start = ph.phobic_partition_sort(hk, np_)
    for mute in (0, 10, 200):
        t0 = time.time()
        code = ph.phobic_selftest_sort_wait_timeout(hk, np_, mute, 1000)
        assert code == 7, (mute, ph.STATUS_NAMES.get(code))  # TIMEOUT
        assert time.time() - t0 < 20
    # no muted tile: the bounded wait is never reached and the result is the normal sort
    assert ph.phobic_selftest_sort_wait_timeout(hk, np_, 1 << 40, 1000) == 0
    # the context still works: the normal sort and a build are exact
    s2, st2 = ph.phobic_partition_sort(hk, np_)
    assert torch.equal(st2, ref_start)
    assert torch.equal(torch.sort(s2).values, torch.sort(ref_sorted).values)
    o = orc.Oracle(keys, lam=7.0, alpha=1.0, P=P, threads=0)
    h = ph.phobic_build_ex(dk, ph.make_params(7.0, 1.0, P, keep_pilots=True))
    assert np.array_equal(h.pilots().cpu().numpy().view(np.uint32), o.pilots)
    h.free()
    assert ph.phobic_selftest_sort_wait_timeout(hk, np_, 0, 0) == 1  # spin_limit 0 is rejected
