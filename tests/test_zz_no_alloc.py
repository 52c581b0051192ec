"""The allocation-free partition sort (phobic_partition_sort_noalloc) against
the regular entry point (phobic_partition_sort), through the C ABI.

Some callers may not allocate device memory while they run: for example, a
process whose device budget is reserved up front, or a framework that owns
every allocation.  The no-alloc entry point serves them with one fixed
internal scratch array.  It must give exactly the regular sort's output
(integer data: bit-exact), also on the second of two calls in a row, when
the shared array still holds the first call's contents.  This file is
collected last on purpose: it runs after every other GPU test."""
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


def _hashes(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 2**64, size=n, dtype=np.uint64)
    return torch.from_numpy(x.view(np.int64)).cuda()


def test_noalloc_sort_matches_allocating_sort_twice(ph):
    # two different calls in a row: larger first, then smaller, so stale
    # contents of the shared scratch would show up in the second result
    for n, P, seed in [(1_000_003, 2500, 1), (300_001, 1024, 2)]:
        hk = _hashes(n, seed)
        NP = -(-n // P)
        ref_sorted, ref_start = ph.phobic_partition_sort(hk, NP)
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        start = torch.full((NP + 1,), -1, dtype=torch.int64, device="cuda")
        ph.phobic_partition_sort_noalloc(hk, NP, out, start)
        torch.cuda.synchronize()
        assert torch.equal(start, ref_start)
        assert torch.equal(out, ref_sorted)


def test_noalloc_sort_at_its_maximum_size(ph):
    """n = PHOBIC_NOALLOC_MAX_KEYS with 2^18 partitions: two digit passes of 9
    bits (512 bins), the widest digits the fixed array is sized for, so the
    sort uses all of the array's key, look-back and counter regions (only the
    histogram region keeps room for a third pass)."""
    n = ph.NOALLOC_MAX_KEYS
    NP = 1 << 18
    for seed in (3, 4):
        hk = _hashes(n, seed)
        ref_sorted, ref_start = ph.phobic_partition_sort(hk, NP)
        out = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        start = torch.full((NP + 1,), -1, dtype=torch.int64, device="cuda")
        ph.phobic_partition_sort_noalloc(hk, NP, out, start)
        torch.cuda.synchronize()
        assert torch.equal(start, ref_start)
        assert torch.equal(out, ref_sorted)


def test_noalloc_rejects_too_many_keys(ph):
    n = ph.NOALLOC_MAX_KEYS + 1
    hk = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty_like(hk)
    start = torch.empty(2, dtype=torch.int64, device="cuda")
    with pytest.raises(ph.PhobicError) as e:
        ph.phobic_partition_sort_noalloc(hk, 1, out, start)
    assert e.value.status == "INVALID_ARG"
