"""Parity at the full benchmark sizes, in the launch configurations bench.py times:
- 1e8 uint64 keys, lambda 7, alpha 0.99, P 2500, interleaved dictionary encoding;
- 2e8 random strings (lengths uniform in [10, 50] over [A-Za-z0-9], Section 5's
  input), lambda 7.5, alpha 0.99, P 2500, interleaved dictionary encoding.

The oracle builds every key on the host cores (OpenMP over partitions; one to two
minutes each).  Every pilot, every packed word, bits/key, and the queries of a
2e6-key sample must then be identical to the CUDA path.  The GPU's answers for
all keys must form a permutation of [0, n)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from tests.test_gpu_parity import compare_structure

N = 100_000_000


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


def test_full_size_build_and_query(ph, orc):
    from paper_2404_18497_b300 import workloads

    keys = workloads.distinct_u64(N, 2)  # the benchmark's key set
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    prm = ph.make_params(7.0, 0.99, 2500, seed=0, encoder=1, keep_pilots=True)
    h = ph.phobic_build_ex(dk, prm)
    gp = h.pilots().cpu().numpy().view(np.uint32)
    out = h.query(dk)
    # bijection of all 1e8 answers
    srt = torch.sort(out).values
    assert torch.equal(srt, torch.arange(N, device="cuda"))
    del srt
    o = orc.Oracle(keys, lam=7.0, alpha=0.99, P=2500, encoder=1, seed=0, threads=0)
    assert np.array_equal(gp, o.pilots)
    compare_structure(ph, o, h, 1)
    assert h.bits_per_key() == o.bits_per_key()
    sample = np.random.default_rng(5).integers(0, N, size=2_000_000)
    got = out.cpu().numpy().view(np.uint64)[sample]
    assert np.array_equal(got, o.query(keys[sample]))


def test_full_size_strings_build_and_query(ph, orc):
    from paper_2404_18497_b300 import workloads

    n = 200_000_000
    data, off = workloads.random_strings(n, 3)  # the benchmark's strings
    dd = torch.from_numpy(data).cuda()
    do = torch.from_numpy(off.view(np.int64)).cuda()
    # master hashes: XXH64 of every string, on the device and in the oracle
    hk = orc.string_hashes(data, off, 0)
    del data
    assert np.array_equal(ph.phobic_hash_strings(dd, do, 0).cpu().numpy().view(np.uint64), hk)
    prm = ph.make_params(7.5, 0.99, 2500, seed=0, encoder=1, keep_pilots=True)
    h = ph.phobic_build_strings(dd, do, prm)
    gp = h.pilots().cpu().numpy().view(np.uint32)
    out = ph.phobic_query_strings(h, dd, do)
    del dd, do
    srt = torch.sort(out).values
    assert torch.equal(srt, torch.arange(n, device="cuda"))
    del srt
    o = orc.Oracle(hashed=hk, lam=7.5, alpha=0.99, P=2500, encoder=1, seed=0, threads=0)
    assert np.array_equal(gp, o.pilots)
    compare_structure(ph, o, h, 1)
    assert h.bits_per_key() == o.bits_per_key()
    sample = np.random.default_rng(6).integers(0, n, size=2_000_000)
    got = out.cpu().numpy().view(np.uint64)[sample]
    assert np.array_equal(got, o.query_hashed(hk[sample]))
