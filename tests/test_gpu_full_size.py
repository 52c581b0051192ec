"""Parity at the full benchmark size: 1e8 keys, lambda 7, alpha 0.99, P 2500,
interleaved dictionary encoding, in the launch configuration bench.py times.

The oracle builds all 1e8 keys on the host cores (OpenMP over partitions; about a
minute).  Every pilot, every packed word, bits/key, and the queries of a
2e6-key sample must then be identical to the CUDA path.  The GPU's answers for
all 1e8 keys must form a permutation of [0, n)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

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
    from tests.test_gpu_parity import compare_structure

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
