"""Batched construction (thousands of key sets of uneven sizes built by one
launch sequence) and its autotuner, against the CPU oracle.

The autotuner only picks speed knobs and, per set, the expected partition size
P in {1024, 2500, 4096}; every set's structure must then be the oracle's build
of that set alone with the same P, word for word."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# the batched benchmark's workload: 4096 sets, sizes log-uniform in [1e3, 1e7]
BATCH_SETS, BATCH_LO, BATCH_HI, BATCH_SEED, KEY_SEED = 4096, 1e3, 1e7, 2024, 11


@pytest.fixture(scope="module")
def ph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


def _decade(n: int) -> int:
    return len(str(int(n))) - 1


def _check_sampled_sets(ph, orc, hs, off, Ps, sample, key_seed, enc):
    from paper_2404_18497_b300 import workloads
    from tests.test_gpu_parity import compare_structure

    for s in sample:
        n = int(off[s + 1] - off[s])
        ks = workloads.stream_keys(int(off[s]), n, key_seed)
        o = orc.Oracle(ks, lam=7.0, alpha=0.99, P=int(Ps[s]), encoder=enc, threads=0)
        assert np.array_equal(hs[s].pilots().cpu().numpy().view(np.uint32), o.pilots), s
        compare_structure(ph, o, hs[s], enc)
        q = ks[:: max(1, n // 50_000)]
        got = hs[s].query(torch.from_numpy(q.view(np.int64)).cuda()).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, o.query(q)), s


def test_stream_keys_device_equals_host(ph):
    from paper_2404_18497_b300 import workloads

    d = workloads.stream_keys_torch(1_000_003, 300_001, 9, "cuda", chunk=65_536)
    assert np.array_equal(d.cpu().numpy().view(np.uint64), workloads.stream_keys(1_000_003, 300_001, 9))


def test_tuner_choices_cache_and_exactness(ph, orc):
    from paper_2404_18497_b300 import workloads

    off = workloads.batch_sets(300, 1e3, 3e5, 77)
    sizes = np.diff(off)
    prm = ph.make_params(7.0, 0.99, 2500, encoder=1, keep_pilots=True)
    ph.phobic_tune_clear()
    Ps, p2, info = ph.phobic_tune_batch(off, prm)
    assert set(Ps.tolist()) <= {1024, 2500, 4096}
    assert p2.warps_per_partition in (1, 2, 4) and p2.candidate_width in (32, 64)
    # the schedule: the faster of one CTA per partition (1) and the work queue (2)
    sn = info["schedule_ns_per_key"]
    assert p2.search_schedule == (1 if sn["cta_per_partition"] < sn["work_queue"] else 2) == info["search_schedule"]
    assert p2.lambda_ == prm.lambda_ and p2.alpha == prm.alpha and p2.encoder == 1 and p2.keep_pilots == 1
    for s in range(sizes.size):
        assert Ps[s] == info["classes"][_decade(sizes[s])]["partition_size"]
    for c, ci in info["classes"].items():
        best = min(ci["ns_per_key"].values())
        assert ci["ns_per_key"][ci["partition_size"]] <= best * 1.03 + 1e-9
        assert all(v > 1.4 for v in ci["bits_per_key"].values())  # above log2(e)
    # a second call is answered from the cache with the same choices
    Ps2, p3, info2 = ph.phobic_tune_batch(off, prm)
    assert np.array_equal(Ps, Ps2)
    assert (p3.warps_per_partition, p3.candidate_width, p3.search_schedule) == (
        p2.warps_per_partition, p2.candidate_width, p2.search_schedule)
    assert info2["cached_launch"] == 1 and info2["cached_classes"] == len(info["classes"])

    keys = workloads.stream_keys_torch(0, int(off[-1]), 5, "cuda")
    hs = ph.phobic_build_batch(keys, off, p2, partition_sizes=Ps)
    for s, h in enumerate(hs):
        assert ph.phobic_get_info(h)["partition_size"] == Ps[s]
    rng = np.random.default_rng(1)
    _check_sampled_sets(ph, orc, hs, off, Ps, sorted(rng.choice(sizes.size, 10, replace=False)), 5, 1)
    for h in hs:
        h.free()


def test_batch_full_size(ph, orc):
    """The batched benchmark's workload in the launch configuration bench.py
    times: 4096 sets (about 4.45e9 keys), lambda 7, alpha 0.99, IC-D, autotuned.
    Sampled sets are rebuilt by the oracle and must match word for word; for
    every set, the answers for all of its keys are a permutation of [0, n_s)."""
    from paper_2404_18497_b300 import workloads

    off = workloads.batch_sets(BATCH_SETS, BATCH_LO, BATCH_HI, BATCH_SEED)
    sizes = np.diff(off)
    total = int(off[-1])
    prm = ph.make_params(7.0, 0.99, 2500, encoder=1, keep_pilots=True)
    Ps, p2, _ = ph.phobic_tune_batch(off, prm)
    keys = workloads.stream_keys_torch(0, total, KEY_SEED, "cuda")
    hs = ph.phobic_build_batch(keys, off, p2, partition_sizes=Ps)
    ph.phobic_trim(0)
    rng = np.random.default_rng(3)
    small = np.flatnonzero(sizes <= 200_000)
    sample = set(rng.choice(small, 8, replace=False).tolist())
    sample.add(int(np.argmin(np.abs(sizes.astype(np.float64) - 1e6))))
    sample.add(int(np.argmax(sizes)))
    _check_sampled_sets(ph, orc, hs, off, Ps, sorted(sample), KEY_SEED, 1)

    seen = torch.zeros(total, dtype=torch.bool, device="cuda")
    maxima = []
    for s, h in enumerate(hs):
        a, b = int(off[s]), int(off[s + 1])
        out = h.query(keys[a:b])
        maxima.append(out.max())
        seen[out + a] = True
    assert bool(torch.all(torch.stack(maxima).cpu() < torch.from_numpy(sizes.astype(np.int64))))
    assert bool(seen.all())
    for h in hs:
        h.free()
    del keys, seen
    ph.phobic_trim(0)
