"""The partition-sharded build on a GPU: G virtual shards, one host thread and
one CUDA stream each, run the orchestration of paper_2404_18497_b300/shard.py
with the library's stages (hash, partition sort, table offsets, search of a
partition range, assembly).  Their exchanges go through host memory here
(ThreadComm) instead of NCCL; no kernel waits on another shard's.  Every
shard must end with the structure phobic_build_ex makes from all keys on one
device: the same export bytes."""
import threading

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


class ThreadComm:
    """In-process exchanges between G threads (test transport)."""

    class Hub:
        def __init__(self, world):
            self.world = world
            self.bar = threading.Barrier(world)
            self.slot = [None] * world

    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def _swap(self, item):
        torch.cuda.synchronize()
        self.hub.slot[self.rank] = item
        self.hub.bar.wait()
        got = list(self.hub.slot)
        self.hub.bar.wait()
        return got

    def all_gather_int(self, v):
        return [int(x) for x in self._swap(int(v))]

    def all_to_all(self, send, counts):
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        parts = self._swap([send[offs[q]:offs[q + 1]] for q in range(self.world)])
        return torch.cat([parts[q][self.rank] for q in range(self.world)]).contiguous()

    def all_gather_v(self, t, counts):
        parts = self._swap(t)
        return torch.cat([p[:c] for p, c in zip(parts, counts)]).contiguous()

    def all_reduce_sum_(self, t):
        parts = self._swap(t.clone())
        acc = parts[0].clone()
        for p in parts[1:]:
            acc += p
        t.copy_(acc)
        torch.cuda.synchronize()
        self.hub.bar.wait()

    def all_reduce_max_int(self, v):
        return max(self._swap(int(v)))


def _run_shards(ph, keys, params, world, cuts):
    from paper_2404_18497_b300 import shard

    hub = ThreadComm.Hub(world)
    out, err = [None] * world, [None] * world

    def body(r):
        s = torch.cuda.Stream()
        try:
            with torch.cuda.stream(s):
                mine = keys[cuts[r]:cuts[r + 1]].contiguous()
                h = shard.sharded_build(mine, params, ThreadComm(hub, r), shard.DeviceStages(s))
                out[r] = h.export()
                h.free()
        except Exception as e:  # reported by the test below
            err[r] = e
            hub.bar.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out, err


CASES = [
    # n, lambda, alpha, P, encoder, mode, shards
    (1_000_000, 7.0, 0.99, 2500, "IC-D", "additive", 2),
    (300_001, 7.0, 1.0, 2500, "IC-C", "additive", 3),
    (200_000, 6.0, 0.97, 1000, "IC-R", "xor", 2),
    (50_000, 7.0, 0.9, 2500, "IC-EF", "additive", 4),
    (3_000, 7.0, 0.99, 2500, "IC-D", "additive", 4),  # 2 partitions over 4 shards
]


@pytest.mark.parametrize("n,lam,alpha,P,enc,mode,world", CASES)
def test_sharded_build_exports_the_single_build(ph, n, lam, alpha, P, enc, mode, world):
    from paper_2404_18497_b300 import workloads

    keys = workloads.stream_keys_torch(0, n, 77, "cuda")
    prm = ph.make_params(lam, alpha, P, seed=9, encoder=enc, mode=mode)
    ref = ph.phobic_build_ex(keys, prm)
    want = ref.export()
    ref.free()
    rng = np.random.default_rng(n)
    cuts = np.concatenate([[0], np.sort(rng.integers(0, n + 1, size=world - 1)), [n]])
    out, err = _run_shards(ph, keys, prm, world, cuts)
    assert err == [None] * world, err
    for r in range(world):
        assert out[r] == want, r


def test_sharded_build_at_1e8_keys(ph):
    """The 1e8-key, lambda 7, alpha 0.99, IC-D workload split over two shards."""
    from paper_2404_18497_b300 import workloads

    n = 100_000_000
    keys = workloads.stream_keys_torch(0, n, 2, "cuda")
    prm = ph.make_params(7.0, 0.99, 2500, seed=1, encoder="IC-D")
    ref = ph.phobic_build_ex(keys, prm)
    want = ref.export()
    ref.free()
    out, err = _run_shards(ph, keys, prm, 2, [0, 40_000_000, n])
    assert err == [None, None], err
    assert out[0] == want and out[1] == want


def test_search_of_a_partition_range(ph):
    """phobic_search_partitions over [j0, j1) writes exactly those partitions'
    pilots (the whole build's values) and leaves the rest untouched."""
    from paper_2404_18497_b300 import workloads

    n, P = 400_000, 2500
    keys = workloads.stream_keys_torch(0, n, 5, "cuda")
    prm = ph.make_params(7.0, 0.99, P, seed=3, encoder="IC-C", keep_pilots=True)
    ref = ph.phobic_build_ex(keys, prm)
    want = ref.pilots().cpu().numpy().view(np.uint32)
    ref.free()
    NP = (n + P - 1) // P
    B = -(-P // 7)
    hk = ph.phobic_hash_u64(keys, 3)
    srt, start = ph.phobic_partition_sort(hk, NP)
    T, (M, _, _) = ph.phobic_table_offsets(start, 0.99)
    j0, j1 = 37, 101
    pil = torch.full((B * NP,), -1, dtype=torch.int32, device="cuda")
    pil.view(B, NP)[:, j0:j1] = 0
    ph.phobic_search_partitions(srt, start, T, n, NP, j0, j1, prm, pil, None)
    got = pil.cpu().numpy().view(np.uint32).reshape(B, NP)
    assert np.array_equal(got[:, j0:j1], want.reshape(B, NP)[:, j0:j1])
    assert (got[:, :j0] == 0xFFFFFFFF).all() and (got[:, j1:] == 0xFFFFFFFF).all()
    with pytest.raises(ph.PhobicError):  # a partition count that is not ceil(n / P)
        ph.phobic_search_partitions(srt, start, T, n, NP + 1, j0, j1, prm, pil, None)
    with pytest.raises(ph.PhobicError):  # starts that do not end at n
        bad = start.clone()
        bad[-1] += 1
        ph.phobic_assemble(bad, n, pil, None, prm)
