"""The N > 1 path on CPU: two gloo ranks, as bench.py runs them under torchrun.

Key sets are independent problems, so each rank builds its own (seed 2 + 1000 r)
with no collective on the data path; the ranks only meet in a barrier and a max
of their timings.  Here the oracle stands in for the device build; what is
checked is the host-side logic: distinct per-rank key sets, every rank's result
a bijection onto [0, n), the max over ranks, and the aggregate throughput
(all ranks' keys over the slowest rank's time)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out_dir):
    import torch.distributed as dist

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    from oracle import oracle as o
    from paper_2404_18497_b300 import workloads

    w, r, _ = bench.dist_env()
    assert (w, r) == (world, rank)
    keys = workloads.distinct_u64(n, 2 + 1000 * rank)  # the benchmark's per-rank key set
    bench.barrier(world)
    h = o.Oracle(keys, lam=7.0, alpha=0.99, P=2500, encoder=1, threads=1)
    pos = h.query(keys)
    my_time = 0.25 + 0.5 * rank  # a fixed per-rank "duration" to check the reduction
    slowest = bench.reduce_max(my_time, world)
    bench.barrier(world)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([slowest, int(np.array_equal(np.sort(pos), np.arange(n, dtype=np.uint64))),
                      int(keys[:4].sum() % (1 << 40))], dtype=np.float64))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    import torch.multiprocessing as mp

    world, n = 2, 20_000
    mp.spawn(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert all(x[0] == 0.75 for x in res)  # max over ranks reached every rank
    assert all(x[1] == 1 for x in res)     # each rank's MPHF is a bijection onto [0, n)
    assert res[0][2] != res[1][2]          # the ranks built different key sets
    # bench.py's aggregate: every rank's keys over the slowest rank's time
    assert world * n / res[0][0] == pytest.approx(2 * 20_000 / 0.75)
