"""The partition-sharded build (Section 4: partitions are independent, so one
MPHF's construction splits by partition ranges across processes) on CPU: gloo
ranks run the real orchestration of paper_2404_18497_b300/shard.py (owner
ranges, the all-to-all of master hashes, the composition of the build's
partition starts, the merge of pilots and occupancy by summation), with the
oracle standing in for each device stage.  The merged result must be the
single build's: every pilot, the partition starts, and the free-slot remap
that the merged occupancy implies, word for word."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_2404_18497_b300 import shard, workloads
    from tests.shard_stages import OracleStages, remap_from_taken

    n, lam, alpha, P, mode, cuts_seed, dup = (case[k] for k in ("n", "lam", "alpha", "P", "mode", "cuts", "dup"))
    s_max = case.get("s_max", 0)
    keys = workloads.distinct_u64(n, 11)
    if dup:
        keys[-1] = keys[0]  # a duplicate pair on two different ranks
    if cuts_seed >= 0:
        cuts = np.sort(np.random.default_rng(cuts_seed).integers(0, n + 1, size=world - 1))
    else:
        cuts = np.linspace(0, n, world + 1)[1:-1]
    cuts = np.concatenate([[0], cuts.astype(np.int64), [n]])
    mine = torch.from_numpy(keys[cuts[rank]:cuts[rank + 1]].view(np.int64).copy())
    st = OracleStages(orc, lam, alpha, P, mode, s_max)
    prm = type("prm", (), dict(partition_size=P, lambda_=lam, alpha=alpha, seed=5))()
    res = {"rank": rank}
    stats = []
    try:
        # optionally a second gloo group for the integer metadata, as bench.py
        # passes one beside its NCCL group
        comm = shard.TorchComm(cpu_group=dist.new_group(backend="gloo") if case.get("cpu_group") else None)
        out = shard.sharded_build(mine, prm, comm, st, stats_out=stats)
    except orc.OracleError as e:
        res["error"] = e.code
    else:
        ref = orc.Oracle(keys, lam=lam, alpha=alpha, P=P, mode=mode, seed=5, threads=1)
        s = stats[0]
        res["pilots_equal"] = bool(np.array_equal(out["pilots"], ref.array("pilots")))
        res["starts_equal"] = bool(np.array_equal(np.diff(out["start"]), ref.array("part_size").astype(np.int64)))
        res["M_equal"] = s.M == ref.u64("M")
        if out["taken"] is not None:
            fs = remap_from_taken(out["taken"], n, s.M)
            res["remap_equal"] = bool(np.array_equal(fs, ref.array("fs")))
            res["taken_count"] = int(np.unpackbits(out["taken"].view(np.uint8)).sum())
        res["searched"] = st.searched
        res["bounds"] = s.bounds
        res["sent"] = s.sent
        res["received"] = s.received
        # every hash was sent to the shard owning its partition
        hk = orc.key_hash(keys[cuts[rank]:cuts[rank + 1]], 5)
        j = np.array([(int(h) * s.num_partitions) >> 64 for h in hk], dtype=np.int64)
        owner = (j * world) // s.num_partitions
        res["sent_by_owner"] = bool(np.array_equal(np.bincount(owner, minlength=world), s.sent))
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


CASES = [
    # world, n, lambda, alpha, P, pilot mode, seed of the uneven key split (-1: even)
    (2, 20_000, 7.0, 0.99, 500, 0, 3),
    (3, 15_000, 6.0, 1.0, 400, 0, 4),
    (2, 9_000, 5.0, 0.9, 300, 1, -1),
    (4, 600, 5.0, 0.97, 500, 0, 5),   # two partitions over four shards: two own none
    (1, 8_000, 7.0, 0.99, 500, 0, -1),  # one shard: no exchange, no second grouping
]


@pytest.mark.parametrize("world,n,lam,alpha,P,mode,cuts", CASES)
def test_sharded_build_equals_single_build(tmp_path, world, n, lam, alpha, P, mode, cuts):
    _check_equals_single_build(tmp_path, world, dict(n=n, lam=lam, alpha=alpha, P=P, mode=mode, cuts=cuts, dup=False))


@pytest.mark.parametrize("world", [1, 3])
def test_sharded_build_with_a_metadata_group(tmp_path, world):
    """Counts and status codes over a separate gloo group give the same build."""
    case = dict(n=12_000, lam=7.0, alpha=0.99, P=500, mode=0, cuts=6, dup=False, cpu_group=True)
    _check_equals_single_build(tmp_path, world, case)


def _check_equals_single_build(tmp_path, world, case):
    import torch.multiprocessing as mp

    n, alpha = case["n"], case["alpha"]
    mp.spawn(_worker, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert "error" not in r, r
        assert r["pilots_equal"] and r["starts_equal"] and r["M_equal"] and r["sent_by_owner"], r
        if alpha < 1:
            assert r["remap_equal"] and r["taken_count"] == n, r
    # shard r searched exactly its partitions [J_r, J_{r+1}), and together all of them
    J = res[0]["bounds"]
    NP = J[-1]
    for r in res:
        assert r["searched"] == list(range(J[r["rank"]], J[r["rank"] + 1]))
        assert r["bounds"] == J
    assert sum(r["received"] for r in res) == n
    assert sorted(j for r in res for j in r["searched"]) == list(range(NP))
    # what each rank sent is what the owners received
    assert [sum(r["sent"][q] for r in res) for q in range(world)] == [r["received"] for r in res]


def test_sharded_build_duplicate_fails_on_every_rank(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    case = dict(n=6_000, lam=6.0, alpha=0.99, P=500, mode=0, cuts=-1, dup=True)
    mp.spawn(_worker, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [r.get("error") for r in res] == [3, 3]  # DUP_HASH on both ranks, no rank left waiting


def test_sharded_build_reports_the_single_builds_error(tmp_path):
    """One rank's partitions hit the search limit (s_max = 1 at lambda 12), another
    rank holds a duplicate pair: every rank reports DUP_HASH, as a single build
    would (duplicates take precedence over the search limit), and the oracle's
    single build agrees."""
    import torch.multiprocessing as mp
    from oracle import oracle as orc
    from paper_2404_18497_b300 import workloads

    world = 2
    case = dict(n=6_000, lam=12.0, alpha=1.0, P=500, mode=0, cuts=-1, dup=True, s_max=1)
    mp.spawn(_worker, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [r.get("error") for r in res] == [3, 3]
    keys = workloads.distinct_u64(6_000, 11)
    keys[-1] = keys[0]
    with pytest.raises(orc.OracleError) as e:
        orc.Oracle(keys, lam=12.0, alpha=1.0, P=500, s_max=1, seed=5, threads=1)
    assert e.value.code == orc.DUP_HASH


def test_shard_bounds_are_the_owner_map():
    from paper_2404_18497_b300 import shard

    for NP in (1, 2, 3, 7, 40, 1000, 40_000):
        for G in (1, 2, 3, 4, 8):
            J = shard.shard_bounds(NP, G)
            assert J[0] == 0 and J[-1] == NP
            for j in range(0, NP, max(1, NP // 500)):
                r = j * G // NP
                assert J[r] <= j < J[r + 1]
