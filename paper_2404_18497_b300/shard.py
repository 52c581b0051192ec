"""Partition-sharded construction of one MPHF across several processes.

Section 4 splits the keys into fine-grained partitions that are searched and
sized independently, tied together only by the prefix sums of their table sizes.
That makes the build shard by partition ranges: with G processes (one device
each), partition j = floor(hk N_P / 2^64) belongs to shard floor(j G / N_P), so
shard r owns the contiguous range [ceil(r N_P / G), ceil((r + 1) N_P / G)).

    1. every process hashes its own keys and groups them by partition;
    2. one all-to-all sends every shard the hashes of its partitions;
    3. each shard groups what it received by partition;
    4. an all-gather of the shards' partition starts gives every process the
       whole build's partition starts, and from them the slot offsets T;
    5. each shard searches its own partitions into a zero-filled pilot matrix
       and occupancy bitmap of the whole build;
    6. one all-reduce (sum) of each merges them: the shards' supports are
       disjoint, so the sum is the union;
    7. every process encodes the same structure from the same inputs, so each
       ends with the MPHF a single build of all n keys makes (replicated for
       queries).

This module holds only that orchestration.  The arithmetic of every step runs
in the library's kernels (`DeviceStages`, the C entry points of phobic.h); the
exchanges are torch.distributed collectives (`TorchComm`, NCCL between devices,
gloo on CPU).  Both are parameters so that the orchestration itself can be
exercised with other stages and transports.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch


# When shards fail differently, all report the error a single build would: a
# partition too large for the search is refused before any search, duplicate
# keys take precedence over the search limit, which takes precedence over a
# bounded wait that ran out (then any other failure).
_ERROR_RANK = {5: 6, 3: 5, 4: 4, 7: 3}


def shard_bounds(num_partitions: int, world: int) -> List[int]:
    """J_0 .. J_G: shard r owns partitions [J_r, J_{r+1}), J_r = ceil(r N_P / G),
    which is exactly the set of j with floor(j G / N_P) = r."""
    return [(r * num_partitions + world - 1) // world for r in range(world + 1)]


def num_partitions(n: int, P: int) -> int:
    return max(1, -(-n // P))


def num_buckets(lam: float, P: int) -> int:
    return max(1, math.ceil(float(P) / float(lam)))


@dataclass
class ShardStats:
    """What one process saw of a sharded build (for tests and benchmarks)."""
    n: int
    num_partitions: int
    bounds: List[int]
    sent: List[int]       # hashes sent to each shard
    received: int         # hashes of this shard's partitions
    M: int


class TorchComm:
    """The exchanges over a torch.distributed process group.  Tensors live on
    `device` (CUDA for NCCL, CPU for gloo).  `cpu_group` (optional, a gloo
    group over the same processes) carries the integer metadata (key counts,
    status codes): those values are on the host already, and sending them over
    a device group would cost a device synchronisation each."""

    def __init__(self, group=None, device=None, cpu_group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.cpu_group = cpu_group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = torch.device(device) if device is not None else torch.device("cpu")

    def _int_exchange(self):
        if self.cpu_group is not None:
            return self.cpu_group, torch.device("cpu")
        return self.group, self.device

    def all_gather_int(self, v: int) -> List[int]:
        grp, dev = self._int_exchange()
        t = torch.tensor([int(v)], dtype=torch.int64, device=dev)
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=grp)
        return [int(x.item()) for x in out]

    def all_to_all(self, send: torch.Tensor, send_counts: Sequence[int]) -> torch.Tensor:
        recv_counts = self._exchange_counts(send_counts)
        out = torch.empty(sum(recv_counts), dtype=send.dtype, device=send.device)
        self.dist.all_to_all_single(out, send, list(recv_counts), list(send_counts), group=self.group)
        return out

    def all_gather_v(self, t: torch.Tensor, counts: Sequence[int]) -> torch.Tensor:
        """Concatenation of every rank's t (rank r contributes counts[r] items)."""
        cap = max(max(counts), 1)
        pad = torch.zeros(cap, dtype=t.dtype, device=t.device)
        pad[: t.numel()] = t
        out = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(out, pad, group=self.group)
        return torch.cat([o[:c] for o, c in zip(out, counts)])

    def all_reduce_sum_(self, t: torch.Tensor) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def all_reduce_max_int(self, v: int) -> int:
        grp, dev = self._int_exchange()
        t = torch.tensor([int(v)], dtype=torch.int64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=grp)
        return int(t.item())

    def _exchange_counts(self, send_counts: Sequence[int]) -> List[int]:
        grp, dev = self._int_exchange()
        s = torch.tensor(list(send_counts), dtype=torch.int64, device=dev)
        r = torch.empty_like(s)
        self.dist.all_to_all_single(r, s, group=grp)
        return [int(x) for x in r.tolist()]


class DeviceStages:
    """The steps of the build on this process's device: the library's kernels
    through its C entry points."""

    def __init__(self, stream=None):
        from paper_2404_18497_b300 import phobic

        self.ph = phobic
        self.stream = stream

    def hash(self, keys: torch.Tensor, seed: int) -> torch.Tensor:
        return self.ph.phobic_hash_u64(keys, seed, stream=self.stream)

    def partition_sort(self, hk: torch.Tensor, num_partitions: int):
        if hk.numel() == 0:
            return hk, torch.zeros(num_partitions + 1, dtype=torch.int64, device=hk.device)
        return self.ph.phobic_partition_sort(hk, num_partitions, stream=self.stream)

    def table_offsets(self, start: torch.Tensor, alpha: float):
        T, (M, _, _) = self.ph.phobic_table_offsets(start, alpha, stream=self.stream)
        return T, M

    def zeros_u32(self, count: int, like: torch.Tensor) -> torch.Tensor:
        return torch.zeros(count, dtype=torch.int32, device=like.device)

    def search(self, sorted_hk, start, T, n, num_partitions, j0, j1, params, pilots, taken) -> int:
        """Status code of the search of partitions [j0, j1) (0 = OK)."""
        try:
            self.ph.phobic_search_partitions(sorted_hk, start, T, n, num_partitions, j0, j1, params, pilots, taken,
                                             stream=self.stream)
        except self.ph.PhobicError as e:
            return e.code
        return 0

    def assemble(self, start, n, pilots, taken, params):
        return self.ph.phobic_assemble(start, n, pilots, taken, params, stream=self.stream)

    def error(self, code: int, what: str) -> Exception:
        return self.ph.PhobicError(code, what)


def sharded_build(keys: torch.Tensor, params, comm, stages=None, stats_out: Optional[list] = None):
    """One MPHF over the keys of all processes of `comm`, each process passing
    its own (disjoint) share `keys`.  Every process returns the same structure,
    the one a single build of all keys with `params` makes.  A failure of any
    shard's search (duplicate keys, search limit) raises on every process
    before the merge, so no process waits in a collective that the others
    skip."""
    st = stages if stages is not None else DeviceStages()
    G, r = comm.world, comm.rank
    n = sum(comm.all_gather_int(keys.numel()))
    if n == 0:
        raise ValueError("no keys on any process")
    P, lam, alpha = int(params.partition_size), float(params.lambda_), float(params.alpha)
    NP = num_partitions(n, P)
    B = num_buckets(lam, P)
    J = shard_bounds(NP, G)

    # 1-2: hash, group by partition, send each shard the hashes of its partitions
    hk = st.hash(keys, int(params.seed))
    srt, start = st.partition_sort(hk, NP)
    at = start[torch.tensor(J, dtype=torch.int64, device=start.device)].tolist()
    sent = [int(at[q + 1] - at[q]) for q in range(G)]
    if G == 1:  # one shard: its hashes are already grouped, nothing to exchange
        rsorted, rstart = srt, start
        del hk
    else:
        recv = comm.all_to_all(srt, sent)
        del srt, hk, start
        # 3: group the received hashes (G runs, each grouped by partition)
        rsorted, rstart = st.partition_sort(recv, NP)
        del recv

    # 4: the whole build's partition starts and T
    held = comm.all_gather_int(rsorted.numel())
    own = rstart[J[r]:J[r + 1]] + sum(held[:r])
    gstart = comm.all_gather_v(own, [J[q + 1] - J[q] for q in range(G)])
    gstart = torch.cat([gstart, torch.tensor([n], dtype=gstart.dtype, device=gstart.device)])
    T, M = st.table_offsets(gstart, alpha)

    # 5: search this shard's partitions into the whole build's matrix and bitmap
    pilots = st.zeros_u32(B * NP, gstart)
    taken = st.zeros_u32((M + 31) // 32 + 1, gstart) if M > n else None
    code = st.search(rsorted, rstart, T, n, NP, J[r], J[r + 1], params, pilots, taken)
    worst = comm.all_reduce_max_int((_ERROR_RANK.get(code, 1) << 8) | code if code else 0) & 0xFF
    if worst != 0:
        raise st.error(worst, "sharded search")
    del rsorted, rstart

    # 6-7: merge (disjoint supports: the sum is the union), then encode
    comm.all_reduce_sum_(pilots)
    if taken is not None:
        comm.all_reduce_sum_(taken)
    if stats_out is not None:
        stats_out.append(ShardStats(n=n, num_partitions=NP, bounds=J, sent=sent, received=int(held[r]), M=M))
    return st.assemble(gstart, n, pilots, taken, params)
