"""Oracle stand-ins for the device stages of the partition-sharded build, on
CPU tensors, so that the sharding orchestration (paper_2404_18497_b300/shard.py)
runs with gloo ranks and no GPU.  Each stage is the oracle's own restatement:
master hashes from or_key_hash, one partition's search from
or_search_one_partition; grouping by partition and prefix sums are plain numpy.
`assemble` returns the merged inputs of the final encoding for comparison with
a single oracle build."""
import math

import numpy as np
import torch


def _u64(t: torch.Tensor) -> np.ndarray:
    return t.numpy().view(np.uint64)


def _i64(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64))


def partition_ids(hk: np.ndarray, num_partitions: int) -> np.ndarray:
    return np.array([(int(h) * num_partitions) >> 64 for h in hk], dtype=np.int64)


class OracleStages:
    def __init__(self, orc, lam, alpha, P, mode=0, s_max=0):
        self.orc, self.lam, self.alpha, self.P, self.mode, self.s_max = orc, lam, alpha, P, mode, s_max
        self.searched = []  # partitions this process searched

    def hash(self, keys, seed):
        return _i64(self.orc.key_hash(_u64(keys), seed))

    def partition_sort(self, hk, num_partitions):
        h = _u64(hk)
        j = partition_ids(h, num_partitions)
        order = np.argsort(j, kind="stable")
        start = np.concatenate([[0], np.cumsum(np.bincount(j, minlength=num_partitions))]).astype(np.int64)
        return _i64(h[order]), torch.from_numpy(start)

    def table_offsets(self, start, alpha):
        nj = np.diff(start.numpy())
        m = nj if alpha == 1.0 else np.maximum(nj, np.array([math.ceil(int(v) / alpha) for v in nj], dtype=np.int64))
        T = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
        return torch.from_numpy(T), int(T[-1])

    def zeros_u32(self, count, like):
        return torch.zeros(count, dtype=torch.int32)

    def search(self, sorted_hk, start, T, n, num_partitions, j0, j1, params, pilots, taken):
        h, st, TT = _u64(sorted_hk), start.numpy(), T.numpy()
        words = taken.numpy().view(np.uint32) if taken is not None else None
        pv = pilots.numpy().view(np.uint32)
        for j in range(j0, j1):  # equal master hashes anywhere: DUP_HASH, whatever else fails
            if np.unique(h[st[j]:st[j + 1]]).size != st[j + 1] - st[j]:
                return self.orc.DUP_HASH
        for j in range(j0, j1):
            try:
                pil, tk = self.orc.search_one_partition(h[st[j]:st[j + 1]], self.lam, self.alpha, self.P,
                                                        mode=self.mode, s_max=self.s_max)
            except self.orc.OracleError as e:
                return e.code
            self.searched.append(j)
            pv[np.arange(pil.size) * num_partitions + j] = pil
            if words is not None:
                for g in TT[j] + np.flatnonzero(tk):
                    words[g >> 5] |= np.uint32(1 << (int(g) & 31))
        return 0

    def assemble(self, start, n, pilots, taken, params):
        return dict(start=start.numpy().copy(), n=n, pilots=pilots.numpy().view(np.uint32).copy(),
                    taken=None if taken is None else taken.numpy().view(np.uint32).copy())

    def error(self, code, what):
        return self.orc.OracleError(code, what)


def remap_from_taken(taken_words: np.ndarray, n: int, M: int) -> np.ndarray:
    """The free-slot remap of slots [n, M) from an occupancy bitmap: F = free
    slots below n ascending, fs[q - n] = F[min(#occupied in [n, q), |F| - 1)]."""
    bits = np.unpackbits(taken_words.view(np.uint8), bitorder="little")[:M].astype(bool)
    F = np.flatnonzero(~bits[:n])
    occ = bits[n:M]
    rank = np.concatenate([[0], np.cumsum(occ)[:-1]]) if occ.size else np.zeros(0, dtype=np.int64)
    if F.size == 0:
        return np.zeros(M - n, dtype=np.uint64)
    return F[np.minimum(rank, F.size - 1)].astype(np.uint64)
