"""Seeded synthetic workloads (host side, numpy PCG64).

These generators feed both the CUDA library and the CPU oracle, which then see
the same bytes.  They contain none of the MPHF's arithmetic: only draws from
numpy's PCG64 generator, sorting (to make keys distinct) and indexing.

Workload recipes follow the paper's settings and the benchmark configurations:
- uniform distinct 64-bit keys;
- positive queries drawn uniformly from the key set;
- Zipf(s = 1) query orders.  A rank r in [1, n] is drawn by inverting the
  continuous 1/r law, r = floor((n + 1)^u) with u uniform in [0, 1), and mapped
  to a key through a seeded permutation;
- random strings of length uniform in [10, 50] over [A-Za-z0-9] (Section 5's
  input).
"""
from __future__ import annotations

import numpy as np

ALNUM = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789", dtype=np.uint8)


def distinct_u64(n: int, seed: int) -> np.ndarray:
    """n distinct uniform-random uint64 values (duplicates are redrawn)."""
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2**64, size=n, dtype=np.uint64, endpoint=False)
    while True:
        s = np.sort(keys)
        if not (s[1:] == s[:-1]).any():
            return keys
        order = np.argsort(keys, kind="stable")
        s = keys[order]
        dup = np.flatnonzero(s[1:] == s[:-1]) + 1
        keys[order[dup]] = rng.integers(0, 2**64, size=dup.size, dtype=np.uint64, endpoint=False)


def uniform_queries(keys: np.ndarray, q: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return keys[rng.integers(0, keys.size, size=q)]


def zipf_queries(keys: np.ndarray, q: int, seed: int) -> np.ndarray:
    """Keys in a Zipf(s = 1) order: rank r has probability ~ 1/r."""
    rng = np.random.default_rng(seed)
    n = keys.size
    u = rng.random(q)
    r = np.floor(np.exp(u * np.log(n + 1.0))).astype(np.int64)
    r = np.clip(r, 1, n)
    perm = rng.permutation(n)
    return keys[perm[r - 1]]


def mixed_queries(keys: np.ndarray, q: int, positive_fraction: float, seed: int) -> np.ndarray:
    """A fraction of positive (member) queries, the rest fresh random values."""
    rng = np.random.default_rng(seed)
    pos = rng.random(q) < positive_fraction
    out = rng.integers(0, 2**64, size=q, dtype=np.uint64, endpoint=False)
    out[pos] = keys[rng.integers(0, keys.size, size=int(pos.sum()))]
    return out


def random_strings(n: int, seed: int, lmin: int = 10, lmax: int = 50):
    """n strings with lengths uniform in [lmin, lmax] over [A-Za-z0-9].
    Returns (bytes uint8[total], offsets uint64[n + 1])."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(lmin, lmax + 1, size=n, dtype=np.int64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    data = ALNUM[rng.integers(0, ALNUM.size, size=int(offsets[-1]), dtype=np.uint8)]
    return data, offsets


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
