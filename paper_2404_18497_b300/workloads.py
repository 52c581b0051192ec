"""Seeded synthetic workloads (host side, numpy PCG64).

These generators feed both the CUDA library and the CPU oracle, which then see
the same bytes.  They contain none of the MPHF's arithmetic: only draws from
numpy's PCG64 generator, sorting (to make keys distinct) and indexing.

Workload recipes follow the paper's settings and the benchmark configurations:
- uniform distinct 64-bit keys;
- positive queries drawn uniformly from the key set;
- Zipf(s = 1) query orders: rank r in [1, n] with probability exactly
  (1/r) / H_n, drawn by rejection-inversion (Hoermann and Derflinger 1996) and
  mapped to a key through a seeded permutation;
- random strings of length uniform in [10, 50] over [A-Za-z0-9] (Section 5's
  input);
- batches of many key sets with log-uniform sizes, whose keys come from a
  counter-based stream (below) that the host and the device produce alike, so
  a test can rebuild any sampled set on the host without copying the batch
  back.

The counter-based stream: key i = fmix64(seed' + i * W), with W the odd 64-bit
Weyl increment 0x9E3779B97F4A7C15, seed' = fmix64(seed) and fmix64 the
MurmurHash3 64-bit finaliser (Appleby).  fmix64 is a bijection on 64-bit words
and i -> seed' + i W is injective for i < 2^64, so all keys of the stream are
distinct.
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


def zipf_ranks(n: int, q: int, rng: np.random.Generator) -> np.ndarray:
    """q ranks in [1, n] with P(r) = (1/r) / H_n (Zipf, exponent 1), by
    rejection-inversion (W. Hoermann, G. Derflinger, "Rejection-inversion to
    generate variates from monotone discrete distributions", ACM TOMACS 6(3),
    1996).

    The hat is the continuous density 1/x with antiderivative H(x) = ln x.
    Rank k owns the interval [H(k - 1/2), H(k + 1/2)), whose length
    ln((k + 1/2) / (k - 1/2)) is at least 1/k because 1/x is convex; the top
    1/k of it, [H(k + 1/2) - 1/k, H(k + 1/2)), is k's acceptance strip.  A
    uniform u over [H(3/2) - 1, H(n + 1/2)) (from the start of rank 1's strip)
    is inverted to x = e^u and rounded to k; u is kept when it lies in k's
    strip and redrawn otherwise.  The kept u are uniform over the union of the
    strips, so k is drawn with probability proportional to 1/k exactly (up to
    double rounding at strip edges)."""
    out = np.empty(q, dtype=np.int64)
    lo, hi = np.log(1.5) - 1.0, np.log(n + 0.5)
    todo = np.arange(q)
    while todo.size:
        u = lo + rng.random(todo.size) * (hi - lo)
        k = np.clip(np.floor(np.exp(u) + 0.5), 1, n)
        ok = u >= np.log(k + 0.5) - 1.0 / k
        out[todo[ok]] = k[ok].astype(np.int64)
        todo = todo[~ok]
    return out


def zipf_queries(keys: np.ndarray, q: int, seed: int) -> np.ndarray:
    """Keys in a Zipf(s = 1) order: the key of rank r is drawn with probability
    (1/r) / H_n; ranks are mapped to keys through a seeded permutation."""
    rng = np.random.default_rng(seed)
    n = keys.size
    r = zipf_ranks(n, q, rng)
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


def random_strings_torch(n: int, seed: int, device, lmin: int = 10, lmax: int = 50):
    """The same distribution as random_strings (lengths uniform in [lmin, lmax],
    characters uniform over [A-Za-z0-9]), drawn on `device` with torch's
    generator (another instance of the workload, generated in seconds).
    Returns (bytes uint8[total], offsets int64[n + 1])."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lens = torch.randint(lmin, lmax + 1, (n,), generator=g, device=device, dtype=torch.int64)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(lens, 0, out=offsets[1:])
    del lens
    total = int(offsets[-1].item())
    alnum = torch.from_numpy(ALNUM.copy()).to(device)
    data = torch.empty(total + 8, dtype=torch.uint8, device=device)
    chunk = 1 << 30
    for c0 in range(0, total, chunk):
        c1 = min(total, c0 + chunk)
        data[c0:c1] = alnum[torch.randint(0, ALNUM.size, (c1 - c0,), generator=g, device=device)]
    data[total:] = 0
    return data, offsets


_W = 0x9E3779B97F4A7C15
_F1 = 0xFF51AFD7ED558CCD
_F2 = 0xC4CEB9FE1A85EC53


def _fmix64_np(k: np.ndarray) -> np.ndarray:
    k = k ^ (k >> np.uint64(33))
    k = k * np.uint64(_F1)
    k = k ^ (k >> np.uint64(33))
    k = k * np.uint64(_F2)
    return k ^ (k >> np.uint64(33))


def _stream_base(seed: int) -> int:
    with np.errstate(over="ignore"):
        return int(_fmix64_np(np.array([seed & (2**64 - 1)], dtype=np.uint64))[0])


def stream_keys(start: int, n: int, seed: int) -> np.ndarray:
    """Keys start .. start + n - 1 of the counter-based stream, on the host."""
    i = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _fmix64_np(np.uint64(_stream_base(seed)) + i * np.uint64(_W))


def _s64(c: int) -> int:
    return c - 2**64 if c >= 2**63 else c


def stream_keys_torch(start: int, n: int, seed: int, device, chunk: int = 1 << 27):
    """The same keys as stream_keys, generated on `device` as an int64 tensor
    (the uint64 bit patterns), in chunks to bound temporary memory."""
    import torch

    out = torch.empty(n, dtype=torch.int64, device=device)
    base, w, f1, f2 = _s64(_stream_base(seed)), _s64(_W), _s64(_F1), _s64(_F2)
    m31 = (1 << 31) - 1  # logical shift right by 33 of a 64-bit word
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        k = torch.arange(start + c0, start + c1, dtype=torch.int64, device=device)
        k.mul_(w).add_(base)
        k.bitwise_xor_((k >> 33) & m31)
        k.mul_(f1)
        k.bitwise_xor_((k >> 33) & m31)
        k.mul_(f2)
        k.bitwise_xor_((k >> 33) & m31)
        out[c0:c1] = k
    return out


def batch_sets(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Set offsets (uint64[count + 1]) of a batch with log-uniform set sizes."""
    sizes = np.maximum(1, log_uniform_sizes(count, lo, hi, seed))
    off = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(sizes, out=off[1:])
    return off


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
