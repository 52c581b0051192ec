"""Space accounting of the oracle, recounted term by term from scratch.

The paper's space figures (Section 4.1 and the per-encoder comparison of
Section 5, Figure 3b) count the encoded pilots with each encoder's metadata,
plus the offsets (stored as differences to their expectation, Section 4) and,
for alpha < 1, the Elias-Fano remap of the slots >= n.  Here every term is
recomputed in numpy from quantities this test derives itself: the partition of
each master hash (floor(hk N_P / 2^64) in Python integers), the table sizes
ceil(n_j / alpha), the offsets T, and the raw pilots of the search.  Only the
pilots come from the oracle (the search is pinned elsewhere: brute force and
first-valid replay), and the Golomb-Rice parameter, pinned by its own test
against the expected-length minimiser.  The bit widths and counts follow from
what each structure must hold:

    header    n, M, N_P, B, P, lambda, alpha, seed, pilot mode: 9 words of 64 bits
    offsets   N_P + 1 values D_j - min D at width bitlen(max D - min D), plus
              min D (64), the slope Q of the expectation (64) and the width (8)
    IC-C      per column N_P values at bitlen(max) bits, plus base (64) and width (8)
    IC-D      per column N_P ranks at bitlen(K - 1) and K sorted distinct values at
              bitlen(max), plus two bases (64 + 64) and two widths (8 + 8)
    IC-R      per column N_P low parts of l bits, N_P + sum(v >> l) unary bits, a
              32-bit select sample per 64 values, two bases (64 + 64), l (8)
    IC-EF     the same with the prefix sums E_j in Elias-Fano form: N_P low parts
              of l = floor(log2((E_last + 1) / N_P)) bits and N_P + (E_last >> l) + 1
              high bits
    IC-CR     the first c columns as IC-C, the others as IC-R, plus c (32)
    mono-X    encoder X over one column of all B N_P pilots in column order
    remap     Elias-Fano of the M - n remapped slots in universe n: N l low bits,
              N + (n >> l) + 1 high bits, a 64-bit sample per 64 values, and
              three 64-bit header words (N, l, universe)

A wrong constant or a dropped term anywhere in the oracle's accounting fails
here, although the paper's +-0.2 bits/key bands would let it through.
"""
import math

import numpy as np
import pytest

ENC_NAMES = {0: "IC-C", 1: "IC-D", 2: "IC-R", 3: "IC-EF", 4: "IC-CR",
             5: "mono-C", 6: "mono-D", 7: "mono-R", 8: "mono-EF"}


def _bitlen(v: int) -> int:
    return int(v).bit_length()


def _partition_sizes(hk: np.ndarray, NP: int) -> np.ndarray:
    j = np.array([(int(h) * NP) >> 64 for h in hk], dtype=np.int64)
    return np.bincount(j, minlength=NP)


def _table_sizes(nj: np.ndarray, alpha: float) -> np.ndarray:
    if alpha == 1.0:
        return nj.copy()
    m = np.array([math.ceil(int(v) / alpha) for v in nj], dtype=np.int64)
    return np.maximum(m, nj)


def _offset_bits(T: np.ndarray, NP: int) -> int:
    M = int(T[-1])
    Q = (M << 32) // NP
    D = [int(T[j]) - ((j * Q) >> 32) for j in range(NP + 1)]
    w = _bitlen(max(D) - min(D))
    return (NP + 1) * w + 64 + 64 + 8


def _compact(col) -> int:
    return len(col) * _bitlen(max(col)) + 64 + 8


def _dictionary(col) -> int:
    d = sorted(set(col))
    return len(col) * _bitlen(len(d) - 1) + len(d) * _bitlen(d[-1]) + 64 + 64 + 8 + 8


def _rice(col, rice_param) -> int:
    N = len(col)
    l = rice_param(sum(col), N)
    high = N + sum(v >> l for v in col)
    return N * l + high + 32 * ((N + 63) // 64) + 64 + 64 + 8


def _elias_fano_column(col) -> int:
    N = len(col)
    last = sum(col)
    U = last + 1
    l = _bitlen(U // N) - 1 if U >= N else 0
    return N * l + N + (last >> l) + 1 + 32 * ((N + 63) // 64) + 64 + 64 + 8


def _pilot_bits(pil: np.ndarray, encoder: int, c: int, rice_param) -> int:
    B, NP = pil.shape
    if encoder >= 5:
        cols = [pil.reshape(-1).astype(np.int64).tolist()]
        encoder -= 5
    else:
        cols = [pil[b].astype(np.int64).tolist() for b in range(B)]
    total = 0
    for b, col in enumerate(cols):
        if encoder == 0 or (encoder == 4 and b < c):
            total += _compact(col)
        elif encoder == 1:
            total += _dictionary(col)
        elif encoder in (2, 4):
            total += _rice(col, rice_param)
        else:
            total += _elias_fano_column(col)
    if encoder == 4:
        total += 32
    return total


def _remap_bits(n: int, M: int) -> int:
    N = M - n
    if N == 0:
        return 0
    l = _bitlen(n // N) - 1 if n >= N else 0
    return N * l + N + (n >> l) + 1 + 64 * ((N + 63) // 64) + 3 * 64


CASES = [
    # n, lambda, alpha, P, encoder, compact columns
    (40_000, 7.0, 1.0, 2500, 0, 0),
    (40_000, 7.0, 0.99, 2500, 1, 0),
    (30_000, 6.0, 0.97, 800, 2, 0),
    (30_000, 6.0, 0.9, 800, 3, 0),
    (30_000, 5.0, 0.99, 600, 4, 20),
    (20_000, 5.0, 1.0, 500, 5, 0),
    (20_000, 5.0, 0.95, 500, 6, 0),
    (20_000, 5.0, 0.99, 500, 7, 0),
    (20_000, 5.0, 0.8, 500, 8, 0),
    (2, 7.0, 0.7, 2500, 1, 0),
    (1, 3.0, 1.0, 2500, 0, 0),
]


@pytest.mark.parametrize("n,lam,alpha,P,enc,c", CASES)
def test_every_space_term_recounted(orc, n, lam, alpha, P, enc, c):
    rng = np.random.default_rng(1000 + n + enc)
    hk = np.unique(rng.integers(0, 2**64, size=n, dtype=np.uint64))
    assert hk.size == n
    h = orc.Oracle(hashed=hk, lam=lam, alpha=alpha, P=P, encoder=enc, compact_columns=c, threads=4)
    NP = max(1, math.ceil(n / P))
    B = max(1, math.ceil(P / lam))
    assert (h.u64("NP"), h.u64("B")) == (NP, B)
    nj = _partition_sizes(hk, NP)
    m = _table_sizes(nj, alpha)
    T = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    M = int(T[-1])
    assert h.u64("M") == M
    pil = h.pilots
    want = {
        "bits_header": 9 * 64,
        "bits_offsets": _offset_bits(T, NP),
        "bits_pilots": _pilot_bits(pil, enc, min(c, B), orc.lib().or_rice_param),
        "bits_remap": _remap_bits(n, M),
    }
    want["bits_total"] = sum(want.values())
    got = {k: h.u64(k) for k in want}
    assert got == want, ENC_NAMES[enc]
    assert h.bits_per_key() == want["bits_total"] / n
