"""Independent pure-Python restatement of PHOBIC for tiny inputs (test helper).

It shares no code with the C oracle.  It follows the same written rules:
hash finaliser, bucket table, bucket order and pilot enumeration.  Every pilot
is found by trying p = 0, 1, 2, ... in order with the query formula of
Section 4 ("Hash Function").  No shortcut is taken: no window scan and no
skipping of self-colliding s.  It is meant for n <= a few hundred.
"""
from __future__ import annotations

import math

MASK = (1 << 64) - 1
C_SEED = 0x9E3779B97F4A7C15
C_BUCKET = 0x5851F42D4C957F2D
C_PILOT = 0x2545F4914F6CDD1D


def mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def fastrange(h: int, m: int) -> int:
    return (h * m) >> 64


def key_hash(key: int, seed: int) -> int:
    return mix64(key ^ mix64(seed ^ C_SEED))


def position(hk: int, p: int, m: int, mode: int) -> int:
    if mode == 0:  # additive displacement: (h(x, floor(p/m)) + p) mod m
        s = p // m
        return (fastrange(mix64(hk ^ mix64(s ^ C_PILOT)), m) + p) % m
    return fastrange(mix64(hk ^ mix64(p ^ C_PILOT)), m)


def table(lam: float, alpha: float, P: int):
    eps = min(1.0, lam / (5.0 * math.sqrt(P)))

    def beta_star(x):
        return 1.0 if x >= 1.0 else x + (1.0 - x) * math.log1p(-x)

    out = []
    for k in range(2049):
        x = k / 2048.0
        if alpha == 1.0:
            g = 1.0 if x >= 1.0 else eps * x + (1.0 - eps) * beta_star(x)
        else:
            ax = alpha * x
            g = (eps * ax + (1.0 - eps) * beta_star(ax)) / (eps * alpha + (1.0 - eps) * beta_star(alpha))
        v = g * 4294967296.0
        r = math.floor(v + 0.5)  # round half away from zero for non-negative v
        out.append(min(max(r, 0), 1 << 32))
    return out


def bucket(hk: int, tab, B: int) -> int:
    x = mix64(hk ^ C_BUCKET)
    k = x >> 53
    f = (x >> 21) & 0xFFFFFFFF
    v = tab[k] + (((tab[k + 1] - tab[k]) * f) >> 32)
    return min(B - 1, (v * B) >> 32)


def build(keys, lam=3.0, alpha=1.0, P=8, mode=0, seed=0, pmax=1 << 24):
    """Returns (pilots[b][j], T, n_j, m_j, per-key local position)."""
    n = len(keys)
    NP = max(1, -(-n // P))
    B = max(1, math.ceil(P / lam))
    tab = table(lam, alpha, P)
    hks = [key_hash(k, seed) for k in keys]
    parts = [[] for _ in range(NP)]
    for hk in hks:
        parts[fastrange(hk, NP)].append(hk)
    pilots = [[0] * NP for _ in range(B)]
    n_j, m_j = [], []
    for j, pk in enumerate(parts):
        nj = len(pk)
        m = nj if alpha == 1.0 else max(nj, math.ceil(nj / alpha))
        n_j.append(nj)
        m_j.append(m)
        buckets = {}
        for hk in pk:
            buckets.setdefault(bucket(hk, tab, B), []).append(hk)
        order = sorted(buckets, key=lambda b: (-len(buckets[b]), -b))
        taken = [False] * m
        for b in order:
            ks = buckets[b]
            p = 0
            while True:
                pos = [position(hk, p, m, mode) for hk in ks]
                if len(set(pos)) == len(pos) and not any(taken[x] for x in pos):
                    break
                p += 1
                if p > pmax:
                    raise RuntimeError("pilot search limit")
            for x in pos:
                taken[x] = True
            pilots[b][j] = p
    T = [0]
    for m in m_j:
        T.append(T[-1] + m)
    return pilots, T, n_j, m_j
