"""The export format as a contract between implementations (no GPU needed).

Files written from the oracle's arrays in the documented layout must pass the
library's host-side inspection, which reports the oracle's parameters and
space.  Corrupted files must be refused, each for the check that guards it.
Every check holds without a device, because phobic_inspect reads the bytes on
the host only.
"""
import json
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
from oracle_export import oracle_export  # noqa: E402

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ph():
    from paper_2404_18497_b300 import build, phobic

    build.build()
    phobic.lib()
    return phobic


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle

    oracle.build_oracle_lib()
    return oracle


def _keys(n, seed):
    return np.random.default_rng(seed).integers(0, 2**64, size=n, dtype=np.uint64)


CASES = [(enc, alpha, mode) for enc in range(9) for alpha, mode in ((1.0, 0), (0.97, 1))]


@pytest.mark.parametrize("enc,alpha,mode", CASES)
def test_oracle_files_pass_inspection(ph, orc, enc, alpha, mode):
    keys = _keys(40_000 + enc, 70 + enc)
    o = orc.Oracle(keys, lam=6.5, alpha=alpha, P=1000, encoder=enc, mode=mode, compact_columns=5, seed=11,
                   threads=4)
    data = oracle_export(o)
    info = ph.phobic_inspect(data)
    assert info["n"] == keys.size and info["M"] == o.u64("M")
    assert info["num_partitions"] == o.u64("NP") and info["num_buckets"] == o.u64("B")
    assert info["partition_size"] == 1000 and info["lambda"] == 6.5 and info["alpha"] == alpha
    assert info["encoder"] == enc and info["pilot_mode"] == mode and info["seed"] == 11
    assert info["compact_columns"] == (5 if enc == 4 else 0)
    for k in ("bits_header", "bits_offsets", "bits_pilots", "bits_remap", "bits_total"):
        assert info[k] == o.u64(k), k
    assert info["device_bytes"] == 8 * 2048 + len(data) - 8 * 28  # the packed bucket table + the arrays


def _words(data):
    return np.frombuffer(data, dtype=np.uint64).copy()


def _offsets(w):
    """Start word of each of the seven arrays."""
    at = [28]
    for c in w[16:23]:
        at.append(at[-1] + int(c))
    return at


def _refused(ph, w):
    with pytest.raises(ph.PhobicError) as e:
        ph.phobic_inspect(w.tobytes())
    assert e.value.status == "FORMAT"


def test_corrupt_files_are_refused(ph, orc):
    keys = _keys(60_000, 81)
    od = orc.Oracle(keys, lam=6.5, alpha=0.97, P=1000, encoder=1, threads=4)
    orr = orc.Oracle(keys, lam=6.5, alpha=0.97, P=1000, encoder=2, threads=4)
    for o in (od, orr):
        w = _words(oracle_export(o))
        ph.phobic_inspect(w.tobytes())  # the intact file passes
        at = _offsets(w)
        bad = w.copy(); bad[0] ^= np.uint64(1); _refused(ph, bad)              # magic
        bad = w.copy(); bad[1] = 2; _refused(ph, bad)                           # version
        _refused(ph, w[:-1])                                                    # truncated
        _refused(ph, np.concatenate([w, w[:1]]))                                # trailing word
        bad = w.copy(); bad[5] += np.uint64(1); _refused(ph, bad)               # B not the one lambda and P imply
        bad = w.copy(); bad[10] = 9; _refused(ph, bad)                          # unknown encoder
        bad = w.copy(); bad[14] += np.uint64(1); _refused(ph, bad)              # offsets no longer start at 0
        last = int(w[4]) * int(w[12])  # bit of D_{N_P}, the last offset
        bad = w.copy(); bad[at[0] + last // 64] ^= np.uint64(1 << (last % 64)); _refused(ph, bad)  # T_{N_P} != M
        bad = w.copy(); bad[at[1]] |= np.uint64(40 << 56); _refused(ph, bad)     # a column width above 32
        # the Elias-Fano remap: a missing one in the high part, a wrong sample
        hi = at[5]
        nz = hi + int(np.flatnonzero(w[at[5]:at[6]])[2])
        bad = w.copy(); bad[nz] &= bad[nz] - np.uint64(1); _refused(ph, bad)
        bad = w.copy(); bad[at[6] + 1] += np.uint64(1); _refused(ph, bad)
    # IC-D: a rank past its column's dictionary
    w = _words(oracle_export(od))
    at = _offsets(w)
    meta = w[at[1]:at[2]]
    rw = (meta[0::2] >> np.uint64(56)).astype(np.int64)
    db = (meta[1::2] & np.uint64((1 << 56) - 1)).astype(np.int64)
    dw = (meta[1::2] >> np.uint64(56)).astype(np.int64)
    K = np.diff(db) // np.maximum(dw[:-1], 1)
    b = int(np.flatnonzero((K < (1 << rw[:-1]) ) & (dw[:-1] > 0))[0])  # a column whose rank width has room
    bit0 = int(meta[2 * b] & np.uint64((1 << 56) - 1))  # partition 0's rank of column b
    bad = w.copy()
    for t in range(int(rw[b])):  # rank = 2^rw - 1 >= K
        o = bit0 + t
        bad[at[2] + o // 64] |= np.uint64(1 << (o % 64))
    _refused(ph, bad)
    # IC-R: a unary region with a one missing
    w = _words(oracle_export(orr))
    at = _offsets(w)
    ns = (orr.u64("NP") + 63) // 64
    sw = (orr.u64("B") * ns + 1) // 2
    nz = at[3] + sw + int(np.flatnonzero(w[at[3] + sw:at[4]])[5])
    bad = w.copy(); bad[nz] &= bad[nz] - np.uint64(1); _refused(ph, bad)


def test_inspection_work_is_linear_in_the_file(ph, orc):
    """A header may claim any number of keys; checks whose loops the file does
    not pay for in bits (zero-width offsets, widths and ranks) are made in
    closed form, so a tiny file claiming 2^40 keys is answered at once."""
    import time

    # one partition: every offset difference is 0, so the offsets have width 0
    o = orc.Oracle(_keys(1_500, 95), lam=7.0, alpha=1.0, P=2500, encoder=0, threads=1)
    w = _words(oracle_export(o))
    assert w[12] == 0 and w[4] == 1
    ph.phobic_inspect(w.tobytes())
    bad = w.copy(); bad[13] += np.uint64(1 << 32); _refused(ph, bad)  # T_{N_P} != M in closed form
    # the same file claiming 2^40 keys in 2^40 / 2500 partitions, every width 0
    P, NP = 2500, (1 << 40) // 2500
    big = w.copy()
    big[2] = big[3] = NP * P          # n = M
    big[4] = NP
    big[13] = P << 32                 # Q: T_j = j P exactly
    at = _offsets(big)
    big[at[1]:at[2]] &= np.uint64((1 << 56) - 1)  # every column width 0
    t = time.time()
    info = ph.phobic_inspect(big.tobytes())  # a valid, degenerate structure: every pilot 0
    assert time.time() - t < 1.0
    assert info["n"] == NP * P and info["num_partitions"] == NP


def test_inspection_survives_random_corruption(ph, orc):
    """Random corruptions of valid files (bit flips anywhere, random words,
    truncations, header fields) are each accepted or refused with FORMAT, and
    never crash the process: the checks read only inside the buffer."""
    rng = np.random.default_rng(2024)
    keys = _keys(20_000, 97)
    files = []
    for enc, alpha in ((1, 0.97), (2, 0.97), (3, 1.0), (4, 0.97), (6, 0.97), (7, 1.0), (8, 0.97), (0, 0.97)):
        o = orc.Oracle(keys, lam=6.5, alpha=alpha, P=1000, encoder=enc, compact_columns=7, threads=4)
        files.append(_words(oracle_export(o)))
    outcomes = {"OK": 0, "FORMAT": 0}
    for w in files:
        for t in range(250):
            bad = w.copy()
            kind = t % 5
            if kind == 0:  # flip one bit anywhere
                i = int(rng.integers(0, bad.size))
                bad[i] ^= np.uint64(1 << int(rng.integers(0, 64)))
            elif kind == 1:  # a random word anywhere
                bad[int(rng.integers(0, bad.size))] = rng.integers(0, 2**64, dtype=np.uint64)
            elif kind == 2:  # a header field set to a random small or huge value
                i = int(rng.integers(2, 28))
                bad[i] = np.uint64(int(rng.integers(0, 1 << 20)) if t % 2 else int(rng.integers(0, 2**63)))
            elif kind == 3:  # truncated
                bad = bad[: int(rng.integers(0, bad.size))]
            else:  # several bit flips in the arrays
                for _ in range(8):
                    i = int(rng.integers(28, bad.size))
                    bad[i] ^= np.uint64(1 << int(rng.integers(0, 64)))
            try:
                ph.phobic_inspect(bad.tobytes())
                outcomes["OK"] += 1
            except ph.PhobicError as e:
                assert e.status == "FORMAT"
                outcomes["FORMAT"] += 1
    assert outcomes["FORMAT"] > 1000  # most corruptions are caught


def test_fileinfo_tool(ph, orc, tmp_path, capsys):
    from paper_2404_18497_b300 import fileinfo

    o = orc.Oracle(_keys(30_000, 90), lam=7.0, alpha=0.99, P=2500, encoder=7, threads=4)
    f = tmp_path / "s.bin"
    f.write_bytes(oracle_export(o))
    assert fileinfo.main([str(f), "--json"]) == 0
    r = json.loads(capsys.readouterr().out)
    assert r["valid"] and r["encoder"] == "mono-R" and r["n"] == 30_000
    assert abs(r["bits_per_key"] - o.bits_per_key()) < 1e-12
    f.write_bytes(oracle_export(o)[:-8])
    assert fileinfo.main([str(f), "--json"]) == 2
    assert json.loads(capsys.readouterr().out)["status"] == "FORMAT"
