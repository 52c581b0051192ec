"""Published XXH64 known answers (tests/golden/xxh64_known_answers.json).

Each case is (message bytes, seed, expected hash).  The self-test buffers of
the xxHash command-line tool are generated here from their published
definition; they hold none of XXH64's arithmetic.
"""
import json
import os

_FIXTURE = os.path.join(os.path.dirname(__file__), "golden", "xxh64_known_answers.json")


def _buffer_v08(n, g0, mul):
    out, g = bytearray(), g0
    for _ in range(n):
        out.append(g >> 56)
        g = (g * mul) % 2**64
    return bytes(out)


def _buffer_v06(n, g0):
    out, g = bytearray(), g0
    for _ in range(n):
        out.append((g >> 24) & 0xFF)
        g = (g * g) % 2**32
    return bytes(out)


def cases():
    with open(_FIXTURE) as f:
        fx = json.load(f)
    out = []
    st = fx["selftest_buffer"]
    for c in st["cases"]:
        out.append((_buffer_v08(c["len"], st["prime32"], st["prime64"]), c["seed"], int(c["hash"], 16)))
    st = fx["selftest_buffer_v06"]
    for c in st["cases"]:
        out.append((_buffer_v06(c["len"], st["prime32"]), c["seed"], int(c["hash"], 16)))
    for c in fx["strings"]:
        out.append((c["text"].encode("ascii"), c["seed"], int(c["hash"], 16)))
    return out


def by_seed():
    """The cases grouped by seed: {seed: (data u8 array, offsets u64 array, expected list)}."""
    import numpy as np

    groups = {}
    for msg, seed, want in cases():
        groups.setdefault(seed, []).append((msg, want))
    out = {}
    for seed, items in groups.items():
        data = b"".join(m for m, _ in items)
        offs = np.concatenate([[0], np.cumsum([len(m) for m, _ in items])]).astype(np.uint64)
        arr = np.frombuffer(data + b"\0" * 8, dtype=np.uint8).copy()
        out[seed] = (arr, offs, [w for _, w in items])
    return out
