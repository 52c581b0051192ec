"""Inspects a file written from phobic_export bytes.

    python -m paper_2404_18497_b300.fileinfo STRUCTURE.bin [--keys KEYS.npy] [--json]

The checks and the parameters come from phobic_inspect, which validates the bytes
on the host exactly as phobic_import would before copying them to a device, so
no GPU is needed to tell whether a file is loadable and what it holds.  With
--keys (a .npy array of uint64 keys), the structure is imported on cuda:0 and
every key is queried: the tool then also reports whether the keys map one-to-one
onto [0, n).

Exit status: 0 valid (and, with --keys, a bijection), 1 a valid file whose
queries are not a bijection, 2 bytes that phobic_import would refuse.
"""
from __future__ import annotations

import argparse
import json
import sys

ENCODER_NAMES = {0: "IC-C", 1: "IC-D", 2: "IC-R", 3: "IC-EF", 4: "IC-CR",
                 5: "mono-C", 6: "mono-D", 7: "mono-R", 8: "mono-EF"}
BUCKET_FUNCTIONS = {0: "beta_eps", 1: "beta_star", 2: "skewed 60/30", 3: "uniform"}


def describe(info: dict) -> dict:
    """Human-readable fields of phobic_inspect's info."""
    n = info["n"]
    out = {
        "n": n,
        "table_slots_M": info["M"],
        "partitions": info["num_partitions"],
        "buckets_per_partition": info["num_buckets"],
        "partition_size": info["partition_size"],
        "lambda": info["lambda"],
        "alpha": info["alpha"],
        "epsilon": info["epsilon"],
        "encoder": ENCODER_NAMES.get(info["encoder"], str(info["encoder"])),
        "pilot_form": "additive displacement" if info["pilot_mode"] == 0 else "xor",
        "bucket_function": BUCKET_FUNCTIONS.get(info["bucket_function"], str(info["bucket_function"])),
        "seed": info["seed"],
        "bits_per_key": info["bits_total"] / n if n else float("nan"),
        "bits_per_key_parts": {k: info["bits_" + k] / n if n else float("nan")
                               for k in ("header", "offsets", "pilots", "remap")},
        "device_bytes_when_imported": info["device_bytes"],
    }
    if info["encoder"] == 4:
        out["compact_columns"] = info["compact_columns"]
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("structure", help="file holding phobic_export bytes")
    ap.add_argument("--keys", help=".npy array of uint64 keys to query on cuda:0")
    ap.add_argument("--json", action="store_true", help="one JSON object on stdout")
    a = ap.parse_args(argv)

    from . import phobic

    with open(a.structure, "rb") as f:
        data = f.read()
    report = {"file": a.structure, "bytes": len(data)}
    try:
        info = phobic.phobic_inspect(data)
    except phobic.PhobicError as e:
        report.update(valid=False, status=e.status)
        print(json.dumps(report) if a.json else f"{a.structure}: not a loadable structure ({e.status})")
        return 2
    report.update(valid=True, **describe(info))
    code = 0
    if a.keys:
        import numpy as np
        import torch

        keys = np.load(a.keys)
        h = phobic.phobic_import(data)
        try:
            out = h.query(torch.from_numpy(keys.astype(np.uint64).view(np.int64)).cuda())
            ok = keys.size == info["n"] and bool(
                torch.equal(torch.sort(out).values, torch.arange(keys.size, device="cuda")))
        finally:
            h.free()
        report.update(keys_queried=int(keys.size), bijection=ok)
        code = 0 if ok else 1
    if a.json:
        print(json.dumps(report))
    else:
        for k, v in report.items():
            print(f"{k:28s} {v}")
    return code


if __name__ == "__main__":
    sys.exit(main())
