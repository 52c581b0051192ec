"""Export files written from the oracle's own arrays (test infrastructure).

The layout is the one phobic_export documents: a 28-word header, then the
packed offsets, the column metadata, the packed values / ranks / low parts,
the dictionary or the select samples followed by the unary bits, and the
Elias-Fano remap.  Nothing here comes from the CUDA path: a file built this way
lets the library's inspection and its GPU query path be checked against a
structure that the library never built.
"""
import struct

import numpy as np

MAGIC = 0x31304349424F4850  # "PHOBIC01"
VERSION = 1
M56 = (1 << 56) - 1


def _meta(o, enc, ncol):
    """Column metadata words: base | width << 56 (and the second word per column)."""
    if enc == 0:
        w, base = o.array("col_w").astype(np.uint64), o.array("col_base").astype(np.uint64)
        return base | (w << np.uint64(56))
    out = np.zeros(2 * ncol, dtype=np.uint64)
    if enc == 1:
        out[0::2] = o.array("col_rbase").astype(np.uint64) | (o.array("col_rw").astype(np.uint64) << np.uint64(56))
        out[1::2] = o.array("col_dbase").astype(np.uint64) | (o.array("col_dw").astype(np.uint64) << np.uint64(56))
    else:
        out[0::2] = o.array("col_lbase").astype(np.uint64) | (o.array("col_l").astype(np.uint64) << np.uint64(56))
        out[1::2] = o.array("col_hbase").astype(np.uint64)
    return out


def oracle_export(o, key_kind=0) -> bytes:
    """phobic_export-format bytes of the oracle structure `o` (an oracle.Oracle)."""
    prm = o.prm
    encoder = int(prm.encoder)
    mono = encoder >= 5
    enc = encoder - 5 if mono else encoder
    B = o.u64("B")
    ncol = 1 if mono else B
    cmix = min(int(prm.compact_columns), B) if encoder == 4 else 0
    arrays = [o.array("off_words").astype(np.uint64), _meta(o, enc, ncol)]
    if enc == 0:
        arrays += [o.array("pil_words"), np.zeros(0, np.uint64)]
    elif enc == 1:
        arrays += [o.array("rank_words"), o.array("dict_words")]
    else:
        samp = o.array("rice_samples").astype(np.uint32)
        padded = np.zeros(2 * ((samp.size + 1) // 2), dtype=np.uint32)
        padded[: samp.size] = samp
        arrays += [o.array("rice_low"), np.concatenate([padded.view(np.uint64), o.array("rice_high")])]
    if o.u64("ef_N"):
        arrays += [o.array("ef_low"), o.array("ef_high"), o.array("ef_samples")]
    else:
        arrays += [np.zeros(0, np.uint64)] * 3
    arrays = [np.ascontiguousarray(a).astype(np.uint64) for a in arrays]
    lam = struct.unpack("<Q", struct.pack("<d", float(prm.lambda_)))[0]
    alp = struct.unpack("<Q", struct.pack("<d", float(prm.alpha)))[0]
    hdr = [MAGIC, VERSION, o.u64("n"), o.u64("M"), o.u64("NP"), B, int(prm.partition_size), lam, alp, int(prm.seed),
           encoder | (int(prm.bucket_fn) << 32) | (cmix << 40), int(prm.pilot_mode) | (key_kind << 32),
           o.u64("off_w"), o.u64("off_Q"), o.u64("off_dmin") & (2**64 - 1), o.u64("ef_l")]
    hdr += [a.size for a in arrays]
    hdr += [o.u64(k) for k in ("bits_header", "bits_offsets", "bits_pilots", "bits_remap", "bits_total")]
    assert len(hdr) == 28
    return np.concatenate([np.array(hdr, dtype=np.uint64)] + arrays).tobytes()
