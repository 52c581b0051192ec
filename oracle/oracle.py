"""ctypes front end of the PHOBIC CPU oracle (test infrastructure only).

``build_oracle_lib()`` compiles ``phobic_oracle.c`` with gcc into
``liboracle.so`` next to it.  ``Oracle`` wraps one built structure and hands
its arrays out as numpy copies.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phobic_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

OK, INVALID_ARG, OOM, DUP_HASH, SEARCH_LIMIT = 0, 1, 2, 3, 4
ENC_IC_C, ENC_IC_D, ENC_IC_R, ENC_IC_EF, ENC_IC_CR = 0, 1, 2, 3, 4
# mono-X: encoder X over one column holding all pilots in column order
ENC_MONO_C, ENC_MONO_D, ENC_MONO_R, ENC_MONO_EF = 5, 6, 7, 8
PILOT_ADDITIVE, PILOT_XOR = 0, 1


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"oracle status {code} {what}")
        self.code = code


def build_oracle_lib(force: bool = False) -> str:
    """Compile the oracle (plain gcc, OpenMP over partitions, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "phobic_oracle.h"))
    ):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, "-lm",
        ]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("partition_size", ctypes.c_uint32),
        ("encoder", ctypes.c_uint32),
        ("pilot_mode", ctypes.c_uint32),
        ("s_max", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("bucket_fn", ctypes.c_uint32),
        ("compact_columns", ctypes.c_uint32),
    ]


BUCKET_OPTIMIZED, BUCKET_BETA_STAR, BUCKET_SKEWED, BUCKET_UNIFORM = 0, 1, 2, 3


def params(lam=7.0, alpha=1.0, P=2500, encoder=ENC_IC_C, mode=PILOT_ADDITIVE, s_max=0, seed=0, bucket_fn=0,
           compact_columns=0):
    return _Params(float(lam), float(alpha), int(P), int(encoder), int(mode), int(s_max), int(seed),
                   int(bucket_fn), int(compact_columns))


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle_lib())
        u64, u32, dbl, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
        P = ctypes.POINTER(_Params)
        L.or_mix64.restype = u64; L.or_mix64.argtypes = [u64]
        L.or_mulhi64.restype = u64; L.or_mulhi64.argtypes = [u64, u64]
        L.or_bitlen.restype = u32; L.or_bitlen.argtypes = [u64]
        L.or_rice_param.restype = u32; L.or_rice_param.argtypes = [u64, u64]
        L.or_beta_star.restype = dbl; L.or_beta_star.argtypes = [dbl]
        L.or_gamma.restype = dbl; L.or_gamma.argtypes = [dbl, dbl, dbl]
        L.or_epsilon.restype = dbl; L.or_epsilon.argtypes = [dbl, u32]
        L.or_bucket_table.restype = None; L.or_bucket_table.argtypes = [dbl, dbl, u32, vp]
        L.or_gamma_fn.restype = dbl; L.or_gamma_fn.argtypes = [dbl, dbl, dbl, u32]
        L.or_bucket_table_fn.restype = None; L.or_bucket_table_fn.argtypes = [dbl, dbl, u32, u32, vp]
        L.or_num_buckets.restype = u32; L.or_num_buckets.argtypes = [dbl, u32]
        L.or_num_partitions.restype = u64; L.or_num_partitions.argtypes = [u64, u32]
        L.or_bucket.restype = u32; L.or_bucket.argtypes = [u64, vp, u32]
        L.or_key_hash.restype = u64; L.or_key_hash.argtypes = [u64, u64]
        L.or_key_hash_array.restype = None; L.or_key_hash_array.argtypes = [vp, u64, u64, vp]
        L.or_string_hash_array.restype = None; L.or_string_hash_array.argtypes = [vp, vp, u64, u64, vp]
        L.or_bucket_hash.restype = u64; L.or_bucket_hash.argtypes = [u64]
        L.or_position_hash.restype = u64; L.or_position_hash.argtypes = [u64, u64, u64]
        L.or_table_size.restype = u64; L.or_table_size.argtypes = [u64, dbl]
        L.or_string_hash.restype = u64; L.or_string_hash.argtypes = [vp, u64, u64]
        L.or_build.restype = ctypes.c_int; L.or_build.argtypes = [vp, u64, P, ctypes.c_int, ctypes.POINTER(vp)]
        L.or_build_hashed.restype = ctypes.c_int
        L.or_build_hashed.argtypes = [vp, u64, P, ctypes.c_int, ctypes.POINTER(vp)]
        L.or_free.restype = None; L.or_free.argtypes = [vp]
        L.or_query.restype = None; L.or_query.argtypes = [vp, vp, u64, vp]
        L.or_query_hashed.restype = None; L.or_query_hashed.argtypes = [vp, vp, u64, vp]
        L.or_bits_per_key.restype = dbl; L.or_bits_per_key.argtypes = [vp]
        L.or_get_u64.restype = u64; L.or_get_u64.argtypes = [vp, ctypes.c_char_p]
        L.or_get_array.restype = vp
        L.or_get_array.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(u64), ctypes.POINTER(u32)]
        L.or_partition_sizes.restype = ctypes.c_int; L.or_partition_sizes.argtypes = [vp, u64, P, vp]
        L.or_search_partitions.restype = ctypes.c_int
        L.or_search_partitions.argtypes = [vp, u64, P, vp, u64, ctypes.c_int, vp]
        L.or_verify_first_valid.restype = ctypes.c_int; L.or_verify_first_valid.argtypes = [vp, vp]
        L.or_search_one_partition.restype = ctypes.c_int
        L.or_search_one_partition.argtypes = [vp, u64, P, vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


class Oracle:
    """One MPHF built by the oracle."""

    def __init__(self, keys=None, *, hashed=None, lam=7.0, alpha=1.0, P=2500, encoder=ENC_IC_C,
                 mode=PILOT_ADDITIVE, s_max=0, seed=0, threads=0, bucket_fn=0, compact_columns=0):
        L = lib()
        self.prm = params(lam, alpha, P, encoder, mode, s_max, seed, bucket_fn, compact_columns)
        h = ctypes.c_void_p()
        if hashed is not None:
            hk = _u64(hashed)
            st = L.or_build_hashed(_ptr(hk), hk.size, ctypes.byref(self.prm), threads, ctypes.byref(h))
        else:
            k = _u64(keys)
            st = L.or_build(_ptr(k), k.size, ctypes.byref(self.prm), threads, ctypes.byref(h))
        if st != OK:
            raise OracleError(st, "build")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().or_free(h)
            self._h = None

    def u64(self, name: str) -> int:
        v = lib().or_get_u64(self._h, name.encode())
        if name == "off_dmin":
            v = int(np.uint64(v).astype(np.int64))
        return int(v)

    def array(self, name: str) -> Optional[np.ndarray]:
        cnt, eb = ctypes.c_uint64(), ctypes.c_uint32()
        p = lib().or_get_array(self._h, name.encode(), ctypes.byref(cnt), ctypes.byref(eb))
        if not p:
            return None
        dt = {4: np.uint32, 8: np.uint64}[eb.value]
        buf = (ctypes.c_char * (cnt.value * eb.value)).from_address(p)
        return np.frombuffer(buf, dtype=dt).copy()

    def query(self, keys) -> np.ndarray:
        k = _u64(keys)
        out = np.empty_like(k)
        lib().or_query(self._h, _ptr(k), k.size, _ptr(out))
        return out

    def query_hashed(self, hk) -> np.ndarray:
        k = _u64(hk)
        out = np.empty_like(k)
        lib().or_query_hashed(self._h, _ptr(k), k.size, _ptr(out))
        return out

    def bits_per_key(self) -> float:
        return float(lib().or_bits_per_key(self._h))

    def verify_first_valid(self, hashed) -> bool:
        hk = _u64(hashed)
        return bool(lib().or_verify_first_valid(self._h, _ptr(hk)))

    @property
    def pilots(self) -> np.ndarray:
        B, NP = self.u64("B"), self.u64("NP")
        return self.array("pilots").reshape(B, NP)


# ---- free functions ----
def key_hash(keys, seed: int) -> np.ndarray:
    """master hash codes of 64-bit keys (the oracle's own restatement)"""
    k = _u64(keys)
    out = np.empty_like(k)
    lib().or_key_hash_array(_ptr(k), k.size, seed, _ptr(out))
    return out


def string_hashes(data: np.ndarray, offsets: np.ndarray, seed: int) -> np.ndarray:
    d = np.ascontiguousarray(data, dtype=np.uint8)
    o = _u64(offsets)
    out = np.empty(o.size - 1, dtype=np.uint64)
    lib().or_string_hash_array(_ptr(d), _ptr(o), out.size, seed, _ptr(out))
    return out


def search_one_partition(hk, lam, alpha, P, encoder=ENC_IC_C, mode=PILOT_ADDITIVE, s_max=0, bucket_fn=0):
    """(pilots [B], taken [m] as bool) of one partition holding the hashes hk."""
    L = lib()
    k = _u64(hk)
    prm = params(lam, alpha, P, encoder, mode, s_max, 0, bucket_fn)
    B = L.or_num_buckets(float(lam), int(P))
    m = L.or_table_size(k.size, float(alpha))
    pil = np.zeros(B, dtype=np.uint32)
    taken = np.zeros(m + 1, dtype=np.uint8)
    st = L.or_search_one_partition(_ptr(k) if k.size else None, k.size, ctypes.byref(prm), _ptr(pil), _ptr(taken))
    if st != OK:
        raise OracleError(st, "search_one_partition")
    return pil, taken[:m].astype(bool)


def partition_sizes(hk, lam, alpha, P, seed=0) -> np.ndarray:
    L = lib()
    hk = _u64(hk)
    prm = params(lam, alpha, P, seed=seed)
    NP = L.or_num_partitions(hk.size, P)
    out = np.zeros(NP, dtype=np.uint64)
    st = L.or_partition_sizes(_ptr(hk), hk.size, ctypes.byref(prm), _ptr(out))
    if st != OK:
        raise OracleError(st, "partition_sizes")
    return out


def search_partitions(hk, sel, lam=7.0, alpha=1.0, P=2500, mode=PILOT_ADDITIVE, s_max=0,
                      threads=0) -> np.ndarray:
    L = lib()
    hk = _u64(hk)
    sel = _u64(sel)
    prm = params(lam, alpha, P, ENC_IC_C, mode, s_max)
    B = L.or_num_buckets(lam, P)
    out = np.zeros((sel.size, B), dtype=np.uint32)
    st = L.or_search_partitions(_ptr(hk), hk.size, ctypes.byref(prm), _ptr(sel), sel.size, threads, _ptr(out))
    if st != OK:
        raise OracleError(st, "search_partitions")
    return out


def bucket_table(lam, alpha, P, bucket_fn=0) -> np.ndarray:
    t = np.zeros(2049, dtype=np.uint64)
    lib().or_bucket_table_fn(lam, alpha, P, bucket_fn, _ptr(t))
    return t


def string_hash(b: bytes, seed: int = 0) -> int:
    buf = ctypes.create_string_buffer(b, len(b))
    return int(lib().or_string_hash(ctypes.addressof(buf), len(b), seed))
