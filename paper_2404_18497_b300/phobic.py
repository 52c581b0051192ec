"""Python binding of libphobic (argument marshalling only).

Every function mirrors one C entry point of include/phobic.h under the same
name.  Device buffers are torch CUDA tensors: 64-bit keys as int64 or uint64
(bit patterns are passed through unchanged), outputs as int64.  Streams are
torch.cuda streams; the default is torch's current stream.  All computation
happens in the library's CUDA kernels: if libphobic.so is missing, importing
this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libphobic.so")

OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "DUP_HASH", 4: "SEARCH_LIMIT",
    5: "PARTITION_TOO_LARGE", 6: "CUDA", 7: "TIMEOUT", 8: "FORMAT",
}
ENC_IC_C, ENC_IC_D, ENC_IC_R, ENC_IC_EF, ENC_IC_CR = 0, 1, 2, 3, 4
# mono-X: the column encoder X over one column holding all pilots (Section 5, Fig. 3b)
ENC_MONO_C, ENC_MONO_D, ENC_MONO_R, ENC_MONO_EF = 5, 6, 7, 8
PILOT_ADDITIVE, PILOT_XOR = 0, 1
_ENC = {"IC-C": ENC_IC_C, "IC-D": ENC_IC_D, "IC-R": ENC_IC_R, "IC-EF": ENC_IC_EF, "IC-CR": ENC_IC_CR,
        "mono-C": ENC_MONO_C, "mono-D": ENC_MONO_D, "mono-R": ENC_MONO_R, "mono-EF": ENC_MONO_EF}
_ENC.update({v: v for v in list(_ENC.values())})
_MODE = {"additive": PILOT_ADDITIVE, "xor": PILOT_XOR, PILOT_ADDITIVE: PILOT_ADDITIVE, PILOT_XOR: PILOT_XOR}


class PhobicError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")
        self.code = code
        self.status = STATUS_NAMES.get(code, str(code))


class phobic_params(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("partition_size", ctypes.c_uint32),
        ("encoder", ctypes.c_uint32),
        ("pilot_mode", ctypes.c_uint32),
        ("s_max", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("warps_per_partition", ctypes.c_uint32),
        ("keep_pilots", ctypes.c_uint32),
        ("record_timings", ctypes.c_uint32),
        ("candidate_width", ctypes.c_uint32),
        ("search_schedule", ctypes.c_uint32),
        ("bucket_function", ctypes.c_uint32),
        ("compact_columns", ctypes.c_uint32),
    ]


class phobic_timings(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("sort_ms", "sizes_ms", "search_ms", "encode_ms", "remap_ms", "total_ms")] + [
        ("search_s_tries", ctypes.c_uint64), ("search_steps", ctypes.c_uint64)]


class phobic_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64), ("M", ctypes.c_uint64), ("num_partitions", ctypes.c_uint64),
        ("num_buckets", ctypes.c_uint32), ("partition_size", ctypes.c_uint32),
        ("lambda_", ctypes.c_double), ("alpha", ctypes.c_double), ("epsilon", ctypes.c_double),
        ("encoder", ctypes.c_uint32), ("pilot_mode", ctypes.c_uint32), ("seed", ctypes.c_uint64),
        ("max_partition", ctypes.c_uint64),
        ("bits_header", ctypes.c_uint64), ("bits_offsets", ctypes.c_uint64), ("bits_pilots", ctypes.c_uint64),
        ("bits_remap", ctypes.c_uint64), ("bits_total", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
        ("bucket_function", ctypes.c_uint32), ("compact_columns", ctypes.c_uint32),
    ]


_lib = None
# (name, restype, argtypes): the C ABI, in header order
REQ_BUILD, REQ_QUERY, REQ_RELEASE = 0, 1, 2


class phobic_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("build_slots", ctypes.c_uint32),
                ("max_batch_requests", ctypes.c_uint32), ("max_batch_keys", ctypes.c_uint64),
                ("launch_slots", ctypes.c_uint32), ("serial", ctypes.c_uint32)]


class phobic_completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("kind", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("handle_id", ctypes.c_uint64), ("keys", ctypes.c_uint64), ("t_submit_ns", ctypes.c_int64),
                ("t_start_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64), ("batch_requests", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("batch_id", ctypes.c_uint64)]


COMPLETION_DTYPE = np.dtype([(n, np.dtype(t._type_)) for n, t in phobic_completion._fields_], align=True)


class phobic_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "resident_bytes", "reserved_bytes", "peak_accounted_bytes", "resident_handles", "builds_done",
        "queries_done", "releases_done", "query_launches", "max_batch_requests_seen", "builds_waited_for_memory",
        "pending")]


TUNE_P_CHOICES = (1024, 2500, 4096)
TUNE_MAX_CLASSES = 20


class phobic_tune_class(ctypes.Structure):
    _fields_ = [("sets", ctypes.c_uint32), ("partition_size", ctypes.c_uint32),
                ("ns_per_key", ctypes.c_float * 3), ("bits_per_key", ctypes.c_float * 3)]


class phobic_tune_info(ctypes.Structure):
    _fields_ = [("classes", phobic_tune_class * TUNE_MAX_CLASSES),
                ("warps_per_partition", ctypes.c_uint32), ("candidate_width", ctypes.c_uint32),
                ("launch_ns_per_key", ctypes.c_float * 6), ("total_partitions", ctypes.c_uint64),
                ("cached_classes", ctypes.c_uint32), ("cached_launch", ctypes.c_uint32),
                ("search_schedule", ctypes.c_uint32), ("schedule_ns_per_key", ctypes.c_float * 2)]


_VP, _U64, _U32, _DBL, _INT = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
_PP = ctypes.POINTER(phobic_params)
_SIGS = [
    ("phobic_params_init", None, [_PP]),
    ("phobic_build", _INT, [_VP, _U64, _DBL, _DBL, _U32, _U64, _VP, ctypes.POINTER(_VP)]),
    ("phobic_build_ex", _INT, [_VP, _U64, _PP, _VP, ctypes.POINTER(_VP)]),
    ("phobic_build_batch", _INT, [_VP, _VP, _U32, _VP, _PP, _VP, ctypes.POINTER(_VP)]),
    ("phobic_build_host", _INT, [_VP, _U64, _PP, _VP, ctypes.POINTER(_VP)]),
    ("phobic_query", _INT, [_VP, _VP, _VP, _U64, _VP]),
    ("phobic_build_strings", _INT, [_VP, _VP, _U64, _PP, _VP, ctypes.POINTER(_VP)]),
    ("phobic_query_strings", _INT, [_VP, _VP, _VP, _VP, _U64, _VP]),
    ("phobic_query_host", _INT, [_VP, _VP, _VP, _U64, _VP]),
    ("phobic_bits_per_key", _DBL, [_VP]),
    ("phobic_get_info", _INT, [_VP, ctypes.POINTER(phobic_info)]),
    ("phobic_export", _INT, [_VP, _VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("phobic_import", _INT, [_VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    ("phobic_inspect", _INT, [_VP, ctypes.c_size_t, ctypes.POINTER(phobic_info)]),
    ("phobic_copy_pilots", _INT, [_VP, _VP, _VP]),
    ("phobic_get_timings", _INT, [_VP, ctypes.POINTER(phobic_timings)]),
    ("phobic_kernel_launches", _U64, []),
    ("phobic_free", None, [_VP]),
    ("phobic_status_str", ctypes.c_char_p, [_INT]),
    ("phobic_hash_u64", _INT, [_VP, _U64, _U64, _VP, _VP]),
    ("phobic_hash_strings", _INT, [_VP, _VP, _U64, _U64, _VP, _VP]),
    ("phobic_partition_sort", _INT, [_VP, _U64, _U64, _VP, _VP, _VP]),
    ("phobic_partition_sort_noalloc", _INT, [_VP, _U64, _U64, _VP, _VP, _VP]),
    ("phobic_selftest_sort_wait_timeout", _INT, [_VP, _U64, _U64, _U64, _U32, _VP, _VP, _VP]),
    ("phobic_bucket_table", _INT, [_DBL, _DBL, _U32, _VP]),
    ("phobic_bucket_table_ex", _INT, [_DBL, _DBL, _U32, _U32, _VP]),
    ("phobic_tune_batch", _INT, [_VP, _U32, _PP, _VP, _VP, _PP, ctypes.POINTER(phobic_tune_info)]),
    ("phobic_tune_clear", None, []),
    ("phobic_trim", _INT, [_U64]),
    ("phobic_query_multi", _INT, [_VP, _VP, _VP, _VP, _U32, _VP]),
    ("phobic_server_config_init", None, [ctypes.POINTER(phobic_server_config)]),
    ("phobic_server_create", _INT, [ctypes.POINTER(phobic_server_config), ctypes.POINTER(_VP)]),
    ("phobic_server_submit_build", _INT, [_VP, _VP, _U64, _PP, _VP, ctypes.POINTER(_U64)]),
    ("phobic_server_submit_query", _INT, [_VP, _U64, _VP, _VP, _U64, _VP, ctypes.POINTER(_U64)]),
    ("phobic_server_submit_release", _INT, [_VP, _U64, ctypes.POINTER(_U64)]),
    ("phobic_server_poll", _INT, [_VP, _VP, _U32, ctypes.POINTER(_U32)]),
    ("phobic_server_drain", _INT, [_VP, _DBL]),
    ("phobic_server_handle", _INT, [_VP, _U64, ctypes.POINTER(_VP)]),
    ("phobic_server_get_stats", _INT, [_VP, ctypes.POINTER(phobic_server_stats)]),
    ("phobic_server_destroy", None, [_VP]),
    ("phobic_pool_bytes", _INT, [ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    ("phobic_table_offsets", _INT, [_VP, _U64, _DBL, _VP, _VP, _VP]),
    ("phobic_search_partitions", _INT, [_VP, _U64, _VP, _VP, _U64, _U64, _U64, _U64, _PP, _VP, _VP, _VP]),
    ("phobic_assemble", _INT, [_VP, _U64, _VP, _VP, _PP, _VP, ctypes.POINTER(_VP)]),
]


def lib() -> ctypes.CDLL:
    """The loaded libphobic.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libphobic.so is not built ({LIB_PATH}); run python -m paper_2404_18497_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return [s[0] for s in _SIGS]


def _check(code: int, what: str):
    if code != OK:
        raise PhobicError(code, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev_u64(t: torch.Tensor, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError(f"{what} must be int64 or uint64")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t


def make_params(lam=7.0, alpha=1.0, P=2500, seed=0, encoder="IC-C", mode="additive", s_max=0,
                keep_pilots=False, warps_per_partition=0, record_timings=False,
                candidate_width=0, search_schedule=0, bucket_function=0, compact_columns=0) -> phobic_params:
    p = phobic_params()
    lib().phobic_params_init(ctypes.byref(p))
    p.lambda_ = float(lam)
    p.alpha = float(alpha)
    p.partition_size = int(P)
    p.seed = int(seed) & ((1 << 64) - 1)
    p.encoder = _ENC[encoder]
    p.pilot_mode = _MODE[mode]
    if s_max:
        p.s_max = int(s_max)
    p.keep_pilots = 1 if keep_pilots else 0
    p.warps_per_partition = int(warps_per_partition)
    p.record_timings = 1 if record_timings else 0
    p.candidate_width = int(candidate_width)
    p.search_schedule = int(search_schedule)
    p.bucket_function = int(bucket_function)
    p.compact_columns = int(compact_columns)
    return p


class Handle:
    """One built MPHF (owns the C handle unless borrowed)."""

    def __init__(self, ptr: int, borrowed: bool = False):
        self._h = ctypes.c_void_p(ptr)
        self._borrowed = borrowed

    @property
    def ptr(self) -> ctypes.c_void_p:
        if not self._h.value:
            raise ValueError("handle was freed")
        return self._h

    def free(self):
        if self._h.value and not self._borrowed:
            lib().phobic_free(self._h)
        self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # conveniences over the entry points below
    def query(self, keys: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        return phobic_query(self, keys, out, stream)

    def bits_per_key(self) -> float:
        return phobic_bits_per_key(self)

    def info(self) -> dict:
        return phobic_get_info(self)

    def export(self) -> bytes:
        return phobic_export(self)

    def pilots(self, stream=None) -> torch.Tensor:
        return phobic_copy_pilots(self, stream)


# ---------------------------------------------------------------- entry points
def phobic_build(keys: torch.Tensor, lam=7.0, alpha=1.0, P=2500, seed=0, stream=None) -> Handle:
    k = _dev_u64(keys, "keys")
    h = ctypes.c_void_p()
    _check(lib().phobic_build(k.data_ptr(), k.numel(), float(lam), float(alpha), int(P), int(seed),
                              _stream(stream), ctypes.byref(h)), "phobic_build")
    return Handle(h.value)


def phobic_build_ex(keys: torch.Tensor, params: phobic_params, stream=None) -> Handle:
    k = _dev_u64(keys, "keys")
    h = ctypes.c_void_p()
    _check(lib().phobic_build_ex(k.data_ptr(), k.numel(), ctypes.byref(params), _stream(stream), ctypes.byref(h)),
           "phobic_build_ex")
    return Handle(h.value)


def phobic_build_batch(keys: torch.Tensor, set_offsets, params: phobic_params, partition_sizes=None,
                       stream=None) -> list:
    """One handle per key set; set s is keys[set_offsets[s]:set_offsets[s+1]]."""
    k = _dev_u64(keys, "keys")
    off = np.ascontiguousarray(np.asarray(set_offsets, dtype=np.uint64))
    ns = off.size - 1
    if ns < 1 or int(off[-1]) > k.numel():
        raise ValueError("bad set offsets")
    ps = None if partition_sizes is None else np.ascontiguousarray(np.asarray(partition_sizes, dtype=np.uint32))
    if ps is not None and ps.size != ns:
        raise ValueError("one partition size per set")
    outs = (ctypes.c_void_p * ns)()
    _check(lib().phobic_build_batch(k.data_ptr(), off.ctypes.data, ns, None if ps is None else ps.ctypes.data,
                                    ctypes.byref(params), _stream(stream), outs), "phobic_build_batch")
    return [Handle(outs[i]) for i in range(ns)]


def phobic_tune_batch(set_offsets, params: phobic_params, stream=None):
    """Autotuned (partition sizes per set, params with the search knobs, info dict)
    for a batch with these set offsets; see phobic_tune_batch in the header."""
    off = np.ascontiguousarray(np.asarray(set_offsets, dtype=np.uint64))
    ns = off.size - 1
    if ns < 1:
        raise ValueError("bad set offsets")
    ps = np.zeros(ns, dtype=np.uint32)
    pout = phobic_params()
    info = phobic_tune_info()
    _check(lib().phobic_tune_batch(off.ctypes.data, ns, ctypes.byref(params), _stream(stream), ps.ctypes.data,
                                   ctypes.byref(pout), ctypes.byref(info)), "phobic_tune_batch")
    classes = {}
    for c in range(TUNE_MAX_CLASSES):
        tc = info.classes[c]
        if tc.sets:
            classes[c] = dict(sets=tc.sets, partition_size=tc.partition_size,
                              ns_per_key=dict(zip(TUNE_P_CHOICES, map(float, tc.ns_per_key))),
                              bits_per_key=dict(zip(TUNE_P_CHOICES, map(float, tc.bits_per_key))))
    combos = [(w, cw) for w in (1, 2, 4) for cw in (32, 64)]
    d = dict(classes=classes, warps_per_partition=info.warps_per_partition, candidate_width=info.candidate_width,
             launch_ns_per_key={f"w{w}/c{cw}": float(v) for (w, cw), v in zip(combos, info.launch_ns_per_key)},
             total_partitions=int(info.total_partitions), cached_classes=info.cached_classes,
             cached_launch=info.cached_launch, search_schedule=info.search_schedule,
             schedule_ns_per_key={"cta_per_partition": float(info.schedule_ns_per_key[0]),
                                  "work_queue": float(info.schedule_ns_per_key[1])})
    return ps, pout, d


def phobic_query_multi(handles, keys, outs, stream=None) -> None:
    """One coalesced launch: keys[r] against handles[r] into outs[r]."""
    n = len(handles)
    if not (len(keys) == len(outs) == n):
        raise ValueError("one key and one output tensor per handle")
    hs = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    ks = (ctypes.c_void_p * n)(*[_dev_u64(k, "keys").data_ptr() for k in keys])
    os_ = (ctypes.c_void_p * n)()
    cs = (ctypes.c_uint64 * n)()
    for i, (k, o) in enumerate(zip(keys, outs)):
        o = _dev_u64(o, "out")
        if o.numel() < k.numel():
            raise ValueError("out shorter than keys")
        os_[i] = o.data_ptr()
        cs[i] = k.numel()
    _check(lib().phobic_query_multi(hs, ks, os_, cs, n, _stream(stream)), "phobic_query_multi")


class Server:
    """Serving loop over resident MPHFs (see phobic_server_* in the header).
    Keys and outputs are CUDA tensors that the caller keeps alive until the
    request's completion has been polled."""

    def __init__(self, hbm_budget_bytes=0, build_slots=2, max_batch_requests=1024, max_batch_keys=1 << 24,
                 launch_slots=4, serial=False):
        c = phobic_server_config()
        lib().phobic_server_config_init(ctypes.byref(c))
        c.hbm_budget_bytes, c.build_slots, c.max_batch_requests = int(hbm_budget_bytes), build_slots, max_batch_requests
        c.max_batch_keys, c.launch_slots, c.serial = int(max_batch_keys), launch_slots, int(bool(serial))
        p = ctypes.c_void_p()
        _check(lib().phobic_server_create(ctypes.byref(c), ctypes.byref(p)), "phobic_server_create")
        self._s = p
        self._buf = np.zeros(4096, dtype=COMPLETION_DTYPE)

    @staticmethod
    def _ev(ready):
        return None if ready is None else ready.cuda_event if hasattr(ready, "cuda_event") else int(ready)

    def submit_build(self, keys: torch.Tensor, params: phobic_params, ready=None) -> int:
        k = _dev_u64(keys, "keys")
        rid = _U64()
        _check(lib().phobic_server_submit_build(self._s, k.data_ptr(), k.numel(), ctypes.byref(params),
                                                self._ev(ready), ctypes.byref(rid)), "phobic_server_submit_build")
        return int(rid.value)

    def submit_query(self, handle_id: int, keys: torch.Tensor, out: torch.Tensor, ready=None) -> int:
        k, o = _dev_u64(keys, "keys"), _dev_u64(out, "out")
        if o.numel() < k.numel():
            raise ValueError("out shorter than keys")
        rid = _U64()
        _check(lib().phobic_server_submit_query(self._s, int(handle_id), k.data_ptr(), o.data_ptr(), k.numel(),
                                                self._ev(ready), ctypes.byref(rid)), "phobic_server_submit_query")
        return int(rid.value)

    def submit_release(self, handle_id: int) -> int:
        rid = _U64()
        _check(lib().phobic_server_submit_release(self._s, int(handle_id), ctypes.byref(rid)),
               "phobic_server_submit_release")
        return int(rid.value)

    def poll(self) -> np.ndarray:
        """Completed requests since the last poll (structured array, oldest first)."""
        out = []
        while True:
            cnt = _U32()
            _check(lib().phobic_server_poll(self._s, self._buf.ctypes.data, self._buf.size, ctypes.byref(cnt)),
                   "phobic_server_poll")
            out.append(self._buf[: cnt.value].copy())
            if cnt.value < self._buf.size:
                break
        return np.concatenate(out)

    def drain(self, timeout_s: float = 600.0) -> None:
        _check(lib().phobic_server_drain(self._s, float(timeout_s)), "phobic_server_drain")

    def handle(self, handle_id: int) -> Handle:
        p = ctypes.c_void_p()
        _check(lib().phobic_server_handle(self._s, int(handle_id), ctypes.byref(p)), "phobic_server_handle")
        return Handle(p.value, borrowed=True)

    def stats(self) -> dict:
        st = phobic_server_stats()
        _check(lib().phobic_server_get_stats(self._s, ctypes.byref(st)), "phobic_server_get_stats")
        return {f[0]: int(getattr(st, f[0])) for f in phobic_server_stats._fields_}

    def close(self) -> None:
        if self._s is not None and self._s.value:
            lib().phobic_server_destroy(self._s)
        self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def phobic_trim(keep_bytes: int = 0) -> None:
    _check(lib().phobic_trim(int(keep_bytes)), "phobic_trim")


def phobic_pool_bytes() -> tuple:
    r, u = _U64(), _U64()
    _check(lib().phobic_pool_bytes(ctypes.byref(r), ctypes.byref(u)), "phobic_pool_bytes")
    return int(r.value), int(u.value)


def phobic_tune_clear() -> None:
    lib().phobic_tune_clear()


def phobic_build_host(keys: np.ndarray, params: phobic_params, stream=None) -> Handle:
    k = np.ascontiguousarray(keys).view(np.uint64)
    h = ctypes.c_void_p()
    _check(lib().phobic_build_host(k.ctypes.data, k.size, ctypes.byref(params), _stream(stream), ctypes.byref(h)),
           "phobic_build_host")
    return Handle(h.value)


def phobic_query(h: Handle, keys: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    k = _dev_u64(keys, "keys")
    if out is None:
        out = torch.empty(k.numel(), dtype=torch.int64, device=k.device)
    _dev_u64(out, "out")
    if out.numel() < k.numel():
        raise ValueError("out is too small")
    _check(lib().phobic_query(h.ptr, k.data_ptr(), out.data_ptr(), k.numel(), _stream(stream)), "phobic_query")
    return out


def _dev_bytes(t: torch.Tensor, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous CUDA uint8 tensor")
    return t


def phobic_build_strings(data: torch.Tensor, offsets: torch.Tensor, params: phobic_params, stream=None) -> Handle:
    d = _dev_bytes(data, "data")
    o = _dev_u64(offsets, "offsets")
    h = ctypes.c_void_p()
    _check(lib().phobic_build_strings(d.data_ptr(), o.data_ptr(), o.numel() - 1, ctypes.byref(params),
                                      _stream(stream), ctypes.byref(h)), "phobic_build_strings")
    return Handle(h.value)


def phobic_query_strings(h: Handle, data: torch.Tensor, offsets: torch.Tensor, out: Optional[torch.Tensor] = None,
                         stream=None) -> torch.Tensor:
    d = _dev_bytes(data, "data")
    o = _dev_u64(offsets, "offsets")
    m = o.numel() - 1
    if out is None:
        out = torch.empty(max(m, 0), dtype=torch.int64, device=o.device)
    _check(lib().phobic_query_strings(h.ptr, d.data_ptr(), o.data_ptr(), out.data_ptr(), m, _stream(stream)),
           "phobic_query_strings")
    return out


def phobic_query_host(h: Handle, keys: np.ndarray, out: Optional[np.ndarray] = None, stream=None) -> np.ndarray:
    k = np.ascontiguousarray(keys).view(np.uint64)
    if out is None:
        out = np.empty(k.size, dtype=np.uint64)
    _check(lib().phobic_query_host(h.ptr, k.ctypes.data, out.ctypes.data, k.size, _stream(stream)),
           "phobic_query_host")
    return out


def phobic_bits_per_key(h: Handle) -> float:
    return float(lib().phobic_bits_per_key(h.ptr))


def phobic_get_info(h: Handle) -> dict:
    i = phobic_info()
    _check(lib().phobic_get_info(h.ptr, ctypes.byref(i)), "phobic_get_info")
    return {f[0].rstrip("_"): getattr(i, f[0]) for f in phobic_info._fields_}


def phobic_export(h: Handle) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().phobic_export(h.ptr, None, ctypes.byref(n)), "phobic_export")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().phobic_export(h.ptr, buf, ctypes.byref(n)), "phobic_export")
    return buf.raw[: n.value]


def phobic_import(data: bytes, stream=None) -> Handle:
    buf = ctypes.create_string_buffer(data, len(data))
    h = ctypes.c_void_p()
    _check(lib().phobic_import(buf, len(data), _stream(stream), ctypes.byref(h)), "phobic_import")
    return Handle(h.value)


def phobic_inspect(data: bytes) -> dict:
    """Validates phobic_export bytes on the host (no device) and returns the
    info the imported handle would report; raises PhobicError (FORMAT) when
    phobic_import would refuse them."""
    buf = ctypes.create_string_buffer(data, len(data))
    i = phobic_info()
    _check(lib().phobic_inspect(buf, len(data), ctypes.byref(i)), "phobic_inspect")
    return {f[0].rstrip("_"): getattr(i, f[0]) for f in phobic_info._fields_}


def phobic_copy_pilots(h: Handle, stream=None) -> torch.Tensor:
    info = phobic_get_info(h)
    out = torch.empty((info["num_buckets"], info["num_partitions"]), dtype=torch.int32, device="cuda")
    _check(lib().phobic_copy_pilots(h.ptr, out.data_ptr(), _stream(stream)), "phobic_copy_pilots")
    return out


def phobic_get_timings(h: Handle) -> dict:
    t = phobic_timings()
    _check(lib().phobic_get_timings(h.ptr, ctypes.byref(t)), "phobic_get_timings")
    return {f[0]: (float if f[1] is ctypes.c_float else int)(getattr(t, f[0])) for f in phobic_timings._fields_}


def phobic_table_offsets(start: torch.Tensor, alpha: float, stream=None):
    """Slot offsets T [N_P + 1] (int64) from partition starts [N_P + 1], and
    (M, largest n_j, largest m_j)."""
    st = _dev_u64(start, "start")
    np_ = st.numel() - 1
    T = torch.empty(max(np_ + 1, 1), dtype=torch.int64, device=st.device)
    stats = (ctypes.c_uint64 * 3)()
    _check(lib().phobic_table_offsets(st.data_ptr(), np_, float(alpha), T.data_ptr(), stats, _stream(stream)),
           "phobic_table_offsets")
    return T, (int(stats[0]), int(stats[1]), int(stats[2]))


def _dev_u32(t: torch.Tensor, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.int32, torch.uint32):
        raise TypeError(f"{what} must be a CUDA int32 or uint32 tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t


def phobic_search_partitions(sorted_hk: torch.Tensor, start: torch.Tensor, T: torch.Tensor, n: int,
                             num_partitions: int, j0: int, j1: int, params: phobic_params, pilots: torch.Tensor,
                             taken: Optional[torch.Tensor] = None, stream=None) -> None:
    """Pilot search of partitions [j0, j1) of an n-key build into the whole
    build's pilot matrix `pilots` (int32, B x N_P) and occupancy bitmap `taken`
    (int32 words, or None)."""
    st, TT = _dev_u64(start, "start"), _dev_u64(T, "T")
    srt = _dev_u64(sorted_hk, "sorted_hk") if sorted_hk.numel() else None
    pl = _dev_u32(pilots, "pilots")
    tk = None if taken is None else _dev_u32(taken, "taken")
    _check(lib().phobic_search_partitions(None if srt is None else srt.data_ptr(), sorted_hk.numel(), st.data_ptr(),
                                          TT.data_ptr(), int(n), int(num_partitions), int(j0), int(j1),
                                          ctypes.byref(params), pl.data_ptr(), None if tk is None else tk.data_ptr(),
                                          _stream(stream)), "phobic_search_partitions")


def phobic_assemble(start: torch.Tensor, n: int, pilots: torch.Tensor, taken: Optional[torch.Tensor],
                    params: phobic_params, stream=None) -> Handle:
    """The structure of an n-key build from its partition starts, pilots and
    occupancy bitmap."""
    st = _dev_u64(start, "start")
    pl = _dev_u32(pilots, "pilots")
    tk = None if taken is None else _dev_u32(taken, "taken")
    h = ctypes.c_void_p()
    _check(lib().phobic_assemble(st.data_ptr(), int(n), pl.data_ptr(), None if tk is None else tk.data_ptr(),
                                 ctypes.byref(params), _stream(stream), ctypes.byref(h)), "phobic_assemble")
    return Handle(h.value)


def phobic_kernel_launches() -> int:
    return int(lib().phobic_kernel_launches())


def phobic_hash_u64(keys: torch.Tensor, seed: int = 0, out: Optional[torch.Tensor] = None, stream=None):
    k = _dev_u64(keys, "keys")
    if out is None:
        out = torch.empty_like(k, dtype=torch.int64)
    _check(lib().phobic_hash_u64(k.data_ptr(), k.numel(), int(seed), out.data_ptr(), _stream(stream)),
           "phobic_hash_u64")
    return out


def phobic_hash_strings(data: torch.Tensor, offsets: torch.Tensor, seed: int = 0, stream=None) -> torch.Tensor:
    if data.dtype != torch.uint8 or not data.is_cuda:
        raise TypeError("data must be a CUDA uint8 tensor")
    o = _dev_u64(offsets, "offsets")
    n = o.numel() - 1
    out = torch.empty(max(n, 0), dtype=torch.int64, device=o.device)
    _check(lib().phobic_hash_strings(data.data_ptr(), o.data_ptr(), n, int(seed), out.data_ptr(), _stream(stream)),
           "phobic_hash_strings")
    return out


def phobic_partition_sort(hk: torch.Tensor, num_partitions: int, stream=None):
    h = _dev_u64(hk, "hk")
    sorted_ = torch.empty_like(h, dtype=torch.int64)
    start = torch.empty(num_partitions + 1, dtype=torch.int64, device=h.device)
    _check(lib().phobic_partition_sort(h.data_ptr(), h.numel(), int(num_partitions), sorted_.data_ptr(),
                                       start.data_ptr(), _stream(stream)), "phobic_partition_sort")
    return sorted_, start


def phobic_selftest_sort_wait_timeout(hk: torch.Tensor, num_partitions: int, mute_tile: int, spin_limit: int,
                                      stream=None) -> int:
    """Runs the partition sort with one tile withholding its look-back state;
    returns the status code (TIMEOUT when a bounded wait ran out)."""
    h = _dev_u64(hk, "hk")
    sorted_ = torch.empty_like(h, dtype=torch.int64)
    start = torch.empty(num_partitions + 1, dtype=torch.int64, device=h.device)
    return int(lib().phobic_selftest_sort_wait_timeout(h.data_ptr(), h.numel(), int(num_partitions), int(mute_tile),
                                                       int(spin_limit), sorted_.data_ptr(), start.data_ptr(),
                                                       _stream(stream)))


NOALLOC_MAX_KEYS = 1048576


def phobic_partition_sort_noalloc(hk: torch.Tensor, num_partitions: int, sorted_out: torch.Tensor,
                                  start_out: torch.Tensor, stream=None):
    """Same as phobic_partition_sort, but the caller provides both outputs and
    the library uses its fixed internal scratch (no device allocation)."""
    h = _dev_u64(hk, "hk")
    _dev_u64(sorted_out, "sorted_out")
    _dev_u64(start_out, "start_out")
    if sorted_out.numel() < h.numel() or start_out.numel() < num_partitions + 1:
        raise ValueError("output buffers are too small")
    _check(lib().phobic_partition_sort_noalloc(h.data_ptr(), h.numel(), int(num_partitions), sorted_out.data_ptr(),
                                               start_out.data_ptr(), _stream(stream)), "phobic_partition_sort_noalloc")
    return sorted_out, start_out


BUCKET_OPTIMIZED, BUCKET_BETA_STAR, BUCKET_SKEWED, BUCKET_UNIFORM = 0, 1, 2, 3


def phobic_bucket_table(lam: float, alpha: float, P: int, bucket_function: int = 0) -> np.ndarray:
    t = np.zeros(2049, dtype=np.uint64)
    _check(lib().phobic_bucket_table_ex(float(lam), float(alpha), int(P), int(bucket_function), t.ctypes.data),
           "phobic_bucket_table_ex")
    return t


def phobic_status_str(code: int) -> str:
    return lib().phobic_status_str(int(code)).decode()


# the structure's arrays, parsed from phobic_export bytes (used by the parity tests)
HEADER_FIELDS = ["magic", "version", "n", "M", "NP", "B", "P", "lambda_bits", "alpha_bits", "seed", "encoder",
                 "pilot_mode", "off_w", "off_Q", "off_dmin", "ef_l", "n_off_words", "n_col_meta", "n_pil_words",
                 "n_dict_words", "n_ef_low", "n_ef_high", "n_ef_samples", "bits_header", "bits_offsets",
                 "bits_pilots", "bits_remap", "bits_total"]
ARRAYS = ["off_words", "col_meta", "pil_words", "dict_words", "ef_low", "ef_high", "ef_samples"]


def parse_export(data: bytes) -> dict:
    w = np.frombuffer(data, dtype=np.uint64)
    hdr = {k: int(w[i]) for i, k in enumerate(HEADER_FIELDS)}
    hdr["key_kind"] = hdr["pilot_mode"] >> 32
    hdr["pilot_mode"] &= 0xFFFFFFFF
    hdr["bucket_function"] = (hdr["encoder"] >> 32) & 0xFF
    hdr["compact_columns"] = hdr["encoder"] >> 40
    hdr["encoder"] &= 0xFFFFFFFF
    hdr["off_dmin"] = int(np.uint64(hdr["off_dmin"]).astype(np.int64))
    at = len(HEADER_FIELDS)
    for name in ARRAYS:
        c = hdr["n_" + name]
        hdr[name] = w[at: at + c].copy()
        at += c
    if hdr["encoder"] in (ENC_IC_R, ENC_IC_EF, ENC_IC_CR, ENC_MONO_R, ENC_MONO_EF):
        # the dictionary array holds the u32 select samples (of the Rice columns),
        # then the unary bits; a mono encoder has one column of B N_P values
        mono = hdr["encoder"] >= ENC_MONO_C
        ns = ((hdr["B"] * hdr["NP"] if mono else hdr["NP"]) + 63) // 64
        cols = 1 if mono else hdr["B"] - (hdr["compact_columns"] if hdr["encoder"] == ENC_IC_CR else 0)
        sw = (cols * ns + 1) // 2
        d = hdr["dict_words"]
        hdr["rice_samples"] = d[:sw].view(np.uint32)[: cols * ns].copy()
        hdr["rice_high"] = d[sw:].copy()
    return hdr
