"""The C-ABI library loads and exports every entry point its header declares.
Runs without a GPU: only host-side functions are called."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "phobic.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2404_18497_b300 import build

    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phobic_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["phobic_build", "phobic_query", "phobic_bits_per_key", "phobic_free", "phobic_export",
                     "phobic_import"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath], text=True)
    exported = set(re.findall(r"\sT\s(phobic_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2404_18497_b300 import phobic

    assert sorted(phobic.exported_names()) == declared_functions()
    L = phobic.lib()
    for n in declared_functions():
        assert getattr(L, n) is not None


def test_status_strings_and_params(libpath):
    from paper_2404_18497_b300 import phobic

    for code in range(9):
        assert phobic.phobic_status_str(code)
    p = phobic.make_params()
    assert p.lambda_ == 7.0 and p.alpha == 1.0 and p.partition_size == 2500 and p.s_max == 0


def test_struct_layouts_match_header(libpath):
    """sizes of the header's structs as the C compiler lays them out"""
    from paper_2404_18497_b300 import phobic

    code = r'''
    #include <stdio.h>
    #include "phobic.h"
    int main(void) {
        printf("%zu %zu %zu %zu %zu %zu\n", sizeof(phobic_params), sizeof(phobic_info), sizeof(phobic_tune_info),
               sizeof(phobic_server_config), sizeof(phobic_completion), sizeof(phobic_server_stats));
        return 0;
    }
    '''
    exe = os.path.join(ROOT, "paper_2404_18497_b300", "_build", "layout_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    src = exe + ".c"
    with open(src, "w") as f:
        f.write(code)
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    a, b, c, d, e, f = map(int, subprocess.check_output([exe], text=True).split())
    assert d == ctypes.sizeof(phobic.phobic_server_config)
    assert e == ctypes.sizeof(phobic.phobic_completion) == phobic.COMPLETION_DTYPE.itemsize
    assert f == ctypes.sizeof(phobic.phobic_server_stats)
    assert a == ctypes.sizeof(phobic.phobic_params)
    assert b == ctypes.sizeof(phobic.phobic_info)
    assert c == ctypes.sizeof(phobic.phobic_tune_info)


@pytest.mark.parametrize("lam,alpha,P", [(7.0, 1.0, 2500), (7.0, 0.99, 2500), (7.5, 0.99, 2500), (3.0, 1.0, 16),
                                         (9.0, 0.9, 4096), (1.0, 0.5, 1)])
def test_bucket_table_equals_oracle(libpath, orc, lam, alpha, P):
    """The library's host-side table generator (written separately) reproduces the
    oracle's table bit for bit."""
    from paper_2404_18497_b300 import phobic

    assert (phobic.phobic_bucket_table(lam, alpha, P) == orc.bucket_table(lam, alpha, P)).all()
    for fn in (1, 2, 3):  # the ablation bucket functions
        assert (phobic.phobic_bucket_table(lam, alpha, P, fn) == orc.bucket_table(lam, alpha, P, fn)).all(), fn


def test_invalid_arguments_without_gpu(libpath):
    from paper_2404_18497_b300 import phobic

    L = phobic.lib()
    h = ctypes.c_void_p()
    p = phobic.make_params()
    assert L.phobic_build_ex(None, 10, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert L.phobic_build(None, 0, 7.0, 1.0, 2500, 0, None, ctypes.byref(h)) == 1
    assert np.isnan(L.phobic_bits_per_key(None))
    assert L.phobic_query(None, None, None, 0, None) == 1
    assert L.phobic_import(b"nonsense", 8, None, ctypes.byref(h)) == 8
    L.phobic_free(None)
    # the tuner validates before it touches a device
    ps = (ctypes.c_uint32 * 2)()
    out = phobic.phobic_params()
    off = (ctypes.c_uint64 * 3)(0, 5, 5)  # an empty set
    assert L.phobic_tune_batch(off, 2, ctypes.byref(p), None, ps, ctypes.byref(out), None) == 1
    assert L.phobic_tune_batch(None, 2, ctypes.byref(p), None, ps, ctypes.byref(out), None) == 1
    big = phobic.make_params(5000.0, 1.0, 8192)  # every candidate partition size is below lambda
    off2 = (ctypes.c_uint64 * 2)(0, 100)
    assert L.phobic_tune_batch(off2, 1, ctypes.byref(big), None, ps, ctypes.byref(out), None) == 1
    # parameters are checked before the key pointer is used (a stand-in address here)
    small = phobic.make_params(9.0, 1.0, 8)  # P below lambda
    assert L.phobic_build_ex(ctypes.c_void_p(256), 100, ctypes.byref(small), None, ctypes.byref(h)) == 1
    # coalesced query and server entry points reject NULL arguments
    assert L.phobic_query_multi(None, None, None, None, 3, None) == 1
    assert L.phobic_query_multi(None, None, None, None, 0, None) == 0
    rid = ctypes.c_uint64()
    assert L.phobic_server_submit_build(None, None, 0, ctypes.byref(p), None, ctypes.byref(rid)) == 1
    assert L.phobic_server_submit_query(None, 1, None, None, 0, None, ctypes.byref(rid)) == 1
    assert L.phobic_server_submit_release(None, 1, ctypes.byref(rid)) == 1
    assert L.phobic_server_create(None, None) == 1
    L.phobic_server_destroy(None)


def test_noalloc_sort_rejects_sizes_on_the_host(libpath):
    """phobic_partition_sort_noalloc refuses sizes beyond its fixed array before
    it touches the device: more than PHOBIC_NOALLOC_MAX_KEYS keys, or (at the
    maximum n) a partition count whose digit tables would not fit (2^36
    partitions need four passes of 9-bit digits; the array holds three).  The
    pointers are never dereferenced."""
    from paper_2404_18497_b300 import phobic

    L = phobic.lib()
    fake = ctypes.c_void_p(16)
    mx = phobic.NOALLOC_MAX_KEYS
    assert L.phobic_partition_sort_noalloc(fake, mx + 1, 1, fake, fake, None) == 1
    assert L.phobic_partition_sort_noalloc(fake, mx, 1 << 36, fake, fake, None) == 1
    assert L.phobic_partition_sort_noalloc(fake, 0, 1, fake, fake, None) == 1
