"""PHOBIC CPU oracle -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library never does, and the oracle
never imports the library.  See ``phobic_oracle.c`` for what each function
computes and which passage of the paper it follows.
"""
from .oracle import (  # noqa: F401
    Oracle,
    OracleError,
    build_oracle_lib,
    lib,
    params,
)
