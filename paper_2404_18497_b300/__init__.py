"""PHOBIC on B300: partitioned pilot-search MPHF construction and query.

The compute path is libphobic.so (hand-written CUDA for sm_103a, C ABI in
include/phobic.h); ``phobic`` is its Python binding.  Build the library with
``python -m paper_2404_18497_b300.build``.
"""
__all__ = ["phobic", "workloads"]
