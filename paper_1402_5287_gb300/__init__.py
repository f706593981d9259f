"""GB300-native exact multiprecision Hankel / Toeplitz / circulant products.

The compute path is libhmv.so (CUDA C++ for sm_103a, C ABI in include/hmv.h);
`hmv` is its ctypes binding and `inputs` the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "hmv", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force, verbose=verbose)
