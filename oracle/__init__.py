"""CPU oracle for the multiprecision Hankel / Toeplitz / circulant product.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The CUDA library never imports, links or
calls anything here, and nothing here comes from the CUDA library.

Contents
  hmv_oracle.c   plain schoolbook big-integer product from the matrix
                 definitions of Sec. 1 (A_H, A_T, A_C) and the schoolbook sum
                 of Sec. 1, exact on 32-bit limbs, threaded over rows; plus
                 the rounding rule (b-bit round-half-even with the least
                 shared exponent; the paper does not state one).
  algorithm1.py  Algorithm 1 of Sec. 3 on Python integers, step by step, with
                 operation counters (pins the recursion's index arithmetic).

Every function here is pinned by tests/test_oracle_pins.py against brute
force, closed forms, the paper's explicit n = 2 formula and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmv_oracle.c")
_LIB = os.path.join(_HERE, "libhmv_oracle.so")
_lock = threading.Lock()
_lib = None

HANKEL, TOEPLITZ, CIRCULANT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C11, no machine-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-D_POSIX_C_SOURCE=200809L",
                               "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i = ctypes.c_int
            lib.oracle_exact_rows.argtypes = [i, i, i, P, P, i, P, P, i, P, i, P, P, i]
            lib.oracle_exact_rows.restype = i
            lib.oracle_round.argtypes = [i, i, P, P, i, i, P, P, P]
            lib.oracle_round.restype = i
            lib.oracle_round_fixed_shift.argtypes = [i, i, P, P, i, ctypes.c_int64, P, P]
            lib.oracle_round_fixed_shift.restype = i
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def zl_for(b: int) -> int:
    """Limbs that hold any exact row: 2*ceil(b/32) + 1 (n < 2^32 terms)."""
    return 2 * ((b + 31) // 32) + 1


def exact_rows(kind: int, n: int, b: int, a, x, rows=None, nthreads: int | None = None):
    """Exact Z_i for the given rows.  a, x: FixedVec-like (limbs, neg).

    Returns (z_mag uint32 [R, zl], z_neg uint8 [R]).
    """
    lib = _load()
    rows = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    zl = zl_for(b)
    z = np.zeros((len(rows), zl), dtype=np.uint32)
    zn = np.zeros(len(rows), dtype=np.uint8)
    al = np.ascontiguousarray(a.limbs, dtype=np.uint32)
    an = np.ascontiguousarray(a.neg, dtype=np.uint8)
    xl = np.ascontiguousarray(x.limbs, dtype=np.uint32)
    xn = np.ascontiguousarray(x.neg, dtype=np.uint8)
    st = lib.oracle_exact_rows(kind, n, b, _ptr(al), _ptr(an), al.shape[0], _ptr(xl), _ptr(xn),
                               len(rows), _ptr(rows), zl, _ptr(z), _ptr(zn),
                               nthreads or default_threads())
    if st != 0:
        raise RuntimeError(f"oracle_exact_rows failed with status {st}")
    return z, zn


def round_rows(z: np.ndarray, zn: np.ndarray, b: int, e_in: int):
    """b-bit RNE with the least shared exponent.  Returns (limbs, neg, E_y)."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.uint32)
    zn = np.ascontiguousarray(zn, dtype=np.uint8)
    L = (b + 31) // 32
    y = np.zeros((z.shape[0], L), dtype=np.uint32)
    yn = np.zeros(z.shape[0], dtype=np.uint8)
    e = np.zeros(1, dtype=np.int32)
    st = lib.oracle_round(z.shape[0], z.shape[1], _ptr(z), _ptr(zn), b, e_in, _ptr(y), _ptr(yn), _ptr(e))
    if st != 0:
        raise RuntimeError(f"oracle_round failed with status {st}")
    return y, yn, int(e[0])


def round_rows_fixed(z: np.ndarray, zn: np.ndarray, b: int, shift: int):
    """RNE(|Z| / 2^shift) to b bits for a shift chosen elsewhere."""
    lib = _load()
    z = np.ascontiguousarray(z, dtype=np.uint32)
    zn = np.ascontiguousarray(zn, dtype=np.uint8)
    L = (b + 31) // 32
    y = np.zeros((z.shape[0], L), dtype=np.uint32)
    yn = np.zeros(z.shape[0], dtype=np.uint8)
    st = lib.oracle_round_fixed_shift(z.shape[0], z.shape[1], _ptr(z), _ptr(zn), b, shift, _ptr(y), _ptr(yn))
    if st != 0:
        raise RuntimeError(f"oracle_round_fixed_shift failed with status {st}")
    return y, yn


def matvec(kind: int, n: int, a, x, nthreads: int | None = None):
    """Rounded product: returns (limbs, neg, E_y) for all n rows."""
    z, zn = exact_rows(kind, n, a.b, a, x, None, nthreads)
    return round_rows(z, zn, a.b, a.exponent + x.exponent)


def z_to_ints(z: np.ndarray, zn: np.ndarray) -> list[int]:
    out = []
    for r in range(z.shape[0]):
        m = int.from_bytes(np.ascontiguousarray(z[r], dtype="<u4").tobytes(), "little")
        out.append(-m if zn[r] else m)
    return out


def limbs_to_ints(y: np.ndarray, yn: np.ndarray) -> list[int]:
    return z_to_ints(y, yn)
