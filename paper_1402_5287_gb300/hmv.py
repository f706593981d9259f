"""ctypes binding of libhmv (include/hmv.h): argument marshalling only.

Every step of the product runs in the CUDA library; there is no CPU path.
Loading fails loudly if libhmv.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .inputs import FixedVec

HANKEL, TOEPLITZ, CIRCULANT = 0, 1, 2
AUTO, SCHOOLBOOK, KARATSUBA, FFT64, NTT = 0, 1, 2, 3, 4
FLAG_TIMING, FLAG_SIMT_LEAF, FLAG_DIGIT_SPLIT1, FLAG_DIGIT_SPLIT2, FLAG_TILE128 = 1, 2, 4, 8, 16
FLAG_DIGIT_TOOM4, FLAG_DIGIT_TOOM6, FLAG_DIGIT_TOOM8 = 32, 64, 256
FLAG_TILE256 = 128
STATUS = {0: "HMV_OK", 1: "HMV_EINVAL", 2: "HMV_ENOMEM", 3: "HMV_ECUDA", 4: "HMV_ETIMEOUT",
          5: "HMV_ENOTLOADED", 6: "HMV_EFFTBOUND", 7: "HMV_EUNSUPPORTED", 8: "HMV_EINTERNAL"}
EUNSUPPORTED = 7

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhmv.so")
EXPORTS = ["hmv_plan", "hmv_load_matrix", "hmv_matvec", "hmv_free", "hmv_get_stats", "hmv_reset_stats",
           "hmv_status_string", "hmv_version", "hmv_schoolbook_noalloc", "hmv_batch_create",
           "hmv_batch_load_matrix", "hmv_batch_matvec", "hmv_batch_get_info", "hmv_batch_free",
           "hmv_plan_bytes", "hmv_matvec_many"]
NOALLOC_SCRATCH_BYTES = 4 << 20


class HmvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("b", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("method", ctypes.c_int32), ("levels", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("piece_bits", ctypes.c_int32)]


class Vec(ctypes.Structure):
    _fields_ = [("len", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("b", ctypes.c_int32),
                ("exponent", ctypes.c_int32), ("limbs", ctypes.c_void_p), ("neg", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("leaves", ctypes.c_int32), ("leaf_rows_max", ctypes.c_int32),
                ("digits", ctypes.c_int32), ("leaf_tiles", ctypes.c_int64), ("leaf_macs", ctypes.c_double),
                ("leaf_macs_issued", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("ms_prepass", ctypes.c_double), ("ms_leaf", ctypes.c_double), ("ms_post", ctypes.c_double),
                ("ms_round", ctypes.c_double), ("ms_total", ctypes.c_double), ("launches_leaf", ctypes.c_int64),
                ("launches_total", ctypes.c_int64), ("matvecs", ctypes.c_int64),
                ("fft_piece_bits", ctypes.c_int32), ("fft_log2_len", ctypes.c_int32), ("fft_bound", ctypes.c_double),
                ("fft_max_dist", ctypes.c_double), ("fft_matvecs", ctypes.c_int64),
                ("fft_fallbacks", ctypes.c_int64), ("ms_fft", ctypes.c_double),
                ("leaf_tile_digits", ctypes.c_int32), ("digit_products", ctypes.c_int32)]


class Scalar(ctypes.Structure):
    _fields_ = [("limbs", ctypes.POINTER(ctypes.c_uint32)), ("nlimbs", ctypes.c_int32), ("neg", ctypes.c_int32),
                ("exponent", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("matrices", ctypes.c_int32), ("pairs", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("leaf_tiles", ctypes.c_int64), ("leaf_macs", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("kernels_per_graph", ctypes.c_int64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """The CUDA library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libhmv.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.hmv_plan.argtypes = [ctypes.POINTER(Desc), vp, ctypes.POINTER(vp)]
        lib.hmv_plan.restype = ctypes.c_int
        lib.hmv_load_matrix.argtypes = [vp, ctypes.POINTER(Vec)]
        lib.hmv_load_matrix.restype = ctypes.c_int
        lib.hmv_matvec.argtypes = [vp, ctypes.POINTER(Vec), ctypes.POINTER(Vec)]
        lib.hmv_matvec.restype = ctypes.c_int
        lib.hmv_free.argtypes = [vp]
        lib.hmv_free.restype = None
        lib.hmv_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        lib.hmv_get_stats.restype = ctypes.c_int
        lib.hmv_reset_stats.argtypes = [vp]
        lib.hmv_reset_stats.restype = ctypes.c_int
        lib.hmv_status_string.argtypes = [ctypes.c_int]
        lib.hmv_status_string.restype = ctypes.c_char_p
        lib.hmv_version.argtypes = []
        lib.hmv_version.restype = ctypes.c_int32
        i32 = ctypes.c_int32
        lib.hmv_schoolbook_noalloc.argtypes = [i32, i32, i32, vp, vp, i32, vp, vp, i32, vp, vp,
                                               ctypes.POINTER(i32), vp]
        lib.hmv_schoolbook_noalloc.restype = ctypes.c_int
        lib.hmv_batch_create.argtypes = [i32, ctypes.POINTER(Desc), vp, ctypes.c_uint64, ctypes.POINTER(vp)]
        lib.hmv_batch_create.restype = ctypes.c_int
        lib.hmv_batch_load_matrix.argtypes = [vp, i32, ctypes.POINTER(Vec)]
        lib.hmv_batch_load_matrix.restype = ctypes.c_int
        lib.hmv_batch_matvec.argtypes = [vp, ctypes.POINTER(Vec), ctypes.POINTER(Vec)]
        lib.hmv_batch_matvec.restype = ctypes.c_int
        lib.hmv_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
        lib.hmv_batch_get_info.restype = ctypes.c_int
        lib.hmv_batch_free.argtypes = [vp]
        lib.hmv_batch_free.restype = None
        lib.hmv_plan_bytes.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_uint64)]
        lib.hmv_plan_bytes.restype = ctypes.c_int
        lib.hmv_measure_montgomery_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.hmv_measure_montgomery_rate.restype = ctypes.c_int
        lib.hmv_trim_memory.argtypes = []
        lib.hmv_trim_memory.restype = ctypes.c_int
        lib.hmv_test_leaf_stall.argtypes = [i32, ctypes.c_int64]
        lib.hmv_test_leaf_stall.restype = ctypes.c_int
        lib.hmv_matvec_many.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(Vec), ctypes.POINTER(Vec)]
        lib.hmv_matvec_many.restype = ctypes.c_int
        lib.hmv_dot.argtypes = [vp, ctypes.POINTER(Vec), ctypes.POINTER(Vec), ctypes.POINTER(ctypes.c_uint32), i32,
                                ctypes.POINTER(ctypes.c_uint8)]
        lib.hmv_dot.restype = ctypes.c_int
        lib.hmv_lincomb.argtypes = [vp, i32, ctypes.POINTER(Scalar), ctypes.POINTER(Vec), ctypes.POINTER(Vec)]
        lib.hmv_lincomb.restype = ctypes.c_int
        _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise HmvError(st, where)


def _host_vec(v: FixedVec, nrhs: int = 1) -> tuple[Vec, tuple]:
    limbs = np.ascontiguousarray(v.limbs, dtype=np.uint32)
    neg = np.ascontiguousarray(v.neg, dtype=np.uint8)
    vec = Vec(v.count // nrhs, nrhs, v.b, v.exponent, limbs.ctypes.data, neg.ctypes.data, 0, 0)
    return vec, (limbs, neg)


def schoolbook_noalloc(n: int, b: int, kind: int, h_ptrs: tuple[int, int], h_exponent: int,
                      x_ptrs: tuple[int, int], x_exponent: int, y_ptrs: tuple[int, int], stream=None) -> int:
    """hmv_schoolbook_noalloc on device pointers (limbs, neg); returns E_y.

    For callers that cannot allocate device memory: the call uses only the
    given buffers and the library's fixed scratch array.
    """
    lib = load_library()
    e = ctypes.c_int32(0)
    s = ctypes.c_void_p(0 if stream is None else int(stream))
    _check(lib.hmv_schoolbook_noalloc(n, b, kind, h_ptrs[0], h_ptrs[1], h_exponent, x_ptrs[0], x_ptrs[1],
                                      x_exponent, y_ptrs[0], y_ptrs[1], ctypes.byref(e), s),
           "hmv_schoolbook_noalloc")
    return int(e.value)


def measure_montgomery_rate(stream=None) -> float:
    """Montgomery products per second this GPU sustains (the NTT path's roofline)."""
    r = ctypes.c_double(0)
    _check(load_library().hmv_measure_montgomery_rate(ctypes.c_void_p(0 if stream is None else int(stream)),
                                                      ctypes.byref(r)), "hmv_measure_montgomery_rate")
    return r.value


def trim_memory() -> None:
    """hmv_trim_memory: hand the library's unused pooled device memory back."""
    _check(load_library().hmv_trim_memory(), "hmv_trim_memory")


def arm_leaf_stall(launches: int, wait_ns: int = 20_000_000) -> None:
    """hmv_test_leaf_stall: the next `launches` direct leaf launches hold back
    one accumulator release and limit every wait to wait_ns (tests of the
    failure path only; 0 disarms)."""
    _check(load_library().hmv_test_leaf_stall(launches, wait_ns), "hmv_test_leaf_stall")


def plan_bytes(n: int, b: int, kind: int = HANKEL, method: int = AUTO, levels: int = -1, nrhs: int = 1,
               flags: int = 0, piece_bits: int = 0) -> int:
    """Device bytes hmv_plan would allocate (no allocation, no GPU needed)."""
    lib = load_library()
    d = Desc(n, b, nrhs, kind, method, levels, flags, piece_bits)
    out = ctypes.c_uint64(0)
    _check(lib.hmv_plan_bytes(ctypes.byref(d), ctypes.byref(out)), "hmv_plan_bytes")
    return int(out.value)


def matvec_many_device(plans, xs_ptrs, ys_ptrs, x_exponents) -> list[int]:
    """hmv_matvec_many on device pointers: one product per plan in one step."""
    lib = load_library()
    n = len(plans)
    pa = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    xa = (Vec * n)()
    ya = (Vec * n)()
    for i, p in enumerate(plans):
        xa[i] = Vec(p.n, 1, p.b, x_exponents[i], xs_ptrs[i][0], xs_ptrs[i][1], 1, 0)
        ya[i] = Vec(p.n, 1, p.b, 0, ys_ptrs[i][0], ys_ptrs[i][1], 1, 0)
    _check(lib.hmv_matvec_many(n, pa, xa, ya), "hmv_matvec_many")
    return [int(ya[i].exponent) for i in range(n)]


def _device_vec(plan, ptrs, exponent=0):
    """Vec for a device vector (limbs pointer, sign pointer) of the plan's n and b."""
    return Vec(plan.n, 1, plan.b, exponent, ptrs[0], ptrs[1], 1, 0)


def dot_device(plan, x_ptrs, y_ptrs) -> int:
    """hmv_dot: the exact integer sum_i X_i Y_i of two device vectors' signed
    mantissas (its value is that integer times 2^(E_x + E_y - 2b))."""
    lib = load_library()
    zl = 2 * plan.L32 + 2
    z = (ctypes.c_uint32 * zl)()
    zn = ctypes.c_uint8()
    xv, yv = _device_vec(plan, x_ptrs), _device_vec(plan, y_ptrs)
    _check(lib.hmv_dot(plan.handle, ctypes.byref(xv), ctypes.byref(yv), z, zl, ctypes.byref(zn)), "hmv_dot")
    m = int.from_bytes(bytes(z), "little")
    return -m if zn.value else m


def lincomb_device(plan, terms, y_ptrs) -> int:
    """hmv_lincomb: y = RNE_b(sum c * x) over terms [(c_int, c_exponent,
    (limbs_ptr, neg_ptr), x_exponent)]; returns y's exponent."""
    lib = load_library()
    k = len(terms)
    cs = (Scalar * k)()
    xs = (Vec * k)()
    keep = []
    for i, (c, ce, xp, xe) in enumerate(terms):
        mag = abs(int(c))
        nl = max(1, (mag.bit_length() + 31) // 32)
        arr = (ctypes.c_uint32 * nl).from_buffer_copy(mag.to_bytes(4 * nl, "little"))
        keep.append(arr)
        cs[i] = Scalar(ctypes.cast(arr, ctypes.POINTER(ctypes.c_uint32)), nl, 1 if c < 0 else 0, ce)
        xs[i] = _device_vec(plan, xp, xe)
    yv = _device_vec(plan, y_ptrs)
    _check(lib.hmv_lincomb(plan.handle, k, cs, xs, ctypes.byref(yv)), "hmv_lincomb")
    return int(yv.exponent)


class Plan:
    """One plan = one matrix order, precision, kind, method and stream."""

    def __init__(self, n: int, b: int, kind: int = HANKEL, method: int = AUTO, levels: int = -1, nrhs: int = 1,
                 flags: int = 0, stream=None, piece_bits: int = 0):
        self.lib = load_library()
        self.n, self.b, self.kind, self.nrhs = n, b, kind, nrhs
        self.L32 = (b + 31) // 32
        d = Desc(n, b, nrhs, kind, method, levels, flags, piece_bits)
        handle = ctypes.c_void_p()
        s = ctypes.c_void_p(0 if stream is None else int(stream))
        _check(self.lib.hmv_plan(ctypes.byref(d), s, ctypes.byref(handle)), "hmv_plan")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.hmv_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- host
    def load_matrix(self, h: FixedVec):
        vec, keep = _host_vec(h)
        _check(self.lib.hmv_load_matrix(self.handle, ctypes.byref(vec)), "hmv_load_matrix")
        del keep

    def matvec(self, x: FixedVec) -> FixedVec:
        """Host in, host out (copies to and from the device inside the call)."""
        xv, keep = _host_vec(x, self.nrhs)
        rows = self.n * self.nrhs
        y_limbs = np.zeros((rows, self.L32), dtype=np.uint32)
        y_neg = np.zeros(rows, dtype=np.uint8)
        yv = Vec(self.n, self.nrhs, self.b, 0, y_limbs.ctypes.data, y_neg.ctypes.data, 0, 0)
        _check(self.lib.hmv_matvec(self.handle, ctypes.byref(xv), ctypes.byref(yv)), "hmv_matvec")
        del keep
        return FixedVec(y_limbs, y_neg, self.b, int(yv.exponent))

    # ---------------------------------------------------------------- device
    def load_matrix_device(self, limbs_ptr: int, neg_ptr: int, length: int, exponent: int):
        vec = Vec(length, 1, self.b, exponent, limbs_ptr, neg_ptr, 1, 0)
        _check(self.lib.hmv_load_matrix(self.handle, ctypes.byref(vec)), "hmv_load_matrix")

    def matvec_device(self, x_limbs_ptr: int, x_neg_ptr: int, x_exponent: int, y_limbs_ptr: int,
                      y_neg_ptr: int) -> int:
        """Device pointers in and out (ordered on the plan's stream); returns E_y."""
        xv = Vec(self.n, self.nrhs, self.b, x_exponent, x_limbs_ptr, x_neg_ptr, 1, 0)
        yv = Vec(self.n, self.nrhs, self.b, 0, y_limbs_ptr, y_neg_ptr, 1, 0)
        _check(self.lib.hmv_matvec(self.handle, ctypes.byref(xv), ctypes.byref(yv)), "hmv_matvec")
        return int(yv.exponent)

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib.hmv_get_stats(self.handle, ctypes.byref(s)), "hmv_get_stats")
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def reset_stats(self):
        _check(self.lib.hmv_reset_stats(self.handle), "hmv_reset_stats")


class Batch:
    """Many matrices (each with a block of right-hand sides) advanced by one
    CUDA graph launch per call (hmv_batch_*)."""

    def __init__(self, problems, stream=None, wave_bytes: int = 32 << 30):
        """problems: list of dicts with n, b and optionally kind, nrhs, levels,
        flags and method (AUTO, KARATSUBA or NTT)."""
        self.lib = load_library()
        self.problems = [{"kind": HANKEL, "nrhs": 1, "levels": -1, "flags": 0, "method": AUTO, **pr}
                         for pr in problems]
        arr = (Desc * len(problems))()
        for i, pr in enumerate(self.problems):
            arr[i] = Desc(pr["n"], pr["b"], pr["nrhs"], pr["kind"], pr["method"], pr["levels"], pr["flags"], 0)
        handle = ctypes.c_void_p()
        s = ctypes.c_void_p(0 if stream is None else int(stream))
        _check(self.lib.hmv_batch_create(len(problems), arr, s, wave_bytes, ctypes.byref(handle)), "hmv_batch_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.hmv_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_matrix(self, index: int, h: FixedVec):
        vec, keep = _host_vec(h)
        _check(self.lib.hmv_batch_load_matrix(self.handle, index, ctypes.byref(vec)), "hmv_batch_load_matrix")
        del keep

    def matvec(self, xs):
        """Host blocks in, host blocks out."""
        n = len(self.problems)
        xa = (Vec * n)()
        ya = (Vec * n)()
        keep, outs = [], []
        for i, (pr, x) in enumerate(zip(self.problems, xs)):
            v, k = _host_vec(x, pr["nrhs"])
            xa[i] = v
            keep.append(k)
            rows = pr["n"] * pr["nrhs"]
            yl = np.zeros((rows, (pr["b"] + 31) // 32), dtype=np.uint32)
            yn = np.zeros(rows, dtype=np.uint8)
            outs.append((yl, yn))
            ya[i] = Vec(pr["n"], pr["nrhs"], pr["b"], 0, yl.ctypes.data, yn.ctypes.data, 0, 0)
        _check(self.lib.hmv_batch_matvec(self.handle, xa, ya), "hmv_batch_matvec")
        return [FixedVec(yl, yn, pr["b"], int(ya[i].exponent)) for i, ((yl, yn), pr) in
                enumerate(zip(outs, self.problems))]

    def matvec_device(self, xs_ptrs, ys_ptrs, x_exponents):
        """Device blocks: xs_ptrs/ys_ptrs are lists of (limbs, neg) pointers; returns exponents."""
        n = len(self.problems)
        xa = (Vec * n)()
        ya = (Vec * n)()
        for i, pr in enumerate(self.problems):
            xa[i] = Vec(pr["n"], pr["nrhs"], pr["b"], x_exponents[i], xs_ptrs[i][0], xs_ptrs[i][1], 1, 0)
            ya[i] = Vec(pr["n"], pr["nrhs"], pr["b"], 0, ys_ptrs[i][0], ys_ptrs[i][1], 1, 0)
        _check(self.lib.hmv_batch_matvec(self.handle, xa, ya), "hmv_batch_matvec")
        return [int(ya[i].exponent) for i in range(n)]

    def info(self) -> dict:
        s = BatchInfo()
        _check(self.lib.hmv_batch_get_info(self.handle, ctypes.byref(s)), "hmv_batch_get_info")
        return {name: getattr(s, name) for name, _ in BatchInfo._fields_}
