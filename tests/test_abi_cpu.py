"""The C-ABI library builds for sm_103a, loads and exports every entry point
declared in include/hmv.h; descriptor checks answer without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hmv_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return hmv.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"hmv_plan", "hmv_load_matrix", "hmv_matvec", "hmv_free"} <= names
    for name in names:
        assert hasattr(lib, name), name
    assert set(hmv.EXPORTS) <= names


def test_status_strings_and_version(lib):
    assert lib.hmv_status_string(0) == b"ok"
    assert lib.hmv_status_string(1) == b"invalid argument"
    assert lib.hmv_status_string(7) == b"unsupported configuration"
    assert lib.hmv_status_string(8) == b"internal consistency check failed"
    assert lib.hmv_status_string(99) == b"unknown status"
    assert lib.hmv_version() >= 100


def test_status_codes_match_the_header():
    """Every hmv_status value in include/hmv.h has its name in the binding's table."""
    text = open(os.path.join(ROOT, "include", "hmv.h")).read()
    body = re.search(r"typedef enum \{(.*?)\} hmv_status;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    codes = {int(v): k for k, v in re.findall(r"(HMV_\w+)\s*=\s*(\d+)", body)}
    assert codes == hmv.STATUS


@pytest.mark.parametrize("field,value", [("n", 0), ("b", 0), ("b", (1 << 20) + 1), ("nrhs", 0), ("kind", 3),
                                         ("method", 9), ("levels", -2), ("levels", 17), ("flags", 1 << 9),
                                         ("flags", hmv.FLAG_TILE128 | hmv.FLAG_TILE256),
                                         ("piece_bits", 5), ("piece_bits", -1)])
def test_plan_rejects_bad_descriptors_without_gpu(lib, field, value):
    d = hmv.Desc(16, 64, 1, 0, 0, -1, 0, 0)
    setattr(d, field, value)
    out = ctypes.c_void_p()
    assert lib.hmv_plan(ctypes.byref(d), None, ctypes.byref(out)) == 1
    assert out.value is None


@pytest.mark.parametrize("b,flags,method", [(4096, hmv.FLAG_DIGIT_TOOM4 | hmv.FLAG_DIGIT_SPLIT1, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM4 | hmv.FLAG_DIGIT_SPLIT2, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM4 | hmv.FLAG_DIGIT_TOOM6, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM6 | hmv.FLAG_DIGIT_SPLIT1, 0),
                                           (96, hmv.FLAG_DIGIT_TOOM4, 0), (160, hmv.FLAG_DIGIT_TOOM6, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM4 | hmv.FLAG_SIMT_LEAF, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM6 | hmv.FLAG_SIMT_LEAF, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM4, 3), (4096, hmv.FLAG_DIGIT_TOOM4, 1),
                                           (4096, hmv.FLAG_DIGIT_TOOM6, 3), (224, hmv.FLAG_DIGIT_TOOM8, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM8 | hmv.FLAG_DIGIT_TOOM6, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM8 | hmv.FLAG_SIMT_LEAF, 0),
                                           (4096, hmv.FLAG_DIGIT_TOOM8, 3)])
def test_toom_rejects_bad_combinations_without_gpu(lib, b, flags, method):
    """Toom-K needs K parts of at least one limb, the integer tensor-core path
    and no second digit split."""
    d = hmv.Desc(16, b, 1, 0, method, -1, flags, 0)
    out = ctypes.c_void_p()
    assert lib.hmv_plan(ctypes.byref(d), None, ctypes.byref(out)) == 1
    assert out.value is None


def test_fft_piece_bits_range_without_gpu(lib):
    out = ctypes.c_void_p()
    for w in (3, 21, -1):
        d = hmv.Desc(16, 64, 1, 0, 3, -1, 0, w)
        assert lib.hmv_plan(ctypes.byref(d), None, ctypes.byref(out)) == 1


def test_null_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.hmv_plan(None, None, ctypes.byref(out)) == 1
    assert lib.hmv_load_matrix(None, None) == 1
    assert lib.hmv_matvec(None, None, None) == 1
    lib.hmv_free(None)  # NULL is ignored


def test_struct_layouts_match_header():
    assert ctypes.sizeof(hmv.Desc) == 32
    assert ctypes.sizeof(hmv.Vec) == 40
    assert hmv.Vec.limbs.offset == 16 and hmv.Vec.neg.offset == 24 and hmv.Vec.on_device.offset == 32
    assert ctypes.sizeof(hmv.Stats) == 4 * 4 + 8 + 8 * 2 + 8 + 8 * 5 + 8 * 3 + 4 * 2 + 8 * 5 + 4 * 2


def test_toom8_depth_bound_without_gpu(lib):
    """Toom-8's int64 interpolation sums are bounded for index depths up to 7:
    the plan refuses the split where its products need depth 8 (n = 20000),
    and HMV_AUTO then picks another split."""
    assert hmv.plan_bytes(8000, 33220, flags=hmv.FLAG_DIGIT_TOOM8) > 0
    with pytest.raises(hmv.HmvError):
        hmv.plan_bytes(20000, 33220, flags=hmv.FLAG_DIGIT_TOOM8)
    assert hmv.plan_bytes(20000, 33220) > 0


def test_leaf_stall_hook_checks_its_arguments(lib):
    """The failure-path test hook validates its arguments on the host (no GPU
    work is queued by it)."""
    assert lib.hmv_test_leaf_stall(-1, 20_000_000) == 1
    assert lib.hmv_test_leaf_stall(1, 10) == 1            # below the 1 ms floor
    assert lib.hmv_test_leaf_stall(1, 3_000_000_000) == 1  # above the 2 s default
    assert lib.hmv_test_leaf_stall(0, 20_000_000) == 0     # disarmed


def test_server_plan_choice_falls_back_beyond_the_ntt_size():
    """A server on the NTT path gives a request the NTT plan where the
    convolution fits 2^26 points, the tensor-core plan otherwise; footprints
    from hmv_plan_bytes (no allocation)."""
    from paper_1402_5287_gb300.serving import plan_choice
    m, size = plan_choice(8000, 33220, hmv.HANKEL, hmv.NTT)
    assert m == hmv.NTT and size == hmv.plan_bytes(8000, 33220, method=hmv.NTT)
    m, size = plan_choice(9000, 33220, hmv.HANKEL, hmv.NTT)  # (2n-1)(2P-1) > 2^26
    assert m == hmv.AUTO and size == hmv.plan_bytes(9000, 33220)
    assert plan_choice(4096, 8192, hmv.TOEPLITZ, hmv.AUTO) == (hmv.AUTO, hmv.plan_bytes(4096, 8192, kind=hmv.TOEPLITZ))
