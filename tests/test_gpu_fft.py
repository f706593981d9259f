"""Split-FP64 FFT path: exact whenever its proven error bound is below 1/2,
and an exact integer-path result (counted as a fallback) otherwise."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import uniform_vec, workload

from test_gpu_parity import assert_same, oracle_matvec, sampled_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def run_fft(n, b, h, x, kind=hmv.HANKEL, w=0):
    with hmv.Plan(n, b, kind=kind, method=hmv.FFT64, piece_bits=w) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        return y, p.stats()


def test_fft_small_workload_all_rows():
    n, b, h, x = workload("small")
    y, st = run_fft(n, b, h, x)
    assert st["fft_matvecs"] == 1 and st["fft_fallbacks"] == 0
    assert st["fft_bound"] < 0.5 and st["fft_max_dist"] <= st["fft_bound"]
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("w", [4, 7, 8, 12, 16])
def test_fft_forced_piece_widths(w):
    n, b = 100, 1000
    h = uniform_vec(70 + w, 0, 2 * n - 1, b, 0)
    x = uniform_vec(70 + w, 1, n, b, 1)
    y, st = run_fft(n, b, h, x, w=w)
    assert st["fft_piece_bits"] == w and st["fft_matvecs"] == 1
    assert st["fft_max_dist"] <= st["fft_bound"] < 0.5
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
def test_fft_toeplitz_and_circulant(kind):
    n, b = 90, 600
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = uniform_vec(81, 0, hlen, b)
    x = uniform_vec(81, 1, n, b)
    y, st = run_fft(n, b, h, x, kind=kind)
    assert st["fft_matvecs"] == 1
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    assert_same(y, oracle_matvec(ok, n, h, x))


def test_fft_hilbert_auto_width_and_16_bit_fallback():
    n, b, h, x = workload("hilbert")
    with hmv.Plan(n, b) as p:
        p.load_matrix(h)
        want = p.matvec(x)
    y, st = run_fft(n, b, h, x)
    assert st["fft_fallbacks"] == 0 and st["fft_bound"] < 0.5 and st["fft_max_dist"] <= st["fft_bound"]
    assert_same(y, want)
    y16, st16 = run_fft(n, b, h, x, w=16)
    assert st16["fft_fallbacks"] == 1 and st16["fft_bound"] >= 0.5
    assert_same(y16, want)
    sampled_parity(oracle.HANKEL, n, h, x, y, 6, 5)


def test_fft_large_workload_auto_width_and_16_bit_fallback():
    n, b, h, x = workload("large")
    y, st = run_fft(n, b, h, x)
    assert st["fft_piece_bits"] == 10 and st["fft_log2_len"] == 27
    assert st["fft_fallbacks"] == 0 and st["fft_max_dist"] <= st["fft_bound"] < 0.5
    sampled_parity(oracle.HANKEL, n, h, x, y, 6, 6)
    y16, st16 = run_fft(n, b, h, x, w=16)
    assert st16["fft_fallbacks"] == 1
    assert_same(y16, y)
