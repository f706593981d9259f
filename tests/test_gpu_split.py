"""Karatsuba in the digit dimension (HMV_FLAG_DIGIT_SPLIT1/2): bit-exact
parity with the oracle, and with the unsplit product at full size."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import uniform_vec, workload

from test_gpu_parity import assert_same, oracle_matvec, sampled_parity

pytestmark = pytest.mark.gpu

SPLITS = [hmv.FLAG_DIGIT_SPLIT1, hmv.FLAG_DIGIT_SPLIT2]


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def run(n, b, h, x, flags, kind=hmv.HANKEL, nrhs=1):
    with hmv.Plan(n, b, kind=kind, flags=flags, nrhs=nrhs) as p:
        p.load_matrix(h)
        return p.matvec(x), p.stats()


@pytest.mark.parametrize("flags", SPLITS)
@pytest.mark.parametrize("n,b", [(64, 2048), (100, 700), (1, 64), (7, 33), (30, 1), (140, 4100)])
def test_split_all_rows(flags, n, b):
    h = uniform_vec(60 + n, 0, 2 * n - 1, b, 1)
    x = uniform_vec(60 + n, 1, n, b, -1)
    y, st = run(n, b, h, x, flags)
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("flags", SPLITS)
@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
def test_split_toeplitz_circulant(flags, kind):
    n, b = 90, 600
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = uniform_vec(71, 0, hlen, b)
    x = uniform_vec(71, 1, n, b)
    y, _ = run(n, b, h, x, flags, kind=kind)
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    assert_same(y, oracle_matvec(ok, n, h, x))


def test_split_worst_case_digits():
    n, b = 70, 2046
    m = int("80" * ((b + 7) // 8), 16) & ((1 << b) - 1)
    from paper_1402_5287_gb300.inputs import FixedVec
    h = FixedVec.from_ints([-m] * (2 * n - 1), b, 0)
    x = FixedVec.from_ints([-m] * n, b, 0)
    want = oracle_matvec(oracle.HANKEL, n, h, x)
    for f in SPLITS:
        assert_same(run(n, b, h, x, f)[0], want)


def test_split_large_workload_matches_unsplit():
    n, b, h, x = workload("large")
    y0, _ = run(n, b, h, x, 0)
    for f in SPLITS:
        y, st = run(n, b, h, x, f)
        assert_same(y, y0)
    sampled_parity(oracle.HANKEL, n, h, x, y, 4, 9)
