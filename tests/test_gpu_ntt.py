"""The exact NTT path (HMV_NTT) against the CPU oracle, through the C ABI:
16-bit pieces, one cyclic convolution modulo two primes, Chinese remainder,
carries; every result bit for bit."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec, workload
from test_gpu_parity import THREADS, assert_same, oracle_matvec, sampled_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def ntt(n, b, h, x, kind=hmv.HANKEL, nrhs=1):
    with hmv.Plan(n, b, kind=kind, method=hmv.NTT, nrhs=nrhs) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        st = p.stats()
    assert st["fft_piece_bits"] == 16
    return y


@pytest.mark.parametrize("n,b", [(1, 1), (2, 17), (3, 32), (17, 33), (64, 2048), (130, 1000), (257, 700),
                                 (300, 4096), (45, 33220)])
def test_ntt_all_rows(n, b):
    h = uniform_vec(9100 + n, 0, 2 * n - 1, b, 1)
    x = uniform_vec(9100 + n, 1, n, b, -1)
    assert_same(ntt(n, b, h, x), oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
def test_ntt_toeplitz_and_circulant(kind):
    n, b = 90, 600
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = uniform_vec(9200, 0, hlen, b)
    x = uniform_vec(9200, 1, n, b)
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    assert_same(ntt(n, b, h, x, kind=kind), oracle_matvec(ok, n, h, x))


def test_ntt_extreme_digits_and_signs():
    """All-ones mantissas with mixed signs make every convolution coefficient
    as large as it can be (the bound that two primes must cover), and a
    single non-zero entry an exact selection."""
    n, b = 200, 2048
    mm = (1 << b) - 1
    h = FixedVec.from_ints([mm if k % 3 else -mm for k in range(2 * n - 1)], b, 0)
    x = FixedVec.from_ints([-mm if j % 2 else mm for j in range(n)], b, 0)
    assert_same(ntt(n, b, h, x), oracle_matvec(oracle.HANKEL, n, h, x))
    h = FixedVec.from_ints([mm] * (2 * n - 1), b, 0)
    x = FixedVec.from_ints([mm] * n, b, 0)
    assert_same(ntt(n, b, h, x), oracle_matvec(oracle.HANKEL, n, h, x))
    hk = FixedVec.from_ints([(1 << (b - 1)) if k == 77 else 0 for k in range(2 * n - 1)], b, 0)
    x = uniform_vec(9300, 1, n, b)
    assert_same(ntt(n, b, hk, x), oracle_matvec(oracle.HANKEL, n, hk, x))
    z = FixedVec.from_ints([0] * n, b, 2)
    y = ntt(n, b, h, z)
    assert y.exponent == 2 and not y.limbs.any() and not y.neg.any()


def test_ntt_block_rhs_and_plan_reuse():
    n, b, k = 120, 1500, 3
    h = uniform_vec(9400, 0, 2 * n - 1, b)
    parts = [uniform_vec(9400 + r, 1, n, b) for r in range(k)]
    X = FixedVec(np.concatenate([p.limbs for p in parts]), np.concatenate([p.neg for p in parts]), b, 0)
    with hmv.Plan(n, b, method=hmv.NTT, nrhs=k) as p:
        p.load_matrix(h)
        Y = p.matvec(X)
        Y2 = p.matvec(X)
    zs = [oracle.exact_rows(oracle.HANKEL, n, b, h, part, None, THREADS) for part in parts]
    yl, yn, e = oracle.round_rows(np.concatenate([z[0] for z in zs]), np.concatenate([z[1] for z in zs]), b,
                                  h.exponent)
    assert_same(Y, FixedVec(yl, yn, b, e))
    assert_same(Y2, Y)


def test_ntt_refuses_what_two_primes_cannot_hold():
    with pytest.raises(hmv.HmvError) as ei:
        hmv.Plan(9000, 33220, method=hmv.NTT)
    assert ei.value.status == 7  # HMV_EUNSUPPORTED
    with pytest.raises(hmv.HmvError):
        hmv.Plan(100, 1000, method=hmv.NTT, levels=2)


def test_ntt_benchmark_workload_sampled_and_equal_to_the_tensor_core_path():
    """n = 8000, b = 33220: 256 seeded rows (every residue mod 64) against the
    oracle, and all rows equal to the cost model's Karatsuba/Toom plan."""
    n, b, h, x = workload("large")
    y = ntt(n, b, h, x)
    rows = sampled_parity(oracle.HANKEL, n, h, x, y, 256, 5, residues=64)
    assert len(rows) >= 256
    with hmv.Plan(n, b) as p:
        p.load_matrix(h)
        yt = p.matvec(x)
    assert_same(y, yt)


def ntt_case(K):
    """(n, b) whose Hankel product needs a transform of exactly 2^K points:
    (2n - 1) S <= 2^K < 2 (2n - 1) S with slot stride S = 2 ceil(b/16) - 1."""
    b = 1000 if K <= 18 else (8192 if K <= 22 else 33220)
    S = 2 * -(-b // 16) - 1
    return ((1 << K) // S + 1) // 2, b


@pytest.mark.parametrize("K", range(13, 26))
def test_ntt_every_pass_split(K):
    """Transforms of 2^13 .. 2^25 points: every split of the stages into
    passes of 6 to 9 (13 = 7 + 6 up to 25 = 9 + 8 + 8) and so every register
    kernel shape, as the last (middle) pass and as a spaced one.  All rows
    against the oracle where that is cheap, else 32 seeded rows (and the
    largest) against it and all rows against the tensor-core path."""
    n, b = ntt_case(K)
    h = uniform_vec(9500 + K, 0, 2 * n - 1, b, 1)
    x = uniform_vec(9500 + K, 1, n, b, 0)
    with hmv.Plan(n, b, method=hmv.NTT) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        st = p.stats()
    assert st["fft_log2_len"] == K
    L32 = -(-b // 32)
    if n * n * L32 * L32 <= 5e9:
        assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))
    else:
        sampled_parity(oracle.HANKEL, n, h, x, y, 32, K)
        with hmv.Plan(n, b) as p:
            p.load_matrix(h)
            assert_same(y, p.matvec(x))
