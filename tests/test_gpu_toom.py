"""Toom-Cook splits of the mantissas (HMV_FLAG_DIGIT_TOOM4/6): bit-exact
parity with the oracle on every row, for every matrix kind, at worst-case
digits, and equality with the Karatsuba split at full size."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec, workload

from test_gpu_parity import assert_same, oracle_matvec, sampled_parity

pytestmark = pytest.mark.gpu

T4 = hmv.FLAG_DIGIT_TOOM4
TOOMS = [(hmv.FLAG_DIGIT_TOOM4, 7), (hmv.FLAG_DIGIT_TOOM6, 11), (hmv.FLAG_DIGIT_TOOM8, 15)]


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def run(n, b, h, x, flags=T4, kind=hmv.HANKEL, nrhs=1, method=hmv.AUTO):
    with hmv.Plan(n, b, kind=kind, method=method, flags=flags, nrhs=nrhs) as p:
        p.load_matrix(h)
        return p.matvec(x), p.stats()


# b: the narrowest splits (one-limb parts), ragged top parts, several tiles
@pytest.mark.parametrize("flags,products", TOOMS)
@pytest.mark.parametrize("n,b", [(64, 2048), (100, 700), (1, 192), (7, 257), (30, 4100), (140, 1000), (3, 193),
                                 (5, 225), (2, 300)])
def test_toom_all_rows(flags, products, n, b):
    h = uniform_vec(70 + n, 0, 2 * n - 1, b, 1)
    x = uniform_vec(70 + n, 1, n, b, -1)
    K = (products + 1) // 2
    if (b + 31) // 32 < K:  # fewer limbs than parts: refused
        with pytest.raises(hmv.HmvError):
            run(n, b, h, x, flags=flags)
        return
    y, st = run(n, b, h, x, flags=flags)
    assert st["digit_products"] == products
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


def test_toom4_narrowest():
    n, b = 9, 97  # four parts: three full limbs and one bit
    h = uniform_vec(71, 0, 2 * n - 1, b)
    x = uniform_vec(71, 1, n, b)
    assert_same(run(n, b, h, x)[0], oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("flags,products", TOOMS)
@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
def test_toom_toeplitz_circulant(flags, products, kind):
    n, b = 90, 600
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = uniform_vec(73, 0, hlen, b)
    x = uniform_vec(73, 1, n, b)
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    assert_same(run(n, b, h, x, flags=flags, kind=kind)[0], oracle_matvec(ok, n, h, x))


@pytest.mark.parametrize("flags,products", TOOMS)
def test_toom_block_rhs_and_method_karatsuba(flags, products):
    n, b, k = 40, 900, 3
    h = uniform_vec(75, 0, 2 * n - 1, b)
    x = uniform_vec(75, 1, n * k, b)
    y, _ = run(n, b, h, x, flags=flags, nrhs=k, method=hmv.KARATSUBA)
    y0, _ = run(n, b, h, x, flags=0, nrhs=k, method=hmv.KARATSUBA)
    assert_same(y, y0)


@pytest.mark.parametrize("flags,products", TOOMS)
def test_toom_worst_case_digits(flags, products):
    """All-ones and 0x8080.. mantissas with mixed signs: every evaluation
    point at its largest magnitude."""
    n, b = 70, 2046
    for m in (int("80" * ((b + 7) // 8), 16) & ((1 << b) - 1), (1 << b) - 1):
        h = FixedVec.from_ints([m if k % 3 else -m for k in range(2 * n - 1)], b, 0)
        x = FixedVec.from_ints([-m if j % 2 else m for j in range(n)], b, 0)
        assert_same(run(n, b, h, x, flags=flags)[0], oracle_matvec(oracle.HANKEL, n, h, x))
        h = FixedVec.from_ints([-m] * (2 * n - 1), b, 0)
        x = FixedVec.from_ints([-m] * n, b, 0)
        assert_same(run(n, b, h, x, flags=flags)[0], oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("flags,products", TOOMS)
def test_toom_zero_vector(flags, products):
    n, b = 20, 512
    h = uniform_vec(77, 0, 2 * n - 1, b)
    x = FixedVec.from_ints([0] * n, b, -3)
    assert_same(run(n, b, h, x, flags=flags)[0], oracle_matvec(oracle.HANKEL, n, h, x))


def test_toom_large_workload_matches_karatsuba_split():
    n, b, h, x = workload("large")
    y2, st2 = run(n, b, h, x, flags=hmv.FLAG_DIGIT_SPLIT2)
    assert st2["digit_products"] == 9
    for flags, products in TOOMS:
        y, st = run(n, b, h, x, flags=flags)
        assert st["digit_products"] == products
        assert_same(y, y2)
    sampled_parity(oracle.HANKEL, n, h, x, y, 3, 13)


def test_matvec_many_mixes_split_and_unsplit_plans():
    """hmv_matvec_many with Toom, Karatsuba-split and unsplit plans in one
    step (the serving path): every result equals the plan's own matvec."""
    import torch
    dev = torch.device("cuda", 0)
    cases = [(60, 3000, hmv.FLAG_DIGIT_TOOM6, hmv.HANKEL), (45, 2000, hmv.FLAG_DIGIT_TOOM4, hmv.TOEPLITZ),
             (50, 1500, hmv.FLAG_DIGIT_SPLIT1, hmv.HANKEL), (30, 700, 0, hmv.CIRCULANT), (20, 300, 0, hmv.HANKEL)]
    plans, keep, xp, yp, exps, want = [], [], [], [], [], []
    for i, (n, b, flags, kind) in enumerate(cases):
        hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
        h = uniform_vec(300 + i, 0, hlen, b, 1)
        x = uniform_vec(300 + i, 1, n, b, -2)
        want.append(run(n, b, h, x, flags=flags, kind=kind, method=hmv.KARATSUBA)[0])
        p = hmv.Plan(n, b, kind=kind, method=hmv.KARATSUBA, flags=flags)
        p.load_matrix(h)
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl, yn = torch.empty_like(xl), torch.empty_like(xn)
        plans.append(p)
        keep.append((xl, xn, yl, yn, b))
        xp.append((xl.data_ptr(), xn.data_ptr()))
        yp.append((yl.data_ptr(), yn.data_ptr()))
        exps.append(x.exponent)
    for _ in range(2):  # twice: the descendants' buffers are reused
        out = hmv.matvec_many_device(plans, xp, yp, exps)
        torch.cuda.synchronize()
        for (xl, xn, yl, yn, b), e, w in zip(keep, out, want):
            assert_same(FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), b, e), w)
    for p in plans:
        p.close()
