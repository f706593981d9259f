"""Lanczos support on the GPU: hmv_dot and hmv_lincomb against exact
arithmetic, and the driver against the oracle's recurrence bit for bit."""
from fractions import Fraction

import numpy as np
import pytest

import paper_1402_5287_gb300 as pkg
from oracle import lanczos as ol
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec
from paper_1402_5287_gb300.lanczos import Lanczos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def dev(v, torch):
    return (torch.from_numpy(v.limbs.view(np.int32)).cuda(), torch.from_numpy(v.neg).cuda())


def ptrs(t):
    return t[0].data_ptr(), t[1].data_ptr()


# (777, 33220), (1500, 33220) and (5000, 4096) take the dense path (digit
# planes on the tensor cores; the last in two 4096-row chunks, the second
# ragged); the others the CUDA-core kernel
@pytest.mark.parametrize("n,b", [(1, 32), (100, 1000), (777, 33220), (64, 2048), (1500, 33220), (5000, 4096)])
def test_dot_is_exact(n, b):
    torch = pytest.importorskip("torch")
    x = uniform_vec(1000 + n, 0, n, b, 0)
    y = uniform_vec(1000 + n, 1, n, b, 0)
    with hmv.Plan(n, b, method=hmv.SCHOOLBOOK) as p:
        xd, yd = dev(x, torch), dev(y, torch)
        torch.cuda.synchronize()
        got = hmv.dot_device(p, ptrs(xd), ptrs(yd))
    assert got == sum(a * c for a, c in zip(x.to_ints(), y.to_ints()))


@pytest.mark.parametrize("n,b", [(1200, 33220), (300, 1000)])
def test_dot_of_a_vector_with_itself_is_exact(n, b):
    """x = y (the dense path encodes the digit planes once)."""
    torch = pytest.importorskip("torch")
    x = uniform_vec(2000 + n, 0, n, b, 0)
    with hmv.Plan(n, b, method=hmv.SCHOOLBOOK) as p:
        xd = dev(x, torch)
        torch.cuda.synchronize()
        got = hmv.dot_device(p, ptrs(xd), ptrs(xd))
    assert got == sum(a * a for a in x.to_ints())


# (1200, 33220): the b-bit scalars take the dense path (Toeplitz digit
# matrices on the tensor cores, two 4096-digit chunks), small ones the
# CUDA-core kernel, in the same call
@pytest.mark.parametrize("n,b", [(50, 512), (300, 4096), (9, 65), (1200, 33220)])
def test_lincomb_matches_oracle(n, b):
    torch = pytest.importorskip("torch")
    xs = [uniform_vec(1100 + n, t, n, b, e) for t, e in enumerate((2, -1, 0))]
    cases = [[(1, 0)], [(3, 5), (-(1 << (b - 1)) - 5, -b)], [(1, 0), (-12345678901, -40), ((1 << b) - 1, 7)],
             [(-1, 0), (1, 100)]]  # the last pair differs in scale by 100 bits
    with hmv.Plan(n, b) as p:
        xd = [dev(v, torch) for v in xs]
        out = (torch.zeros((n, p.L32), dtype=torch.int32, device="cuda"), torch.zeros(n, dtype=torch.uint8,
                                                                                    device="cuda"))
        torch.cuda.synchronize()
        for cs in cases:
            terms = [(c, ce, ptrs(xd[k]), xs[k].exponent) for k, (c, ce) in enumerate(cs)]
            e = hmv.lincomb_device(p, terms, ptrs(out))
            want = ol.lincomb([(c, ce, ol._Vec(xs[k].limbs, xs[k].neg, b, xs[k].exponent))
                               for k, (c, ce) in enumerate(cs)], b)
            assert e == want.exponent
            assert np.array_equal(out[0].cpu().numpy().view(np.uint32), want.limbs)
            assert np.array_equal(out[1].cpu().numpy(), want.neg)
        # in place: y is also the first term
        terms = [(1, 0, ptrs(xd[0]), xs[0].exponent), (-7, 3, ptrs(xd[1]), xs[1].exponent)]
        e = hmv.lincomb_device(p, terms, ptrs(xd[0]))
        want = ol.lincomb([(1, 0, ol._Vec(xs[0].limbs, xs[0].neg, b, xs[0].exponent)),
                           (-7, 3, ol._Vec(xs[1].limbs, xs[1].neg, b, xs[1].exponent))], b)
        assert e == want.exponent and np.array_equal(xd[0][0].cpu().numpy().view(np.uint32), want.limbs)


@pytest.mark.parametrize("n,b,steps,flags", [(40, 512, 6, 0), (200, 2048, 4, 0), (120, 1024, 3, hmv.FLAG_DIGIT_TOOM6),
                                             (64, 800, 3, hmv.FLAG_DIGIT_SPLIT1)])
def test_driver_equals_oracle_recurrence(n, b, steps, flags):
    pytest.importorskip("torch")
    h = uniform_vec(1200 + n, 0, 2 * n - 1, b, 1)
    x = uniform_vec(1200 + n, 1, n, b, 0)
    with hmv.Plan(n, b, flags=flags, method=hmv.KARATSUBA) as p:
        p.load_matrix(h)
        lz = Lanczos(p, x)
        alphas, betas = lz.run(steps)
        v = lz.vector()
    oa, ob, ov = ol.lanczos(h, x, steps)
    assert alphas == oa and betas == ob
    assert v.exponent == ov.exponent and np.array_equal(v.limbs, ov.limbs) and np.array_equal(v.neg, ov.neg)


def test_driver_anti_identity_breakdown():
    pytest.importorskip("torch")
    n, b = 6, 64
    h = FixedVec.from_ints([1 << (b - 1) if k == n - 1 else 0 for k in range(2 * n - 1)], b, 1)
    x = FixedVec.from_ints([1 << (b - 1) if j == 0 else 0 for j in range(n)], b, 1)
    with hmv.Plan(n, b) as p:
        p.load_matrix(h)
        alphas, betas = Lanczos(p, x).run(5)
    assert [a[0] for a in alphas] == [0, 0]
    assert betas[0][0] * Fraction(2) ** betas[0][1] == 1 and betas[1] == (0, 0)
