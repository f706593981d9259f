"""The oracle's Lanczos recurrence (oracle/lanczos.py), pinned on the CPU
against closed forms and against the exact rational recurrence."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import lanczos as ol
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec


def test_round_rational_known_values():
    F = Fraction
    assert ol.round_rational(F(1), 4) == (8, -3)
    assert ol.round_rational(F(-3, 2), 2) == (-3, -1)
    assert ol.round_rational(F(5, 2), 2) == (2, 0)       # 2.5: tie between 2 and 3 -> the even mantissa 2
    assert ol.round_rational(F(7, 2), 2) == (2, 1)       # 3.5: tie between 3 and 4 = 2 * 2^1 -> 4
    assert ol.round_rational(F(0), 7) == (0, 0)
    assert ol.round_rational(F(255, 256), 4) == (8, -3)  # rounds up to 1


def test_anti_identity_closed_form():
    """A = J (h with a single 1 at index n-1), v_0 = e_0: alpha = 0, beta_1 = 1,
    alpha_1 = 0 and then w = e_0 - beta_1 e_0 = 0."""
    n, b = 6, 64
    h = FixedVec.from_ints([1 << (b - 1) if k == n - 1 else 0 for k in range(2 * n - 1)], b, 1)
    x = FixedVec.from_ints([1 << (b - 1) if j == 0 else 0 for j in range(n)], b, 1)
    alphas, betas, _ = ol.lanczos(h, x, 5)
    assert [a[0] for a in alphas] == [0, 0]
    assert betas[0][0] * Fraction(2) ** betas[0][1] == 1
    assert betas[1] == (0, 0)


def exact_lanczos(H, x, steps):
    """The recurrence in exact rational arithmetic (no rounding)."""
    n = len(x)
    v = [Fraction(t) for t in x]
    u = [Fraction(0)] * n
    beta = Fraction(0)
    dvv = sum(t * t for t in v)
    alphas, betas, vs = [], [], [v]
    for k in range(steps):
        w = [sum(H[i][j] * v[j] for j in range(n)) for i in range(n)]
        alpha = sum(a * c for a, c in zip(v, w)) / dvv
        w = [w[i] - alpha * v[i] - beta * u[i] for i in range(n)]
        dww = sum(t * t for t in w)
        beta = dww / dvv
        alphas.append(alpha)
        betas.append(beta)
        u, v, dvv = v, w, dww
        vs.append(v)
        if dww == 0:
            break
    return alphas, betas, vs


@pytest.mark.parametrize("n,b,steps", [(5, 600, 4), (8, 400, 5)])
def test_matches_exact_rational_recurrence(n, b, steps):
    h = uniform_vec(900 + n, 0, 2 * n - 1, b, 0)
    x = uniform_vec(900 + n, 1, n, b, 0)
    hv = [Fraction(m, 2 ** b) for m in h.to_ints()]
    xv = [Fraction(m, 2 ** b) for m in x.to_ints()]
    H = [[hv[i + j] for j in range(n)] for i in range(n)]
    ea, eb, evs = exact_lanczos(H, xv, steps)
    # the exact recurrence itself: successive vectors are orthogonal
    for k in range(len(evs) - 1):
        assert sum(a * c for a, c in zip(evs[k], evs[k + 1])) == 0
    alphas, betas, _ = ol.lanczos(h, x, steps)
    assert len(alphas) == len(ea)
    for (m, e), q in zip(alphas, ea):
        assert abs(m * Fraction(2) ** e - q) <= abs(q) * Fraction(1, 2 ** (b - 60)) + Fraction(1, 2 ** (b - 60))
    for (m, e), q in zip(betas, eb):
        assert abs(m * Fraction(2) ** e - q) <= abs(q) * Fraction(1, 2 ** (b - 60))


def test_lincomb_is_exact_before_one_rounding():
    b = 96
    x = uniform_vec(950, 0, 7, b, 3)
    y = uniform_vec(950, 1, 7, b, -2)
    vx = ol._Vec(x.limbs, x.neg, b, x.exponent)
    vy = ol._Vec(y.limbs, y.neg, b, y.exponent)
    c1, e1, c2, e2 = 12345, -20, -(1 << 40) + 7, 5
    r = ol.lincomb([(c1, e1, vx), (c2, e2, vy)], b)
    got = [Fraction(m) * Fraction(2) ** (r.exponent - b) for m in FixedVec(r.limbs, r.neg, b, r.exponent).to_ints()]
    exact = [c1 * Fraction(2) ** e1 * Fraction(a) * Fraction(2) ** (x.exponent - b) +
             c2 * Fraction(2) ** e2 * Fraction(c) * Fraction(2) ** (y.exponent - b)
             for a, c in zip(x.to_ints(), y.to_ints())]
    ulp = Fraction(2) ** (r.exponent - b)
    assert all(abs(g - t) <= ulp / 2 for g, t in zip(got, exact))
    assert max(abs(t) for t in exact) < 2 ** r.exponent  # least shared exponent
    assert max(abs(t) for t in exact) >= 2 ** (r.exponent - 1) - ulp
