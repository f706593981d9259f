"""Toom-Cook 4-way split of the mantissas (HMV_FLAG_DIGIT_TOOM4), on the CPU.

The exact rows are bilinear in (h, x), so with every mantissa cut into four
parts V = sum_k V_k 2^(ks) the rows are a degree-6 polynomial in t = 2^s:
Z(t) = sum_m C_m t^m, C_m = sum_{k+l=m} A(h_k) x_l (the same observation that
gives the Karatsuba step of Sec. 3, with four parts instead of two).  Seven
products at the points 0, 1, -1, 2, -2, 1/2 (homogenised) and infinity fix
the C_m.  These tests derive the interpolation here, by exact elimination
over the rationals, and check the whole scheme against the oracle's direct
products, independently of the CUDA tables."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec

POINTS = [(0, 1), (1, 1), (-1, 1), (2, 1), (-2, 1), (1, 2), (1, 0)]  # (num, den): t = num/den, (1, 0) = infinity


def evaluation_matrix():
    """Row of point num/den: den^6 (num/den)^m = num^m den^(6-m)."""
    return [[Fraction(num ** m * den ** (6 - m)) for m in range(7)] for num, den in POINTS]


def inverse(M):
    n = len(M)
    A = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        f = A[c][c]
        A[c] = [v / f for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                g = A[r][c]
                A[r] = [a - g * b for a, b in zip(A[r], A[c])]
    return [row[n:] for row in A]


def test_interpolation_has_denominator_360_and_recovers_coefficients():
    Mi = inverse(evaluation_matrix())
    den = 1
    for row in Mi:
        for v in row:
            den = den * v.denominator // np.gcd(den, v.denominator)
    assert den == 360
    rng = np.random.default_rng(4)
    for _ in range(20):
        C = [int(v) for v in rng.integers(-10 ** 12, 10 ** 12, 7)]
        P = [sum(M_row[m] * C[m] for m in range(7)) for M_row in evaluation_matrix()]
        assert [sum(Mi[m][t] * P[t] for t in range(7)) for m in range(7)] == C


def parts(v: int, s: int) -> list[int]:
    sg = -1 if v < 0 else 1
    m = abs(v)
    return [sg * ((m >> (k * s)) & ((1 << s) - 1)) for k in range(4)]


def evaluate(vals, s, point):
    num, den = point
    out = []
    for v in vals:
        p = parts(v, s)
        out.append(sum(p[k] * num ** k * den ** (3 - k) for k in range(4)))
    return out


@pytest.mark.parametrize("n,b", [(5, 130), (9, 257), (16, 1000), (1, 200)])
def test_toom4_rows_equal_direct_rows(n, b):
    h = uniform_vec(500 + n, 0, 2 * n - 1, b, 0)
    x = uniform_vec(500 + n, 1, n, b, 0)
    hv, xv = h.to_ints(), x.to_ints()
    s = 32 * (((b + 31) // 32 + 3) // 4)
    bc = s + 4
    Mi = inverse(evaluation_matrix())
    P = []
    for pt in POINTS:
        he, xe = evaluate(hv, s, pt), evaluate(xv, s, pt)
        assert max(abs(v) for v in he + xe) < 2 ** bc
        z, zn = oracle.exact_rows(oracle.HANKEL, n, bc, FixedVec.from_ints(he, bc, 0), FixedVec.from_ints(xe, bc, 0))
        P.append(oracle.z_to_ints(z, zn))
    z, zn = oracle.exact_rows(oracle.HANKEL, n, b, h, x)
    want = oracle.z_to_ints(z, zn)
    for i in range(n):
        C = [sum(Mi[m][t] * P[t][i] for t in range(7)) for m in range(7)]
        assert all(c.denominator == 1 for c in C)
        assert sum(int(c) << (m * s) for m, c in enumerate(C)) == want[i]
