"""Toom-Cook splits of the mantissas (HMV_FLAG_DIGIT_TOOM4/6/8), on the CPU.

The exact rows are bilinear in (h, x), so with every mantissa cut into K
parts V = sum_k V_k 2^(ks) the rows are a polynomial of degree 2K-2 in
t = 2^s: Z(t) = sum_m C_m t^m, C_m = sum_{k+l=m} A(h_k) x_l (the same
observation that gives the Karatsuba step of Sec. 3, with K parts instead of
two).  2K-1 products at the chosen points (fractions homogenised, plus
infinity) fix the C_m.  These tests derive the interpolation here, by exact
elimination over the rationals, and check the whole scheme against the
oracle's direct products, independently of the CUDA tables."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec

# (num, den): t = num/den, (1, 0) = infinity
POINTS = {4: [(0, 1), (1, 1), (-1, 1), (2, 1), (-2, 1), (1, 2), (1, 0)],
          6: [(0, 1), (1, 1), (-1, 1), (2, 1), (-2, 1), (1, 2), (-1, 2), (3, 1), (-3, 1), (1, 3), (1, 0)],
          8: [(0, 1), (1, 1), (-1, 1), (2, 1), (-2, 1), (1, 2), (-1, 2), (3, 1), (-3, 1), (1, 3), (-1, 3),
              (3, 2), (-3, 2), (2, 3), (1, 0)]}
DEN = {4: 360, 6: 1008000, 8: 54486432000}
GROW = {4: 4, 6: 9, 8: 13}  # bits the evaluated parts can exceed s by


def evaluation_matrix(K):
    """Row of point num/den: den^(2K-2) (num/den)^m = num^m den^(2K-2-m)."""
    deg = 2 * K - 2
    return [[Fraction(num ** m * den ** (deg - m)) for m in range(deg + 1)] for num, den in POINTS[K]]


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


@pytest.mark.parametrize("K", [4, 6, 8])
def test_interpolation_denominator_and_recovery(K):
    P_ = 2 * K - 1
    M = evaluation_matrix(K)
    Mi = inverse(M)
    den = 1
    for row in Mi:
        for v in row:
            den = den * v.denominator // math.gcd(den, v.denominator)
    assert den == DEN[K]
    rng = np.random.default_rng(4)
    for _ in range(20):
        C = [int(v) for v in rng.integers(-10 ** 12, 10 ** 12, P_)]
        P = [sum(M_row[m] * C[m] for m in range(P_)) for M_row in M]
        assert [sum(Mi[m][t] * P[t] for t in range(P_)) for m in range(P_)] == C


def parts(v: int, s: int, K: int) -> list[int]:
    sg = -1 if v < 0 else 1
    m = abs(v)
    return [sg * ((m >> (k * s)) & ((1 << s) - 1)) for k in range(K)]


def evaluate(vals, s, point, K):
    num, den = point
    out = []
    for v in vals:
        p = parts(v, s, K)
        out.append(sum(p[k] * num ** k * den ** (K - 1 - k) for k in range(K)))
    return out


@pytest.mark.parametrize("K,n,b", [(4, 5, 130), (4, 9, 257), (4, 16, 1000), (4, 1, 200),
                                   (6, 5, 200), (6, 7, 1000), (6, 3, 161), (8, 5, 300), (8, 6, 1500), (8, 2, 225)])
def test_toom_rows_equal_direct_rows(K, n, b):
    h = uniform_vec(500 + n, 0, 2 * n - 1, b, 0)
    x = uniform_vec(500 + n, 1, n, b, 0)
    hv, xv = h.to_ints(), x.to_ints()
    s = 32 * (((b + 31) // 32 + K - 1) // K)
    bc = s + GROW[K]
    Mi = inverse(evaluation_matrix(K))
    P = []
    for pt in POINTS[K]:
        he, xe = evaluate(hv, s, pt, K), evaluate(xv, s, pt, K)
        assert max(abs(v) for v in he + xe) < 2 ** bc
        z, zn = oracle.exact_rows(oracle.HANKEL, n, bc, FixedVec.from_ints(he, bc, 0), FixedVec.from_ints(xe, bc, 0))
        P.append(oracle.z_to_ints(z, zn))
    z, zn = oracle.exact_rows(oracle.HANKEL, n, b, h, x)
    want = oracle.z_to_ints(z, zn)
    for i in range(n):
        C = [sum(Mi[m][t] * P[t][i] for t in range(2 * K - 1)) for m in range(2 * K - 1)]
        assert all(c.denominator == 1 for c in C)
        assert sum(int(c) << (m * s) for m, c in enumerate(C)) == want[i]


@pytest.mark.parametrize("K", [4, 6, 8])
def test_evaluated_parts_fit_the_child_width(K):
    """The largest evaluation is sum_k |p|^k |q|^(K-1-k) times 2^s - 1 parts: below 2^GROW."""
    worst = max(sum(abs(num) ** k * abs(den) ** (K - 1 - k) for k in range(K)) for num, den in POINTS[K])
    assert worst < 2 ** GROW[K] and worst >= 2 ** (GROW[K] - 1)


def test_toom8_interpolation_sums_fit_int64_through_depth_7():
    """Den C_m is summed in int64 from int16/int32 post-pass digits |d| <= 510 * 2^L:
    with at most four shifted products meeting at a digit, the bound stays
    below 2^62 for index depths up to 7 (the plan refuses deeper ones)."""
    M = evaluation_matrix(8)
    Mi = inverse(M)
    N = [[int(v * DEN[8]) for v in row] for row in Mi]
    assert all((v * DEN[8]).denominator == 1 for row in Mi for v in row)
    rowsum = max(sum(abs(v) for v in row) for row in N)
    assert 4 * rowsum * 510 * 2 ** 7 < 2 ** 62
    assert 4 * rowsum * 510 * 2 ** 8 >= 2 ** 62
    assert DEN[8] == 7776000 * 7007 and 7776000 < 2 ** 24 and 7007 < 2 ** 24
