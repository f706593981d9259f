"""Lanczos recurrence on the oracle's exact products (the iteration the
paper's introduction names as the consumer of fast multiprecision Hankel
products), with the arithmetic contract of the GPU driver.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

    w = A v_k;  alpha_k = <v_k, w>/<v_k, v_k>;  w -= alpha_k v_k + beta_k v_{k-1};
    beta_{k+1} = <w, w>/<v_k, v_k>;  v_{k+1} = w

Vectors: b-bit mantissas with one shared exponent (value M 2^(E-b)); A v
and the update of w are the exact integers rounded once by the oracle's rule
(least shared exponent, ties to even); inner products exact; alpha and beta
the exact rationals rounded to b-bit floating point with ties to even
(computed with Fractions).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import HANKEL, matvec, round_rows


def round_rational(q: Fraction, b: int) -> tuple[int, int]:
    """(m, e): m 2^e = q rounded to b significant bits, ties to even; 0 -> (0, 0)."""
    if q == 0:
        return 0, 0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length() - b
    while a / Fraction(2) ** e >= 2 ** b:
        e += 1
    while a / Fraction(2) ** e < 2 ** (b - 1):
        e -= 1
    m = round(a / Fraction(2) ** e)  # Fraction.__round__: ties to even
    if m == 2 ** b:
        m //= 2
        e += 1
    return (-m if q < 0 else m), e


def _ints(limbs: np.ndarray, neg: np.ndarray) -> list[int]:
    out = []
    for r in range(limbs.shape[0]):
        m = int.from_bytes(np.ascontiguousarray(limbs[r], dtype="<u4").tobytes(), "little")
        out.append(-m if neg[r] else m)
    return out


class _Vec:
    def __init__(self, limbs, neg, b, exponent):
        self.limbs, self.neg, self.b, self.exponent = limbs, neg, b, exponent


def _round_vector(vals: list[int], scale: int, b: int):
    """Round the exact values v * 2^scale to a b-bit block vector: (limbs, neg, E)."""
    zl = max(1, (max((abs(v).bit_length() for v in vals), default=1) + 31) // 32) + 1
    z = np.zeros((len(vals), zl), dtype=np.uint32)
    zn = np.zeros(len(vals), dtype=np.uint8)
    for i, v in enumerate(vals):
        z[i] = np.frombuffer(abs(v).to_bytes(4 * zl, "little"), dtype="<u4")
        zn[i] = 1 if v < 0 else 0
    return round_rows(z, zn, b, scale + 2 * b)


def lincomb(terms, b: int):
    """terms: [(c, ce, vec)]: value sum c 2^ce * vec; exact, then rounded."""
    s = [ce + v.exponent - b for c, ce, v in terms]
    smin = min(s)
    n = terms[0][2].limbs.shape[0]
    acc = [0] * n
    for (c, ce, v), sk in zip(terms, s):
        m = _ints(v.limbs, v.neg)
        for i in range(n):
            acc[i] += c * m[i] << (sk - smin)
    y, yn, e = _round_vector(acc, smin, b)
    return _Vec(y, yn, b, e)


def dot(x, y) -> int:
    return sum(a * c for a, c in zip(_ints(x.limbs, x.neg), _ints(y.limbs, y.neg)))


def lanczos(h, x0, steps: int):
    """alpha_k, beta_{k+1} as (mantissa, exponent) and the final v, for the
    Hankel matrix of h (2n-1 entries) from x0."""
    b = x0.b
    n = x0.limbs.shape[0]
    v = _Vec(x0.limbs, x0.neg, b, x0.exponent)
    u = None
    beta = (0, 0)
    dvv = dot(v, v)
    alphas, betas = [], []
    for k in range(steps):
        if dvv == 0:
            break
        wl, wn, ew = matvec(HANKEL, n, h, v)
        w = _Vec(wl, wn, b, ew)
        dvw = dot(v, w)
        alpha = round_rational(Fraction(dvw, dvv) * Fraction(2) ** (ew - v.exponent), b)
        terms = [(1, 0, w), (-alpha[0], alpha[1], v)]
        if k > 0 and beta[0] != 0:
            terms.append((-beta[0], beta[1], u))
        w = lincomb(terms, b)
        dww = dot(w, w)
        beta = round_rational(Fraction(dww, dvv) * Fraction(2) ** (2 * w.exponent - 2 * v.exponent), b)
        alphas.append(alpha)
        betas.append(beta)
        u, v, dvv = v, w, dww
        if dww == 0:
            break
    return alphas, betas, v
