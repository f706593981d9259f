"""The decomposition approach of Sec. 2, written out literally.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every entry is a sum of l pieces, a_i = sum_k a_ik and x_j = sum_k x_jk (the
pieces carry their own weights).  Sec. 2 builds
  * the auxiliary Hankel matrix A^ of order m = 2nl from the sequence in
    which the l pieces of each a_i appear twice in a row,
    t = (a_11..a_1l, a_11..a_1l, a_21..a_2l, a_21..a_2l, ...),
  * the vector x^ = (x_11..x_1l, 0 x l, x_21..x_2l, 0 x l, ...),
and recovers y from block sums of y^ = A^ x^.  For this A^ the sums that
give y_i are rows 2l(i-1)+1 .. 2l(i-1)+l of y^ (1-based):
  y^_{2l(i-1)+s} = sum_j sum_q a_{i+j-1, ((s+q-2) mod l)+1} x_jq,
so summing over s = 1..l runs every piece of a_{i+j-1} against every piece
of x_j.  (The printed formula sums rows l(i-1)+1 .. il, which would fit an
A^ without the doubled blocks.)

`decomposition_exact` does this in exact integers; `decomposition_fp64`
does it the way Sec. 2 proposes, with the pieces as doubles and y^ by the
FFT method of Sec. 1 (circulant embedding), so that the accuracy question
left open at the end of Sec. 2 can be measured.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def pieces(v: int, l: int, w: int) -> list[int]:
    """v = sum_k p_k with p_k = (w-bit digit k of |v|, signed) * 2^(w k)."""
    s = -1 if v < 0 else 1
    m = abs(v)
    return [s * (((m >> (w * k)) & ((1 << w) - 1)) << (w * k)) for k in range(l)]


def aux_sequence(a_pieces: list[list]) -> list:
    """t: the pieces of each a_i twice in a row."""
    t = []
    for pc in a_pieces:
        t.extend(pc)
        t.extend(pc)
    return t


def aux_vector(x_pieces: list[list], l: int) -> list:
    xv = []
    for pc in x_pieces:
        xv.extend(pc)
        xv.extend([0] * l)
    return xv


def recover(yhat: list, n: int, l: int) -> list:
    return [sum(yhat[2 * l * i + s] for s in range(l)) for i in range(n)]


def decomposition_exact(a: list[int], x: list[int], l: int, w: int) -> list[int]:
    """y = A_H x through A^ x^ with exact integer pieces (0-based lists)."""
    n = len(x)
    t = aux_sequence([pieces(v, l, w) for v in a])
    xv = aux_vector([pieces(v, l, w) for v in x], l)
    m = 2 * n * l
    t = t + [0] * (2 * m - 1 - len(t))
    yhat = [sum(t[r + c] * xv[c] for c in range(m) if xv[c]) for r in range(m)]
    return recover(yhat, n, l)


def hankel_fft(t: np.ndarray, xv: np.ndarray) -> np.ndarray:
    """y^ = A^ x^ for the Hankel matrix of t (length 2m-1) by the FFT method of
    Sec. 1: with a^ = (t_{m-1}..t_{2m-2}, t_0..t_{m-2}) and the reversed
    x^ padded with zeros, y^ is the first m entries of the circular
    convolution of length 2m-1."""
    m = len(xv)
    ahat = np.concatenate([t[m - 1:2 * m - 1], t[:m - 1]])
    chat = np.concatenate([xv[::-1], np.zeros(m - 1)])
    return np.fft.ifft(np.fft.fft(ahat) * np.fft.fft(chat)).real[:m]


def decomposition_fp64(a: list[Fraction], x: list[Fraction], l: int, w: int, scale_bits: int) -> list[float]:
    """The same with double-precision pieces and a double-precision FFT.
    a, x: exact values v = M 2^-scale_bits; the pieces are M's w-bit digits
    times their weights, rounded to doubles."""
    n = len(x)

    def fpieces(v: Fraction) -> list[float]:
        mant = int(v * (1 << scale_bits))
        return [float(Fraction(p, 1 << scale_bits)) for p in pieces(mant, l, w)]

    t = np.array(aux_sequence([fpieces(v) for v in a]))
    xv = np.array(aux_vector([fpieces(v) for v in x], l))
    m = 2 * n * l
    t = np.concatenate([t, np.zeros(2 * m - 1 - len(t))])
    return recover(list(hankel_fft(t, xv)), n, l)
