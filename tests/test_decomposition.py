"""Sec. 1's FFT formula and Sec. 2's decomposition, written out literally.

* the FFT method of Sec. 1 (a^, x^, first n entries of the circular
  convolution) equals the schoolbook product (exact for small integers);
* the decomposition identity with exact integer pieces recovers y from
  rows 2l(i-1)+1 .. 2l(i-1)+l of y^ = A^ x^;
* with double-precision pieces and a double FFT (what Sec. 2 proposes) the
  result keeps only about double-precision accuracy whatever b is: the
  accuracy question Sec. 2 leaves open, measured.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle.decomposition import decomposition_exact, decomposition_fp64, hankel_fft


def brute(a, x):
    n = len(x)
    return [sum(a[i + j] * x[j] for j in range(n)) for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 10, 33])
def test_sec1_fft_formula(n):
    rng = random.Random(n)
    a = [rng.randint(-99, 99) for _ in range(2 * n - 1)]
    x = [rng.randint(-99, 99) for _ in range(n)]
    y = hankel_fft(np.array(a, dtype=float), np.array(x, dtype=float))
    assert [int(round(v)) for v in y] == brute(a, x)


@pytest.mark.parametrize("n,l,w", [(1, 1, 8), (2, 2, 4), (3, 2, 8), (5, 4, 16), (7, 3, 5), (12, 6, 7)])
def test_decomposition_identity_exact(n, l, w):
    rng = random.Random(100 * n + l)
    b = l * w
    a = [rng.choice((-1, 1)) * rng.getrandbits(b) for _ in range(2 * n - 1)]
    x = [rng.choice((-1, 1)) * rng.getrandbits(b) for _ in range(n)]
    assert decomposition_exact(a, x, l, w) == brute(a, x)


@pytest.mark.parametrize("n", [4, 16, 64])
@pytest.mark.parametrize("w,l", [(16, 2), (16, 8), (16, 32), (32, 8), (8, 32)])
def test_decomposition_fp64_keeps_only_double_accuracy(n, w, l):
    rng = random.Random(7 * n + w + l)
    b = w * l
    a = [Fraction(rng.choice((-1, 1)) * rng.getrandbits(b), 1 << b) for _ in range(2 * n - 1)]
    x = [Fraction(rng.choice((-1, 1)) * rng.getrandbits(b), 1 << b) for _ in range(n)]
    y = brute(a, x)
    yf = decomposition_fp64(a, x, l, w, b)
    err = max(abs(Fraction(v) - t) / abs(t) for v, t in zip(yf, y) if t != 0)
    bits = -math.log2(float(err))
    assert 35 < bits < 56          # about double precision ...
    assert bits < b or b <= 32     # ... so any b above ~50 bits is lost
