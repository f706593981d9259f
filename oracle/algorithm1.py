"""Algorithm 1 of Sec. 3 (recursive half-size Hankel products) on Python ints.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The steps follow the paper's numbering and its 1-based notation: the lists
below carry a dummy entry at index 0 so that a[k] is the paper's a_k.
  step 1  base case: n = 2 uses the explicit formula; n = 1 is y_1 = a_1 x_1
          (the paper's recursion never ends for n = 1: m = m1 = 1); an
          optional cutoff n0 > 2 ends the recursion with the schoolbook sum
          of Sec. 1 instead.
  step 2  m = floor((n+1)/2), m1 = ceil((n+1)/2)
  step 3  f_i = x_{2i-1} - x_{2i}, h_i = x_{2i-1}      (i = 1..m,      x_{n+1} = 0)
  step 4  c_i = a_{2i-1} + a_{2i}, d_i = a_{2i}         (i = 1..2m-1,   a_{2n} = 0)
  step 5  g_i = x_{2i-2} - x_{2i-1}                     (i = 1..m1,     x_0 = x_{n+1} = 0)
  step 6  e_i = a_{2i-1}                                (i = 1..2m1-1,  a_{2n+1} = 0)
  step 7  p = Alg1(m, c, h), q = Alg1(m, d, f), r = Alg1(m1, e, g)
  step 8  y_{2i-1} = p_i - q_i; y_{2i} = p_i + r_i if 2i <= n   (i = 1..m)

The range of f follows the algorithm (1..m), not the text before it (1..m1).
Counters record every multiplication of two non-zero operands and every
addition or subtraction, as in the operation counts of Sec. 3.
"""
from __future__ import annotations


class Counts:
    def __init__(self):
        self.mul = 0
        self.add = 0
        self.leaves = 0


def _nz(u, v):
    """1 if the product u*v has to be formed: a product with a zero operand
    (the padding a_{2n} = a_{2n+1} = x_0 = x_{n+1} = 0) is not a
    multiplication, as in the count of Sec. 3 where a_3 = 0 leaves three."""
    return 1 if (u != 0 and v != 0) else 0


def _get(v, k):
    """v[k] with the paper's zero conventions outside the stored range."""
    return v[k] if 1 <= k < len(v) else 0


def algorithm1(a0: list[int], x0: list[int], cutoff: int = 2, counts: Counts | None = None) -> list[int]:
    """y = A_H x for the Hankel matrix of a0 (len 2n-1), 0-based in and out."""
    n = len(x0)
    if len(a0) != 2 * n - 1:
        raise ValueError("a must have 2n-1 entries")
    cnt = counts if counts is not None else Counts()
    y = _alg1(n, [0] + list(a0), [0] + list(x0), max(2, cutoff), cnt)
    return y[1:]


def _alg1(n: int, a: list[int], x: list[int], n0: int, cnt: Counts) -> list[int]:
    # step 1
    if n == 1:
        cnt.mul += _nz(a[1], x[1])
        cnt.leaves += 1
        return [0, a[1] * x[1]]
    if n == 2:
        cnt.mul += _nz(a[1], x[1]) + _nz(a[2], x[2]) + _nz(a[2], x[1]) + _nz(a[3], x[2])
        cnt.add += 2
        cnt.leaves += 1
        return [0, a[1] * x[1] + a[2] * x[2], a[2] * x[1] + a[3] * x[2]]
    if n <= n0:
        cnt.leaves += 1
        y = [0] * (n + 1)
        for i in range(1, n + 1):
            s = 0
            for j in range(1, n + 1):
                s += a[i + j - 1] * x[j]
                cnt.mul += _nz(a[i + j - 1], x[j])
            cnt.add += n - 1
            y[i] = s
        return y
    # step 2
    m = (n + 1) // 2
    m1 = (n + 2) // 2
    # step 3
    f = [0] * (m + 1)
    h = [0] * (m + 1)
    for i in range(1, m + 1):
        f[i] = _get(x, 2 * i - 1) - _get(x, 2 * i)
        h[i] = _get(x, 2 * i - 1)
        cnt.add += 1
    # step 4
    c = [0] * (2 * m)
    d = [0] * (2 * m)
    for i in range(1, 2 * m):
        c[i] = _get(a, 2 * i - 1) + _get(a, 2 * i)
        d[i] = _get(a, 2 * i)
        cnt.add += 1
    # step 5
    g = [0] * (m1 + 1)
    for i in range(1, m1 + 1):
        g[i] = _get(x, 2 * i - 2) - _get(x, 2 * i - 1)
        cnt.add += 1
    # step 6
    e = [0] * (2 * m1)
    for i in range(1, 2 * m1):
        e[i] = _get(a, 2 * i - 1)
    # step 7
    p = _alg1(m, c, h, n0, cnt)
    q = _alg1(m, d, f, n0, cnt)
    r = _alg1(m1, e, g, n0, cnt)
    # step 8
    y = [0] * (n + 1)
    for i in range(1, m + 1):
        y[2 * i - 1] = p[i] - q[i]
        cnt.add += 1
        if 2 * i <= n:
            y[2 * i] = p[i] + r[i]
            cnt.add += 1
    return y


def one_level(a0: list[int], x0: list[int]):
    """Steps 2-6 once, 0-based: returns (m, m1, c, d, e, f, g, h)."""
    n = len(x0)
    a = [0] + list(a0)
    x = [0] + list(x0)
    m = (n + 1) // 2
    m1 = (n + 2) // 2
    h = [_get(x, 2 * i - 1) for i in range(1, m + 1)]
    f = [_get(x, 2 * i - 1) - _get(x, 2 * i) for i in range(1, m + 1)]
    c = [_get(a, 2 * i - 1) + _get(a, 2 * i) for i in range(1, 2 * m)]
    d = [_get(a, 2 * i) for i in range(1, 2 * m)]
    g = [_get(x, 2 * i - 2) - _get(x, 2 * i - 1) for i in range(1, m1 + 1)]
    e = [_get(a, 2 * i - 1) for i in range(1, 2 * m1)]
    return m, m1, c, d, e, f, g, h
