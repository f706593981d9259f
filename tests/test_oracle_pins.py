"""Pins for the CPU oracle: checks against facts fixed by the paper and by
mathematics, never against the oracle itself.

  * brute force on the explicitly materialised matrices of Sec. 1
    (A_H, A_T, A_C) with Python integers, tiny n
  * the explicit n = 2 formula of Algorithm 1, step 1
  * the 4 -> 3 multiplication identities of Sec. 3 and the one-level
    identities y_{2i-1} = p_i - q_i, y_{2i} = p_i + r_i (Sec. 3)
  * Algorithm 1 (Python ints) equal to brute force, and its operation counts
    within the bounds of Sec. 3
  * Toeplitz = row-reversed Hankel (Sec. 1), unit vectors, linearity
  * the closed form of the Hilbert Hankel h_k = 1/(k+1) with exact rationals
  * rounding against exact rational round-half-even and a brute-force
    search for the least exponent
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.algorithm1 import Counts, algorithm1, one_level
from paper_1402_5287_gb300.inputs import FixedVec, hilbert_hankel, uniform_vec

H, T, C = oracle.HANKEL, oracle.TOEPLITZ, oracle.CIRCULANT


def rand_ints(rng, count, bits):
    return [rng.choice((-1, 1)) * rng.getrandbits(bits) for _ in range(count)]


def exact(kind, n, b, a_ints, x_ints, rows=None, threads=2):
    a = FixedVec.from_ints(a_ints, b, 0)
    x = FixedVec.from_ints(x_ints, b, 0)
    z, zn = oracle.exact_rows(kind, n, b, a, x, rows, threads)
    return oracle.z_to_ints(z, zn)


def materialise(kind, n, a):
    """The matrices of Sec. 1 written out entry by entry (1-based in the paper)."""
    A = [[0] * n for _ in range(n)]
    for i1 in range(1, n + 1):
        for j1 in range(1, n + 1):
            if kind == H:      # (A_H)_{ij} = a_{i+j-1}
                k1 = i1 + j1 - 1
            elif kind == T:    # (A_T)_{ij} = a_{n-i+j}
                k1 = n - i1 + j1
            else:              # (A_C)_{ij} = a_{((i-j) mod n)+1}
                k1 = ((i1 - j1) % n) + 1
            A[i1 - 1][j1 - 1] = a[k1 - 1]
    return A


def brute(A, x):
    return [sum(Aij * xj for Aij, xj in zip(row, x)) for row in A]


@pytest.mark.parametrize("kind", [H, T, C])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 31, 40])
@pytest.mark.parametrize("b", [1, 31, 32, 33, 100])
def test_bruteforce_materialised(kind, n, b):
    rng = random.Random(1000 * n + 10 * b + kind)
    alen = n if kind == C else 2 * n - 1
    a = rand_ints(rng, alen, b)
    x = rand_ints(rng, n, b)
    assert exact(kind, n, b, a, x) == brute(materialise(kind, n, a), x)


def test_full_width_single_products():
    rng = random.Random(7)
    b = 33220
    for _ in range(3):
        a = rand_ints(rng, 1, b)
        x = rand_ints(rng, 1, b)
        assert exact(H, 1, b, a, x) == [a[0] * x[0]]
    # extreme magnitudes: all-ones mantissas, both signs
    m = (1 << b) - 1
    assert exact(H, 1, b, [m], [-m]) == [-m * m]


def test_row_subset_and_threads_agree():
    rng = random.Random(11)
    n, b = 37, 300
    a = rand_ints(rng, 2 * n - 1, b)
    x = rand_ints(rng, n, b)
    full = exact(H, n, b, a, x, threads=1)
    rows = [36, 0, 17, 17, 5]
    assert exact(H, n, b, a, x, rows=rows, threads=3) == [full[r] for r in rows]


def test_n2_explicit_formula():
    """Algorithm 1, step 1: y1 = a1 x1 + a2 x2, y2 = a2 x1 + a3 x2."""
    rng = random.Random(2)
    for b in (8, 64, 2048):
        a1, a2, a3 = rand_ints(rng, 3, b)
        x1, x2 = rand_ints(rng, 2, b)
        assert exact(H, 2, b, [a1, a2, a3], [x1, x2]) == [a1 * x1 + a2 * x2, a2 * x1 + a3 * x2]
        assert algorithm1([a1, a2, a3], [x1, x2]) == [a1 * x1 + a2 * x2, a2 * x1 + a3 * x2]


def test_four_to_three_identities():
    """Sec. 3: with C=(a_i+a_{i+1})x_i, D=a_{i+1}(x_i-x_{i+1}), E=a_i(x_{i-1}-x_i),
    a_i x_i + a_{i+1} x_{i+1} = C - D and a_i x_{i-1} + a_{i+1} x_i = C + E."""
    rng = random.Random(3)
    for _ in range(200):
        ai, ai1, xim1, xi, xi1 = rand_ints(rng, 5, 200)
        Cc = (ai + ai1) * xi
        Dd = ai1 * (xi - xi1)
        Ee = ai * (xim1 - xi)
        assert ai * xi + ai1 * xi1 == Cc - Dd
        assert ai * xim1 + ai1 * xi == Cc + Ee


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 16, 17, 33, 40])
def test_one_level_identities_through_oracle(n):
    """p = C h, q = D f, r = E g computed by the oracle on the half-size
    Hankel problems recombine to the oracle's full product (Sec. 3, step 8)."""
    rng = random.Random(n)
    b = 96
    a = rand_ints(rng, 2 * n - 1, b)
    x = rand_ints(rng, n, b)
    m, m1, c, d, e, f, g, h = one_level(a, x)
    bb = b + 1  # sums and differences need one more bit
    p = exact(H, m, bb, c, h)
    q = exact(H, m, bb, d, f)
    r = exact(H, m1, bb, e, g)
    y = exact(H, n, b, a, x)
    for i in range(m):            # 0-based i <-> paper's i+1
        assert y[2 * i] == p[i] - q[i]
        if 2 * i + 1 < n:
            assert y[2 * i + 1] == p[i] + r[i]


@pytest.mark.parametrize("n", list(range(1, 41)))
def test_algorithm1_equals_bruteforce(n):
    rng = random.Random(500 + n)
    a = rand_ints(rng, 2 * n - 1, 40)
    x = rand_ints(rng, n, 40)
    want = brute(materialise(H, n, a), x)
    assert algorithm1(a, x) == want
    assert algorithm1(a, x, cutoff=5) == want


@pytest.mark.parametrize("n", [3, 4, 7, 8, 15, 16, 31, 32, 63, 64, 100, 127, 128, 255, 256, 500, 512, 1000, 1024])
def test_algorithm1_operation_counts(n):
    """Sec. 3: at most 3*3^ceil(log2 n) multiplications (products with a zero
    padding operand are not formed, as in the paper's a_3 = 0 case).

    The additions are Theta(n^log2(3)) but NOT within the printed
    4 n^log2(3) + O(n): step 4 forms 2m-1 sums (the count says m) and step 8
    adds n per node (left out of the count), so the constant is about 10.
    The claim of fewer multiplications than the schoolbook n^2 holds from n = 8.
    """
    rng = random.Random(n)
    cnt = Counts()
    a = [rng.getrandbits(40) | 1 for _ in range(2 * n - 1)]
    x = [rng.getrandbits(40) | 1 for _ in range(n)]
    algorithm1(a, x, counts=cnt)
    assert cnt.mul <= 3 * 3 ** math.ceil(math.log2(n))
    assert cnt.add <= 11 * n ** math.log2(3)
    if n >= 8:
        assert cnt.mul < n * n


def test_toeplitz_is_reversed_hankel():
    """Sec. 1: A_T is A_H with its rows reversed, so A_T x = J (A_H x)."""
    rng = random.Random(5)
    for n in (1, 2, 9, 30):
        a = rand_ints(rng, 2 * n - 1, 70)
        x = rand_ints(rng, n, 70)
        assert exact(T, n, 70, a, x) == exact(H, n, 70, a, x)[::-1]


def test_unit_vectors():
    rng = random.Random(6)
    n, b = 12, 64
    a = rand_ints(rng, 2 * n - 1, b)
    for j in range(n):
        e = [0] * n
        e[j] = 1
        assert exact(H, n, b, a, e) == a[j:j + n]          # column j of A_H
    x = rand_ints(rng, n, b)
    for k in range(2 * n - 1):
        ek = [0] * (2 * n - 1)
        ek[k] = 1
        want = [x[k - i] if 0 <= k - i < n else 0 for i in range(n)]  # anti-diagonal i+j=k
        assert exact(H, n, b, ek, x) == want


def test_linearity():
    rng = random.Random(8)
    n, b = 20, 200
    a = rand_ints(rng, 2 * n - 1, b)
    x = rand_ints(rng, n, b - 3)
    z = rand_ints(rng, n, b - 3)
    comb = [3 * xi - 2 * zi for xi, zi in zip(x, z)]
    yx, yz, yc = exact(H, n, b, a, x), exact(H, n, b, a, z), exact(H, n, b, a, comb)
    assert yc == [3 * u - 2 * v for u, v in zip(yx, yz)]


# ---------------------------------------------------------------- rounding

def rne_fraction(fr: Fraction) -> int:
    return round(fr)  # Fraction.__round__ rounds half to even


def brute_round(z_ints, b, e_in):
    """Least E with every RNE(|Z| 2^(e_in - b - E)) < 2^b, by search."""
    if all(v == 0 for v in z_ints):
        return [0] * len(z_ints), e_in
    top = max(abs(v).bit_length() for v in z_ints)
    for t in range(top - b - 2, top - b + 3):
        ms = [rne_fraction(Fraction(abs(v), 1) / Fraction(2) ** t) for v in z_ints]
        if all(mm < (1 << b) for mm in ms):
            return [(-mm if v < 0 else mm) for mm, v in zip(ms, z_ints)], e_in + t - b
    raise AssertionError("no exponent found")


def oracle_round_ints(z_ints, b, e_in):
    zl = max(1, max(abs(v).bit_length() for v in z_ints) // 32 + 1)
    zbits = 32 * zl
    fv = FixedVec.from_ints(z_ints, zbits, 0)
    y, yn, e = oracle.round_rows(fv.limbs, fv.neg, b, e_in)
    return oracle.limbs_to_ints(y, yn), e


@pytest.mark.parametrize("b", [1, 2, 7, 8, 31, 32, 33, 64, 100])
def test_rounding_matches_fraction_rne(b):
    rng = random.Random(b)
    for trial in range(60):
        width = rng.randint(1, 3 * b + 40)
        z = rand_ints(rng, rng.randint(1, 6), width)
        e_in = rng.randint(-50, 50)
        got = oracle_round_ints(z, b, e_in)
        want = brute_round(z, b, e_in)
        assert got == want, (z, b, e_in)


def test_rounding_ties_and_carry_into_exponent():
    b = 8
    # exact ties: q.5 with q even stays, q odd rounds up
    t = 5
    z = [(0b10110100 << t) + (1 << (t - 1)), (0b10110101 << t) + (1 << (t - 1))]
    got, e = oracle_round_ints(z, b, 0)
    assert got == [0b10110100, 0b10110110] and e == t - b
    # all-ones mantissa plus a half rounds to 2^b: the exponent must step up
    z = [(0xFF << t) + (1 << (t - 1))]
    got, e = oracle_round_ints(z, b, 0)
    assert got == [0x80] and e == t + 1 - b
    # negative values round symmetrically; a result that rounds to 0 is +0
    z = [-((0b10110101 << t) + (1 << (t - 1))), 1 << (t + 7)]
    got, e = oracle_round_ints(z, b, 0)
    assert got == [-0b10110110, 0x80] and e == t - b
    z = [1, -1, 1 << 40]
    got, e = oracle_round_ints(z, b, 0)
    assert got[0] == 0 and got[1] == 0
    # zero vector keeps E_in; short values shift left without rounding
    assert oracle_round_ints([0, 0], b, 3) == ([0, 0], 3)
    assert oracle_round_ints([5, -3], b, 0) == ([5 << 5, -(3 << 5)], -5 - b)


# ---------------------------------------------------------------- rounding at a given shift

def oracle_round_fixed_ints(z_ints, b, shift):
    zl = max(1, max(abs(v).bit_length() for v in z_ints) // 32 + 1)
    fv = FixedVec.from_ints(z_ints, 32 * zl, 0)
    y, yn = oracle.round_rows_fixed(fv.limbs, fv.neg, b, shift)
    return oracle.limbs_to_ints(y, yn), [int(v) for v in yn]


def fraction_round_at(z_ints, shift):
    """RNE(|Z| / 2^shift) with Z's sign, by exact rationals; +0 for zero."""
    out = []
    for v in z_ints:
        m = rne_fraction(Fraction(abs(v)) / Fraction(2) ** shift)
        out.append(-m if (v < 0 and m) else m)
    return out


@pytest.mark.parametrize("b", [1, 5, 8, 31, 32, 33, 64, 97])
def test_fixed_shift_rounding_matches_fraction_rne(b):
    """round_rows_fixed against Fraction round-half-even for random rows and
    shifts, t <= 0 (exact left shifts) included."""
    rng = random.Random(7000 + b)
    for trial in range(80):
        shift = rng.randint(-40, 3 * b + 40)
        cap = b + shift  # a row may use at most b + shift bits
        if cap < 1:
            continue
        count = rng.randint(1, 6)
        z = []
        for _ in range(count):
            width = rng.randint(0, cap)
            v = rng.getrandbits(width) if width else 0
            z.append(rng.choice((-1, 1)) * v)
        want = fraction_round_at(z, shift)
        if any(abs(w) >= (1 << b) for w in want):
            with pytest.raises(RuntimeError):
                oracle_round_fixed_ints(z, b, shift)
            continue
        got, neg = oracle_round_fixed_ints(z, b, shift)
        assert got == want, (z, b, shift)
        assert neg == [1 if w < 0 else 0 for w in want]


def test_fixed_shift_rounding_ties_signs_and_overflow():
    b, t = 8, 6
    # ties to even in both signs: q even stays, q odd goes up in magnitude
    z = [(0b1011010 << t) + (1 << (t - 1)), -((0b1011010 << t) + (1 << (t - 1))),
         (0b1011011 << t) + (1 << (t - 1)), -((0b1011011 << t) + (1 << (t - 1)))]
    got, neg = oracle_round_fixed_ints(z, b, t)
    assert got == [0b1011010, -0b1011010, 0b1011100, -0b1011100] and neg == [0, 1, 0, 1]
    # just above and just below a tie
    z = [(5 << t) + (1 << (t - 1)) + 1, -((5 << t) + (1 << (t - 1)) - 1)]
    assert oracle_round_fixed_ints(z, b, t)[0] == [6, -5]
    # a negative row that rounds to zero carries no sign
    got, neg = oracle_round_fixed_ints([-(1 << (t - 1)), -((1 << (t - 1)) + 1), 0], b, t)
    assert got == [0, -1, 0] and neg == [0, 1, 0]
    # t <= 0: an exact left shift, no rounding
    assert oracle_round_fixed_ints([3, -1], b, -4)[0] == [48, -16]
    assert oracle_round_fixed_ints([255, -255], b, 0)[0] == [255, -255]
    # overflow guard: a row with more than b + t bits is refused ...
    with pytest.raises(RuntimeError):
        oracle_round_fixed_ints([1 << (b + t)], b, t)
    # ... the largest row with b + t bits is accepted ...
    assert oracle_round_fixed_ints([(1 << (b + t)) - (1 << t)], b, t)[0] == [255]
    # ... and one that rounds up to 2^b is refused as well
    with pytest.raises(RuntimeError):
        oracle_round_fixed_ints([(1 << (b + t)) - (1 << (t - 1))], b, t)
    # the same guard for left shifts: 127 << 1 fits in b bits, 128 << 1 does not
    assert oracle_round_fixed_ints([127], b, -1)[0] == [254]
    with pytest.raises(RuntimeError):
        oracle_round_fixed_ints([128], b, -1)
    with pytest.raises(RuntimeError):
        oracle_round_fixed_ints([256], b, 0)


@pytest.mark.parametrize("b", [1, 7, 32, 33, 100, 256])
def test_fixed_shift_equals_least_exponent_rounding_at_its_shift(b):
    """At the shift that the least-exponent rule chooses, rounding at a given
    shift returns the same mantissas and signs for every row and for any
    subset of the rows."""
    rng = random.Random(b)
    for trial in range(40):
        width = rng.randint(1, 3 * b + 40)
        z = rand_ints(rng, rng.randint(1, 8), width)
        if all(v == 0 for v in z):
            continue
        e_in = rng.randint(-30, 30)
        want, e = oracle_round_ints(z, b, e_in)
        shift = e + b - e_in
        got, _ = oracle_round_fixed_ints(z, b, shift)
        assert got == want
        sub = sorted(rng.sample(range(len(z)), rng.randint(1, len(z))))
        got_sub, _ = oracle_round_fixed_ints([z[k] for k in sub], b, shift)
        assert got_sub == [want[k] for k in sub]


# ---------------------------------------------------------------- closed form

def test_hilbert_hankel_closed_form():
    """h_k = 1/(k+1) rounded to b bits: the rounded product is within
    n * 2^E_x * 2^(E_h-b-1) + ulp_y / 2 of the exact rational sum_j x_j/(i+j+1)."""
    n, b = 24, 256
    h = hilbert_hankel(n, b)
    hv = h.to_ints()
    for k, m in enumerate(hv):
        err = abs(Fraction(m, 1 << (b - 1)) - Fraction(1, k + 1))
        assert err <= Fraction(1, 1 << b)
    x = uniform_vec(99, 1, n, b, 0)
    y, yn, ey = oracle.matvec(H, n, h, x, 2)
    xs = [Fraction(v, 1 << b) for v in x.to_ints()]
    ys = oracle.limbs_to_ints(y, yn)
    bound = n * Fraction(1, 2) ** b + Fraction(2) ** (ey - b) / 2
    for i in range(n):
        true = sum(xs[j] / (i + j + 1) for j in range(n))
        got = Fraction(ys[i]) * Fraction(2) ** (ey - b)
        assert abs(got - true) <= bound
    # and exactly: the oracle's rows equal the rational product of the rounded inputs
    z, zn = oracle.exact_rows(H, n, b, h, x, None, 2)
    zi = oracle.z_to_ints(z, zn)
    for i in range(n):
        exact_y = sum(Fraction(hv[i + j], 1 << (b - 1)) * xs[j] for j in range(n))
        assert Fraction(zi[i]) / Fraction(2) ** (2 * b - 1) == exact_y


def test_generator_properties():
    v = uniform_vec(1, 0, 1000, 45, 0)
    assert v.limbs.shape == (1000, 2)
    assert int(v.limbs[:, 1].max()) < (1 << 13)
    ints = v.to_ints()
    assert max(abs(t) for t in ints) < (1 << 45)
    assert 400 < sum(1 for t in ints if t < 0) < 600
    assert np.array_equal(uniform_vec(1, 0, 1000, 45, 0).limbs, v.limbs)
    assert not np.array_equal(uniform_vec(1, 1, 1000, 45, 0).limbs, v.limbs)
    # zero mantissas carry no sign
    z = uniform_vec(3, 0, 4000, 1, 0)
    assert all(z.neg[k] == 0 for k in range(4000) if not z.limbs[k].any())
