"""Host arithmetic of the Lanczos driver: the rounding of alpha and beta from
exact integer ratios (leading-bits quotient with an exact fallback) against
the oracle's rounding of the same rationals."""
import random
from fractions import Fraction

import pytest

from oracle import lanczos as ol
from paper_1402_5287_gb300 import lanczos as lz


def _cases(seed, count):
    r = random.Random(seed)
    for it in range(count):
        b = r.choice([2, 3, 5, 8, 33, 64, 100, 300])
        n = r.getrandbits(r.randint(1, 3 * b + 200)) + 1
        d = r.getrandbits(r.randint(1, 3 * b + 200)) + 1
        if it % 3 == 0:  # exact ties at b bits (odd b+1-bit quotients) and their neighbours
            q = r.getrandbits(b + 1) | 1 | (1 << b)
            d = r.getrandbits(r.randint(1, 2 * b + 150)) | 1
            n = q * d << r.randint(0, 5)
            if it % 2:
                n += r.choice([-1, 1])
        sign = r.choice([1, -1])
        yield sign * n, r.choice([1, -1]) * d, r.randint(-50, 50), b


@pytest.mark.parametrize("seed", [0, 1])
def test_round_ratio_matches_rational_rounding(seed):
    for num, den, shift, b in _cases(seed, 3000):
        m, e = lz.round_ratio(num, den, shift, b)
        assert (m, e) == ol.round_rational(Fraction(num, den) * Fraction(2) ** shift, b), (num, den, shift, b)


def test_fast_quotient_decides_generic_ratios():
    """Away from ties the leading-bits quotient decides by itself and agrees
    with the exact division; at exact ties it defers."""
    r = random.Random(7)
    for _ in range(500):
        b = r.choice([8, 64, 1000])
        n, d = r.getrandbits(2 * b + 40) | 1, r.getrandbits(2 * b) | 1
        f = lz._round_ratio_fast(n, d, b)
        assert f is not None and f == lz._round_ratio_exact(n, d, b)
    q = (1 << 64) | 1  # 65-bit odd quotient: the 64-bit rounding is a tie
    assert lz._round_ratio_fast(q * 12345, 12345, 64) is None


def test_round_ratio_full_width():
    """b = 33220 with dot-sized operands (2b + 13 bits), as in the step."""
    r = random.Random(11)
    b = 33220
    num, den = r.getrandbits(2 * b + 43), r.getrandbits(2 * b + 13) | 1
    assert lz.round_ratio(num, den, -3, b) == ol.round_rational(Fraction(num, den) / 8, b)


def test_round_ratio_zero_and_errors():
    assert lz.round_ratio(0, 5, 3, 16) == (0, 0)
    with pytest.raises(ZeroDivisionError):
        lz.round_ratio(1, 0, 0, 16)
