"""CPU replica of the NTT path's extraction (no GPU): one warp per row turns
the row's exact convolution coefficients z[t] (|z| < 2^57, after the Chinese
remainder) into Z = sum_t z[t] 2^(16 t) as ZW 32-bit limbs of |Z|, a sign and
an overflow flag.  The replica follows the kernel's schedule lane by lane:
windows of 512 positions, 16 consecutive positions a lane, a base-2^16 carry
chain per lane, the carries handed up one lane per round among the lanes that
hold positions of the row, the window's carry out into the next window, and
the two's-complement negation of a negative row; the result must be Z itself
for every input, including carries that ripple across lanes and windows."""
import random

import pytest

LANES, POS = 32, 16
WIN = LANES * POS


def chain(v, cy):
    for k in range(POS):
        s = v[k] + cy
        v[k] = s & 0xFFFF
        cy = s >> 16  # floor, as the kernel's arithmetic shift
    return cy


def extract_row(z, ZW):
    T = len(z)
    span = max(T, 2 * ZW)
    limbs = [0] * ZW
    wc = 0
    above_nonzero = above_not_ones = False
    for t0 in range(0, span, WIN):
        v = [[z[t0 + POS * l + k] if t0 + POS * l + k < T else 0 for k in range(POS)] for l in range(LANES)]
        last = min(LANES - 1, (span - 1 - t0) // POS)
        pending = [chain(v[l], wc if l == 0 else 0) for l in range(LANES)]
        out = 0
        for _ in range(LANES + 1):
            out += pending[last]
            incoming = [0 if (l == 0 or l > last) else pending[l - 1] for l in range(LANES)]
            if not any(incoming):
                break
            pending = [chain(v[l], incoming[l]) for l in range(LANES)]
        else:
            raise AssertionError("carry rounds did not settle")
        wc = out
        for l in range(LANES):
            tb = t0 + POS * l
            for k in range(POS // 2):
                limb = v[l][2 * k] | (v[l][2 * k + 1] << 16)
                li = tb // 2 + k
                if li < ZW:
                    limbs[li] = limb
                elif l <= last:
                    above_nonzero |= limb != 0
                    above_not_ones |= limb != 0xFFFFFFFF
    negative = wc == -1
    bad = wc not in (0, -1) or (above_not_ones if negative else above_nonzero)
    if negative:
        nz = [w for w in range(ZW) if limbs[w]]
        if not nz:
            bad = True
        else:
            k0 = nz[0]
            for w in range(k0, ZW):
                limbs[w] = ((~limbs[w]) + 1) & 0xFFFFFFFF if w == k0 else (~limbs[w]) & 0xFFFFFFFF
    mag = sum(x << (32 * w) for w, x in enumerate(limbs))
    return mag, negative and mag != 0, bad


def value(z):
    return sum(c << (16 * t) for t, c in enumerate(z))


def check(z, ZW):
    mag, neg, bad = extract_row(z, ZW)
    Z = value(z)
    fits = abs(Z) < (1 << (32 * ZW))
    assert bad == (not fits)
    if fits:
        assert mag == abs(Z) and neg == (Z < 0)


@pytest.mark.parametrize("seed", range(6))
def test_random_coefficients(seed):
    """Coefficients up to the two-prime bound, both signs, rows of 1 to 4
    windows (ZW chosen so that every exact row fits)."""
    rng = random.Random(seed)
    for T in (1, 33, 511, 512, 513, 1500, 2047):
        ZW = (16 * T + 64) // 32 + 2
        z = [rng.randrange(-(1 << 57) + 1, 1 << 57) for _ in range(T)]
        check(z, ZW)


def test_carry_ripples_across_lanes_and_windows():
    """Z = 2^(16 m) - 1 from z[0] = -1, z[m] = 1: every digit below m is
    0xFFFF, so a borrow runs through all of them (lanes and windows); and the
    reverse, Z = 1 - 2^(16 m), a negative row whose magnitude has the same
    run."""
    T, ZW = 2000, 1010
    for m in (1, 15, 16, 17, 511, 512, 513, 1024, 1999):
        z = [0] * T
        z[0], z[m] = -1, 1
        check(z, ZW)
        z[0], z[m] = 1, -1
        check(z, ZW)
        # the largest carries: every coefficient at the bound, one sign
        check([(1 << 57) - 1] * (m + 1) + [0] * (T - m - 1), ZW)
        check([-(1 << 57) + 1] * (m + 1) + [0] * (T - m - 1), ZW)


def test_zero_and_single_positions():
    T, ZW = 700, 360
    check([0] * T, ZW)
    for t in (0, 1, 31, 32, 511, 512, 699):
        for c in (1, -1, (1 << 57) - 1, -(1 << 57) + 1, 0xFFFF, -0x10000):
            z = [0] * T
            z[t] = c
            check(z, ZW)


def test_rows_that_do_not_fit_are_flagged():
    """|Z| >= 2^(32 ZW): the kernel reports an overflow (the limbs of the
    exact product always fit, so this only shows the check works)."""
    T, ZW = 600, 300  # 32 ZW = 9600 bits, positions up to 16 * 599 + 57
    for c in (1, -1, 1 << 40, -(1 << 40)):
        z = [0] * T
        z[T - 1] = c
        check(z, ZW)
    z = [0] * T
    z[599] = 1  # 2^9584: fits
    check(z, ZW)
    z[599] = 1 << 16  # 2^9600: does not
    check(z, ZW)
    z[599] = -(1 << 16)  # -2^9600: does not either
    check(z, ZW)
