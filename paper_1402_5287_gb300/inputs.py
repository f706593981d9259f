"""Seeded synthetic inputs for the multiprecision Hankel product.

This module only draws numbers; it holds none of the product's arithmetic.
Both the CUDA path (bench, GPU tests) and the CPU oracle tests take their
inputs from here, so the two sides always see the same operands.

Number format (block fixed point, one exponent per vector):
    value_k = (-1)^neg_k * M_k * 2^(E - b),   0 <= M_k < 2^b,
with M_k stored as ceil(b/32) little-endian uint32 limbs (entry-major) and
neg_k a uint8 flag.  A zero mantissa always carries neg = 0.

Random generator: every entry e of stream t owns an xoshiro256** state
seeded by four successive splitmix64 outputs (Vigna's published
definitions) started at seed + golden * (1 + t * 2^40 + e).  Each entry
draws its sign first (top bit of the first output), then its limbs, two per
64-bit output, low limb first; bits at or above b are masked off.  Entries
are independent streams, so the draw is vectorised across entries.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GOLDEN = 0x9E3779B97F4A7C15
BASE_SEED = 14025287  # arXiv id digits; seed of workload c is BASE_SEED + c


def limbs_per_entry(b: int) -> int:
    return (b + 31) // 32


@dataclass
class FixedVec:
    """A vector of block fixed-point numbers (host arrays)."""
    limbs: np.ndarray   # uint32 [count, L32]
    neg: np.ndarray     # uint8 [count]
    b: int
    exponent: int

    @property
    def count(self) -> int:
        return int(self.neg.shape[0])

    def to_ints(self) -> list[int]:
        """Signed integer mantissas (value = int * 2^(exponent - b))."""
        out = []
        raw = np.ascontiguousarray(self.limbs, dtype="<u4")
        for k in range(self.count):
            m = int.from_bytes(raw[k].tobytes(), "little")
            out.append(-m if self.neg[k] else m)
        return out

    @staticmethod
    def from_ints(vals, b: int, exponent: int) -> "FixedVec":
        L = limbs_per_entry(b)
        limbs = np.zeros((len(vals), L), dtype=np.uint32)
        neg = np.zeros(len(vals), dtype=np.uint8)
        for k, v in enumerate(vals):
            m = abs(int(v))
            if m >> b:
                raise ValueError(f"entry {k} needs more than {b} bits")
            limbs[k] = np.frombuffer(m.to_bytes(4 * L, "little"), dtype="<u4")
            neg[k] = 1 if v < 0 else 0
        return FixedVec(limbs, neg, b, exponent)


def _rotl(x: np.ndarray, k: int) -> np.ndarray:
    return (x << np.uint64(k)) | (x >> np.uint64(64 - k))


def _splitmix_next(z: np.ndarray):
    z = z + np.uint64(GOLDEN)
    r = z
    r = (r ^ (r >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    r = (r ^ (r >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    r = r ^ (r >> np.uint64(31))
    return z, r


class _Xoshiro:
    """xoshiro256** over a vector of independent states."""

    def __init__(self, seeds: np.ndarray):
        z = seeds.astype(np.uint64)
        self.s = []
        for _ in range(4):
            z, r = _splitmix_next(z)
            self.s.append(r)

    def next(self) -> np.ndarray:
        s0, s1, s2, s3 = self.s
        res = _rotl(s1 * np.uint64(5), 7) * np.uint64(9)
        t = s1 << np.uint64(17)
        s2 = s2 ^ s0
        s3 = s3 ^ s1
        s1 = s1 ^ s2
        s0 = s0 ^ s3
        s2 = s2 ^ t
        s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return res


def uniform_vec(seed: int, stream: int, count: int, b: int, exponent: int = 0) -> FixedVec:
    """`count` entries, sign and b mantissa bits uniform: values in (-2^E, 2^E)."""
    L = limbs_per_entry(b)
    with np.errstate(over="ignore"):
        e = np.arange(count, dtype=np.uint64)
        start = (np.uint64(seed % (1 << 64))
                 + np.uint64(GOLDEN) * (np.uint64(1) + np.uint64(stream) * np.uint64(1 << 40) + e))
        g = _Xoshiro(start)
        neg = (g.next() >> np.uint64(63)).astype(np.uint8)
        limbs = np.zeros((count, L), dtype=np.uint32)
        for w in range((L + 1) // 2):
            r = g.next()
            limbs[:, 2 * w] = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            if 2 * w + 1 < L:
                limbs[:, 2 * w + 1] = (r >> np.uint64(32)).astype(np.uint32)
    top = b - 32 * (L - 1)
    if top < 32:
        limbs[:, L - 1] &= np.uint32((1 << top) - 1)
    zero = ~limbs.any(axis=1)
    neg[zero] = 0
    return FixedVec(limbs, neg, b, exponent)


def hilbert_hankel(n: int, b: int) -> FixedVec:
    """h_k = 1/(k+1), k = 0..2n-2, rounded to nearest-even at b bits, E = 1.

    With E = 1 the value is M * 2^(1-b), so M_k = RNE(2^(b-1) / (k+1)).
    """
    vals = []
    num = 1 << (b - 1)
    for k in range(2 * n - 1):
        d = k + 1
        q, r = divmod(num, d)
        if 2 * r > d or (2 * r == d and (q & 1)):
            q += 1
        vals.append(q)
    return FixedVec.from_ints(vals, b, 1)


def workload(name: str):
    """The named synthetic workloads: returns (n, b, h, x).

    small   : n=64,   b=2048,  h, x uniform in (-1, 1)
    hilbert : n=1024, b=33220, h_k = 1/(k+1) rounded (E=1), x uniform
    large   : n=8000, b=33220, h, x uniform in (-1, 1)
    """
    if name == "small":
        n, b, c = 64, 2048, 0
        h = uniform_vec(BASE_SEED + c, 0, 2 * n - 1, b, 0)
    elif name == "hilbert":
        n, b, c = 1024, 33220, 1
        h = hilbert_hankel(n, b)
    elif name == "large":
        n, b, c = 8000, 33220, 2
        h = uniform_vec(BASE_SEED + c, 0, 2 * n - 1, b, 0)
    else:
        raise KeyError(name)
    x = uniform_vec(BASE_SEED + c, 1, n, b, 0)
    return n, b, h, x


def batched_workload(count: int = 64, nrhs: int = 8):
    """The batched workload: `count` Hankel matrices with n ~ U[32, 2048] and
    b drawn from {4096, 16384, 33220}, each with a block of `nrhs`
    right-hand sides, entries uniform in (-1, 1).  Returns [(n, b, h, x)]
    with x holding the nrhs vectors one after another."""
    import random
    rng = random.Random(BASE_SEED + 3)
    probs = []
    for i in range(count):
        n = rng.randint(32, 2048)
        b = rng.choice([4096, 16384, 33220])
        h = uniform_vec(BASE_SEED + 3, 2 * i, 2 * n - 1, b, 0)
        x = uniform_vec(BASE_SEED + 3, 2 * i + 1, n * nrhs, b, 0)
        probs.append((n, b, h, x))
    return probs
