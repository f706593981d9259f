"""Parity of the CUDA library with the CPU oracle, through the C ABI.

Every comparison is bit-exact: the method is exact integer arithmetic up to
the final b-bit rounding, which both sides perform from the exact rows.
"""
import os
import random

import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, hilbert_hankel, uniform_vec, workload

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def oracle_matvec(kind, n, h, x):
    y, yn, e = oracle.matvec(kind, n, h, x, THREADS)
    return FixedVec(y, yn, h.b, e)


def assert_same(got: FixedVec, want: FixedVec):
    assert got.exponent == want.exponent
    bad = np.nonzero((got.limbs != want.limbs).any(axis=1) | (got.neg != want.neg))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:10]}"


def run(n, b, h, x, kind=hmv.HANKEL, method=hmv.AUTO, levels=-1, flags=0):
    with hmv.Plan(n, b, kind=kind, method=method, levels=levels, flags=flags) as p:
        p.load_matrix(h)
        return p.matvec(x)


def rand_vec(seed, stream, count, b, e=0):
    return uniform_vec(1000 + seed, stream, count, b, e)


# ---------------------------------------------------------------- full parity, small sizes

def test_small_workload_all_rows():
    n, b, h, x = workload("small")
    assert_same(run(n, b, h, x), oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("n,b,levels", [
    (64, 2048, 0), (64, 2048, 1), (200, 512, 2), (300, 2048, 3), (257, 700, 1),
    (130, 64, 0), (129, 1000, 1), (33, 2040, 4), (1, 64, 0), (2, 31, 1), (3, 1, 2), (17, 33, 3),
    (300, 256, 6), (400, 128, 7), (700, 40, 8)])
def test_karatsuba_levels_all_rows(n, b, levels):
    """Several 128-row tiles, ragged row and digit tails, depths 0-8 (int16
    post-pass digits through depth 6, int32 beyond)."""
    h = rand_vec(n + b, 0, 2 * n - 1, b, 1)
    x = rand_vec(n + b, 1, n, b, -2)
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=levels), oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("n,b,levels", [(70, 300, 0), (150, 1024, 2), (45, 2048, 3)])
def test_tensor_core_leaf_equals_cuda_core_leaf(n, b, levels):
    h = rand_vec(7 * n, 0, 2 * n - 1, b)
    x = rand_vec(7 * n, 1, n, b)
    simt = run(n, b, h, x, method=hmv.KARATSUBA, levels=levels, flags=hmv.FLAG_SIMT_LEAF)
    assert_same(simt, oracle_matvec(oracle.HANKEL, n, h, x))
    tc = run(n, b, h, x, method=hmv.KARATSUBA, levels=levels)
    assert_same(tc, simt)


@pytest.mark.parametrize("n,b", [(64, 2048), (37, 100), (5, 33), (100, 32)])
def test_schoolbook_all_rows(n, b):
    h = rand_vec(3 * n, 0, 2 * n - 1, b)
    x = rand_vec(3 * n, 1, n, b)
    assert_same(run(n, b, h, x, method=hmv.SCHOOLBOOK), oracle_matvec(oracle.HANKEL, n, h, x))


@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
@pytest.mark.parametrize("method,levels", [(hmv.KARATSUBA, 2), (hmv.KARATSUBA, 0), (hmv.SCHOOLBOOK, 0)])
def test_toeplitz_and_circulant(kind, method, levels):
    n, b = 90, 600
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = rand_vec(11, 0, hlen, b)
    x = rand_vec(11, 1, n, b)
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    assert_same(run(n, b, h, x, kind=kind, method=method, levels=levels), oracle_matvec(ok, n, h, x))


# ---------------------------------------------------------------- edge cases

def test_worst_case_digits_hit_the_accumulation_bound():
    """Mantissas 0x8080...80 with a minus sign are all-(-128) balanced digits:
    every product is +2^14 and a full window sums to exactly 2^24."""
    n, b = 80, 2046  # the low 255 digits are -128, the top one 0
    m = int("80" * ((b + 7) // 8), 16) & ((1 << b) - 1)
    h = FixedVec.from_ints([-m] * (2 * n - 1), b, 0)
    x = FixedVec.from_ints([-m] * n, b, 0)
    want = oracle_matvec(oracle.HANKEL, n, h, x)
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=0), want)
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=2), want)
    # all-ones mantissas with mixed signs
    mm = (1 << b) - 1
    h = FixedVec.from_ints([mm if k % 3 else -mm for k in range(2 * n - 1)], b, 0)
    x = FixedVec.from_ints([-mm if j % 2 else mm for j in range(n)], b, 0)
    want = oracle_matvec(oracle.HANKEL, n, h, x)
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=1), want)
    # the deepest recursion whose post-pass digits are int16, and one past it
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=6), want)
    assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=7), want)


def test_zero_and_unit_vectors():
    n, b = 50, 256
    h = rand_vec(5, 0, 2 * n - 1, b, 2)
    z = FixedVec.from_ints([0] * n, b, 3)
    y = run(n, b, h, z, levels=1)
    assert y.exponent == 5 and not y.limbs.any() and not y.neg.any()
    for j in (0, 17, n - 1):
        e = FixedVec.from_ints([1 if k == j else 0 for k in range(n)], b, 0)
        assert_same(run(n, b, h, e, levels=2), oracle_matvec(oracle.HANKEL, n, h, e))
    # single non-zero matrix entry: an anti-diagonal selection of x
    hk = FixedVec.from_ints([(1 << (b - 1)) if k == 40 else 0 for k in range(2 * n - 1)], b, 0)
    x = rand_vec(6, 1, n, b)
    assert_same(run(n, b, hk, x, levels=2), oracle_matvec(oracle.HANKEL, n, hk, x))


def test_negative_zero_inputs_are_zero():
    n, b = 8, 40
    h = rand_vec(9, 0, 2 * n - 1, b)
    x = FixedVec.from_ints([0] * n, b, 0)
    x.neg[:] = 1  # -0 everywhere
    y = run(n, b, h, x, levels=1)
    assert not y.limbs.any() and not y.neg.any()


def test_deterministic_and_plan_reuse():
    n, b = 120, 1500
    h = rand_vec(21, 0, 2 * n - 1, b)
    xs = [rand_vec(21 + k, 1, n, b) for k in range(3)]
    with hmv.Plan(n, b, levels=2) as p:
        p.load_matrix(h)
        outs = [p.matvec(x) for x in xs]
        again = p.matvec(xs[0])
    for x, y in zip(xs, outs):
        assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))
    assert_same(again, outs[0])


def test_block_rhs_shares_one_exponent():
    n, b, k = 40, 300, 3
    h = rand_vec(31, 0, 2 * n - 1, b)
    parts = [rand_vec(31 + r, 1, n, b) for r in range(k)]
    parts[1] = FixedVec(parts[1].limbs.copy(), parts[1].neg, b, 0)
    parts[1].limbs[:, -1] >>= 5  # a smaller vector in the block
    X = FixedVec(np.concatenate([p.limbs for p in parts]), np.concatenate([p.neg for p in parts]), b, 0)
    with hmv.Plan(n, b, levels=1, nrhs=k) as p:
        p.load_matrix(h)
        Y = p.matvec(X)
    zs = [oracle.exact_rows(oracle.HANKEL, n, b, h, part, None, THREADS) for part in parts]
    z = np.concatenate([zz[0] for zz in zs])
    zn = np.concatenate([zz[1] for zz in zs])
    yl, yn, e = oracle.round_rows(z, zn, b, h.exponent)
    assert_same(Y, FixedVec(yl, yn, b, e))


@pytest.mark.parametrize("n,b,flags", [(300, 4096, 0), (257, 2048, hmv.FLAG_DIGIT_TOOM4)])
def test_block_of_eight_rhs_all_rows(n, b, flags):
    """A block of eight right-hand sides (block Lanczos) on the cost model's
    plan: every row of every vector against the oracle, one shared exponent."""
    k = 8
    h = rand_vec(61 + n, 0, 2 * n - 1, b)
    parts = [rand_vec(61 + n + r, 1, n, b) for r in range(k)]
    X = FixedVec(np.concatenate([p.limbs for p in parts]), np.concatenate([p.neg for p in parts]), b, 0)
    with hmv.Plan(n, b, nrhs=k, flags=flags) as p:
        p.load_matrix(h)
        Y = p.matvec(X)
    zs = [oracle.exact_rows(oracle.HANKEL, n, b, h, part, None, THREADS) for part in parts]
    yl, yn, e = oracle.round_rows(np.concatenate([zz[0] for zz in zs]), np.concatenate([zz[1] for zz in zs]),
                                  b, h.exponent)
    assert_same(Y, FixedVec(yl, yn, b, e))


def test_invalid_inputs_are_rejected():
    n, b = 10, 70
    h = rand_vec(41, 0, 2 * n - 1, b)
    x = rand_vec(41, 1, n, b)
    with hmv.Plan(n, b, levels=1) as p:
        with pytest.raises(hmv.HmvError) as ei:
            p.matvec(x)
        assert ei.value.status == 5  # not loaded
        bad = FixedVec(h.limbs.copy(), h.neg, b, 0)
        bad.limbs[3, -1] |= np.uint32(1 << (b % 32))  # a bit at position b
        with pytest.raises(hmv.HmvError) as ei:
            p.load_matrix(bad)
        assert ei.value.status == 1
        p.load_matrix(h)
        badx = FixedVec(x.limbs.copy(), x.neg, b, 0)
        badx.limbs[0, -1] |= np.uint32(1 << 31)
        with pytest.raises(hmv.HmvError) as ei:
            p.matvec(badx)
        assert ei.value.status == 1
        short = FixedVec(x.limbs[:-1], x.neg[:-1], b, 0)
        with pytest.raises(hmv.HmvError):
            p.matvec(short)
        y = p.matvec(x)  # the plan still works after rejected calls
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


def test_device_pointer_api_matches_host_api():
    torch = pytest.importorskip("torch")
    n, b = 100, 900
    h = rand_vec(51, 0, 2 * n - 1, b, 1)
    x = rand_vec(51, 1, n, b, 0)
    host = run(n, b, h, x, levels=2)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        hl = torch.from_numpy(h.limbs.view(np.int32)).to(dev)
        hn = torch.from_numpy(h.neg).to(dev)
        xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(x.neg).to(dev)
        yl = torch.zeros_like(xl)
        yn = torch.zeros_like(xn)
    stream.synchronize()
    with hmv.Plan(n, b, levels=2, stream=stream.cuda_stream) as p:
        p.load_matrix_device(hl.data_ptr(), hn.data_ptr(), 2 * n - 1, h.exponent)
        e = p.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
    stream.synchronize()
    got = FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), b, e)
    assert_same(got, host)


# ---------------------------------------------------------------- full-size workloads, sampled rows

def sample_rows(n, nsample, seed, extra=(), residues=0):
    """Seeded random rows plus rows 0 and n-1, the given extra rows and, with
    residues = 2^L, at least one row of every class i mod 2^L (the output
    rows of one class take the same path through L levels of Algorithm 1)."""
    rng = random.Random(seed)
    rows = set(rng.sample(range(n), min(nsample, n))) | {0, n - 1} | set(extra)
    for r in range(min(residues, n)):
        if not any(i % residues == r for i in rows):
            rows.add(r + residues * rng.randrange((n - 1 - r) // residues + 1))
    return sorted(rows)


def sampled_parity(kind, n, h, x, y: FixedVec, nsample, seed, residues=0):
    """Bit-exact check of sampled rows, including every row that attains the
    largest output mantissa (so the exponent choice is checked too)."""
    b = h.b
    mags = [int.from_bytes(y.limbs[i].tobytes(), "little") for i in range(n)]
    top = max(mags)
    rows = sample_rows(n, nsample, seed, [i for i in range(n) if mags[i] == top][:4], residues)
    z, zn = oracle.exact_rows(kind, n, b, h, x, rows, THREADS)
    shift = y.exponent + b - (h.exponent + x.exponent)
    yl, yn = oracle.round_rows_fixed(z, zn, b, shift)
    bad = [rows[k] for k in range(len(rows)) if not (np.array_equal(yl[k], y.limbs[rows[k]]) and yn[k] == y.neg[rows[k]])]
    assert not bad, f"{len(bad)} of {len(rows)} sampled rows differ, first {bad[:10]}"
    yl2, yn2, e2 = oracle.round_rows(z, zn, b, h.exponent + x.exponent)
    assert e2 == y.exponent
    return rows


def test_hilbert_workload_all_rows():
    """n = 1024, b = 33220 (the Hilbert Hankel h_k = 1/(k+1)) on the cost
    model's plan: every row against the oracle."""
    n, b, h, x = workload("hilbert")
    with hmv.Plan(n, b) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        st = p.stats()
    assert st["digit_products"] > 1  # the cost model splits the mantissas here
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))
    # the closed form: |y_i| < sum_j |x_j|/(i+j+1) + slack <= H_n, so E_y <= 3
    assert y.exponent <= 3


def test_hilbert_methods_agree():
    n, b, h, x = workload("hilbert")
    y = run(n, b, h, x)
    for levels in (0, 2):
        assert_same(run(n, b, h, x, method=hmv.KARATSUBA, levels=levels), y)


def test_large_workload_sampled_hankel_and_toeplitz():
    """n = 8000, b = 33220 in the benchmark's configuration (cost-model depth)."""
    n, b, h, x = workload("large")
    with hmv.Plan(n, b) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        st = p.stats()
    assert st["levels"] == 6 and st["leaf_rows_max"] <= 128
    rows = sampled_parity(oracle.HANKEL, n, h, x, y, 256, 2, residues=1 << st["levels"])
    assert len(rows) >= 256 and len({i % 64 for i in rows}) == 64
    with hmv.Plan(n, b, kind=hmv.TOEPLITZ) as p:
        p.load_matrix(h)
        yt = p.matvec(x)
    assert yt.exponent == y.exponent
    assert np.array_equal(yt.limbs, y.limbs[::-1]) and np.array_equal(yt.neg, y.neg[::-1])
    sampled_parity(oracle.TOEPLITZ, n, h, x, yt, 3, 3)
