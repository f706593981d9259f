"""Batched products (hmv_batch_*): every matrix's block of results equals the
single-plan product bit for bit, over several waves and repeated graph
replays with new right-hand sides."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu

PROBLEMS = [dict(n=33, b=4096, nrhs=2), dict(n=130, b=1000, nrhs=1, kind=hmv.TOEPLITZ),
            dict(n=70, b=2048, nrhs=3), dict(n=12, b=300, nrhs=1, kind=hmv.CIRCULANT),
            dict(n=257, b=520, nrhs=2, levels=2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def inputs(seed):
    hs, xs = [], []
    for i, pr in enumerate(PROBLEMS):
        kind = pr.get("kind", hmv.HANKEL)
        hlen = pr["n"] if kind == hmv.CIRCULANT else 2 * pr["n"] - 1
        hs.append(uniform_vec(seed + i, 0, hlen, pr["b"], i % 3))
        xs.append(uniform_vec(seed + i, 1, pr["n"] * pr["nrhs"], pr["b"], -(i % 2)))
    return hs, xs


def single(pr, h, x, stats=False):
    with hmv.Plan(pr["n"], pr["b"], kind=pr.get("kind", hmv.HANKEL), nrhs=pr["nrhs"],
                  levels=pr.get("levels", -1)) as p:
        p.load_matrix(h)
        y = p.matvec(x)
        return (y, p.stats()) if stats else y


@pytest.mark.parametrize("wave_bytes", [1 << 34, 1])
def test_batch_equals_single_plans(wave_bytes):
    hs, xs = inputs(900)
    with hmv.Batch(PROBLEMS, wave_bytes=wave_bytes) as bt:
        for i, h in enumerate(hs):
            bt.load_matrix(i, h)
        ys = bt.matvec(xs)
        info = bt.info()
        # a second call with new right-hand sides replays the same graph
        _, xs2 = inputs(901)
        ys2 = bt.matvec(xs2)
        info2 = bt.info()
    npairs = sum(pr["nrhs"] for pr in PROBLEMS)
    assert info["pairs"] == npairs and info2["graph_launches"] == 2
    widths = set()
    for pr, h, x, y, x2, y2 in zip(PROBLEMS, hs, xs, ys, xs2, ys2):
        y1, st = single(pr, h, x, stats=True)
        widths.add(st["leaf_tile_digits"])
        assert_same(y, y1)
        assert_same(y2, single(pr, h, x2))
    # one leaf launch per wave, so one tile width per wave
    assert info["waves"] == (len(widths) if wave_bytes > 1 else npairs)


def test_batch_against_oracle():
    hs, xs = inputs(950)
    with hmv.Batch(PROBLEMS[:3]) as bt:
        for i in range(3):
            bt.load_matrix(i, hs[i])
        ys = bt.matvec(xs[:3])
    for pr, h, x, y in zip(PROBLEMS[:3], hs, xs, ys):
        kind = pr.get("kind", hmv.HANKEL)
        ok = {hmv.HANKEL: oracle.HANKEL, hmv.TOEPLITZ: oracle.TOEPLITZ, hmv.CIRCULANT: oracle.CIRCULANT}[kind]
        n, k = pr["n"], pr["nrhs"]
        parts = [FixedVec(x.limbs[r * n:(r + 1) * n], x.neg[r * n:(r + 1) * n], x.b, x.exponent) for r in range(k)]
        zs = [oracle.exact_rows(ok, n, pr["b"], h, part, None, 8) for part in parts]
        yl, yn, e = oracle.round_rows(np.concatenate([z[0] for z in zs]), np.concatenate([z[1] for z in zs]),
                                      pr["b"], h.exponent + x.exponent)
        assert_same(y, FixedVec(yl, yn, pr["b"], e))


# members the cost model splits (Toom-6 at b = 33220), members with explicit
# digit-split flags, and unsplit members in one batch
SPLIT_PROBLEMS = [dict(n=32, b=33220, nrhs=2), dict(n=45, b=5000, nrhs=1, flags=hmv.FLAG_DIGIT_TOOM4),
                  dict(n=50, b=3000, nrhs=3, kind=hmv.TOEPLITZ, flags=hmv.FLAG_DIGIT_SPLIT1),
                  dict(n=33, b=4096, nrhs=2), dict(n=20, b=700, nrhs=1, kind=hmv.CIRCULANT),
                  dict(n=24, b=2000, nrhs=2, kind=hmv.CIRCULANT, flags=hmv.FLAG_DIGIT_TOOM6)]


def split_inputs(seed):
    hs, xs = [], []
    for i, pr in enumerate(SPLIT_PROBLEMS):
        kind = pr.get("kind", hmv.HANKEL)
        hlen = pr["n"] if kind == hmv.CIRCULANT else 2 * pr["n"] - 1
        hs.append(uniform_vec(seed + i, 0, hlen, pr["b"], i % 3))
        xs.append(uniform_vec(seed + i, 1, pr["n"] * pr["nrhs"], pr["b"], -(i % 2)))
    return hs, xs


def single_flags(pr, h, x):
    with hmv.Plan(pr["n"], pr["b"], kind=pr.get("kind", hmv.HANKEL), nrhs=pr["nrhs"], method=hmv.AUTO,
                  flags=pr.get("flags", 0)) as p:
        p.load_matrix(h)
        return p.matvec(x), p.stats()


def test_batch_with_digit_split_members():
    """Split members run in rounds (one per right-hand side) with one leaf
    launch per round and tile width; every result equals the member's own
    single-plan product, over two graph replays, and the oracle's."""
    hs, xs = split_inputs(970)
    with hmv.Batch(SPLIT_PROBLEMS) as bt:
        for i, h in enumerate(hs):
            bt.load_matrix(i, h)
        ys = bt.matvec(xs)
        _, xs2 = split_inputs(971)
        ys2 = bt.matvec(xs2)
        info = bt.info()
    assert info["pairs"] == sum(pr["nrhs"] for pr in SPLIT_PROBLEMS) and info["graph_launches"] == 2
    unsplit_widths, split_rounds = set(), {}
    for pr, h, x, y, x2, y2 in zip(SPLIT_PROBLEMS, hs, xs, ys, xs2, ys2):
        y1, st = single_flags(pr, h, x)
        assert_same(y, y1)
        assert_same(y2, single_flags(pr, h, x2)[0])
        if st["digit_products"] > 1:
            for r in range(pr["nrhs"]):
                split_rounds.setdefault(r, set()).add(st["leaf_tile_digits"])
        else:
            unsplit_widths.add(st["leaf_tile_digits"])
    assert split_rounds, "the batch has split members"
    assert info["waves"] == len(unsplit_widths) + sum(len(w) for w in split_rounds.values())
    # the Toom-6 member against the oracle
    pr, h, x, y = SPLIT_PROBLEMS[0], hs[0], xs[0], ys[0]
    n, k = pr["n"], pr["nrhs"]
    parts = [FixedVec(x.limbs[r * n:(r + 1) * n], x.neg[r * n:(r + 1) * n], x.b, x.exponent) for r in range(k)]
    zs = [oracle.exact_rows(oracle.HANKEL, n, pr["b"], h, part, None, 8) for part in parts]
    yl, yn, e = oracle.round_rows(np.concatenate([z[0] for z in zs]), np.concatenate([z[1] for z in zs]),
                                  pr["b"], h.exponent + x.exponent)
    assert_same(y, FixedVec(yl, yn, pr["b"], e))


@pytest.mark.parametrize("method", [hmv.AUTO, hmv.NTT])
def test_batched_workload_at_its_own_shape_sampled_rows(method):
    """The batched workload itself (64 matrices, n ~ U[32, 2048], b from
    {4096, 16384, 33220}, 8 right-hand sides each, one graph launch; every
    member on the tensor-core path, or every member on the exact NTT path):
    for every matrix, 8 seeded (right-hand side, row) pairs plus the row with
    the largest output mantissa of the block against the oracle, bit for bit,
    and the block's shared exponent from those rows."""
    import random

    from paper_1402_5287_gb300.inputs import batched_workload
    from test_gpu_parity import THREADS
    nrhs = 8
    probs = batched_workload(64, nrhs)
    bt = hmv.Batch([dict(n=n, b=b, nrhs=nrhs, method=method) for n, b, _, _ in probs], wave_bytes=48 << 30)
    try:
        for i, (_, _, h, _) in enumerate(probs):
            bt.load_matrix(i, h)
        ys = bt.matvec([x for *_, x in probs])
        info = bt.info()
    finally:
        bt.close()
    assert info["pairs"] == 64 * nrhs
    rng = random.Random(20260)
    for (n, b, h, x), y in zip(probs, ys):
        mags = [int.from_bytes(y.limbs[k].tobytes(), "little") for k in range(n * nrhs)]
        top = max(range(n * nrhs), key=lambda k: mags[k])
        picks = sorted({rng.randrange(n * nrhs) for _ in range(8)} | {top})
        for r in sorted({k // n for k in picks}):
            rows = [k % n for k in picks if k // n == r]
            xr = FixedVec(x.limbs[r * n:(r + 1) * n], x.neg[r * n:(r + 1) * n], b, x.exponent)
            z, zn = oracle.exact_rows(oracle.HANKEL, n, b, h, xr, rows, THREADS)
            shift = y.exponent + b - (h.exponent + x.exponent)
            yl, yn = oracle.round_rows_fixed(z, zn, b, shift)
            got = [r * n + i for i in rows]
            assert np.array_equal(yl, y.limbs[got]) and np.array_equal(yn, y.neg[got]), (n, b, r, rows)
            if top in got:  # the least exponent is decided by the largest row
                assert oracle.round_rows(z, zn, b, h.exponent + x.exponent)[2] == y.exponent


@pytest.mark.parametrize("ntt_members", [(0, 2), (0, 1, 2, 3, 4)])
def test_batch_with_ntt_members(ntt_members):
    """Members on the exact NTT path beside members run in waves (or all of
    them, with no leaf launch at all): each block equals its single-plan
    product bit for bit, over two replays of the graph."""
    hs, xs = inputs(970)
    # an NTT plan has no Karatsuba depth to choose
    specs = [dict({k: v for k, v in pr.items() if k != "levels"}, method=hmv.NTT) if i in ntt_members else pr
             for i, pr in enumerate(PROBLEMS)]
    with hmv.Batch(specs) as bt:
        for i, h in enumerate(hs):
            bt.load_matrix(i, h)
        ys = bt.matvec(xs)
        _, xs2 = inputs(971)
        ys2 = bt.matvec(xs2)
        info = bt.info()
    assert info["graph_launches"] == 2
    if len(ntt_members) == len(PROBLEMS):
        assert info["waves"] == 0 and info["leaf_tiles"] == 0
    for pr, h, x, y, x2, y2 in zip(PROBLEMS, hs, xs, ys, xs2, ys2):
        assert_same(y, single(pr, h, x))
        assert_same(y2, single(pr, h, x2))
