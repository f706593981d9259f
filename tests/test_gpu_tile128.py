"""Leaf tiles 128 product digits wide (HMV_FLAG_TILE128): bit-exact parity
with the oracle on every row, alone and under the digit split, and equality
with the 256-wide tiles in every entry point (single plan, batch, many)."""
import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec, workload

from test_gpu_parity import assert_same, oracle_matvec, sampled_parity

pytestmark = pytest.mark.gpu

T128 = hmv.FLAG_TILE128


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def run(n, b, h, x, flags=0, kind=hmv.HANKEL, method=hmv.KARATSUBA, levels=-1, nrhs=1):
    with hmv.Plan(n, b, kind=kind, method=method, levels=levels, flags=flags, nrhs=nrhs) as p:
        p.load_matrix(h)
        return p.matvec(x), p.stats()


# sizes: one tile, several tiles with a ragged tail in both dimensions, the
# narrowest digit counts (b = 1, 33) and digit counts just past a tile edge
# (1, 64, 0): one j-step per tile, so the second MMA issuer has none;
# (17, 64, 0): 17 j-steps, 2 windows of the first issuer against 1 of the second;
# (70, 2140, 1) and (90, 4178, 2): 268 and 523 digits, where tiles' last
# s-blocks of one and of two K groups ride on the block below (j-steps of 9
# and 10 MMAs); (64, 2048, 1) and (45, 4100, 2) have only the one-group kind
@pytest.mark.parametrize("n,b,levels", [(64, 2048, 1), (129, 1000, 2), (7, 33, 0), (30, 1, 0), (200, 520, 3),
                                        (1, 64, 0), (17, 64, 0), (45, 4100, 2), (300, 264, -1), (70, 2140, 1),
                                        (90, 4178, 2)])
def test_tile128_all_rows(n, b, levels):
    h = uniform_vec(80 + n, 0, 2 * n - 1, b, 2)
    x = uniform_vec(80 + n, 1, n, b, -3)
    y, st = run(n, b, h, x, flags=T128, levels=levels)
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))
    y256, _ = run(n, b, h, x, levels=levels)
    assert_same(y, y256)


@pytest.mark.parametrize("kind", [hmv.TOEPLITZ, hmv.CIRCULANT])
def test_tile128_toeplitz_circulant(kind):
    n, b = 110, 900
    hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
    h = uniform_vec(91, 0, hlen, b)
    x = uniform_vec(91, 1, n, b)
    ok = oracle.TOEPLITZ if kind == hmv.TOEPLITZ else oracle.CIRCULANT
    y, _ = run(n, b, h, x, flags=T128, kind=kind, levels=2)
    assert_same(y, oracle_matvec(ok, n, h, x))


def test_tile128_block_rhs():
    n, b, k = 50, 700, 3
    h = uniform_vec(93, 0, 2 * n - 1, b)
    x = uniform_vec(93, 1, n * k, b)
    y, _ = run(n, b, h, x, flags=T128, nrhs=k, levels=1)
    y256, _ = run(n, b, h, x, nrhs=k, levels=1)
    assert_same(y, y256)


@pytest.mark.parametrize("b", [2046, 2140])
def test_tile128_worst_case_digits(b):
    """All-(-128) balanced digits: every product +2^14, full windows 2^24
    (b = 2140: 268 digits, windows of 9- and 10-MMA j-steps)."""
    n = 80
    m = int("80" * ((b + 7) // 8), 16) & ((1 << b) - 1)
    h = FixedVec.from_ints([-m] * (2 * n - 1), b, 0)
    x = FixedVec.from_ints([-m] * n, b, 0)
    want = oracle_matvec(oracle.HANKEL, n, h, x)
    assert_same(run(n, b, h, x, flags=T128, levels=0)[0], want)
    assert_same(run(n, b, h, x, flags=T128, levels=2)[0], want)


@pytest.mark.parametrize("split", [hmv.FLAG_DIGIT_SPLIT1, hmv.FLAG_DIGIT_SPLIT2, hmv.FLAG_DIGIT_TOOM4,
                                   hmv.FLAG_DIGIT_TOOM6, hmv.FLAG_DIGIT_TOOM8])
def test_tile128_under_digit_split(split):
    n, b = 100, 4100
    h = uniform_vec(95, 0, 2 * n - 1, b, 1)
    x = uniform_vec(95, 1, n, b, -1)
    y, _ = run(n, b, h, x, flags=T128 | split, method=hmv.AUTO)
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


def test_tile128_batch_and_many_mixed_widths():
    problems = [dict(n=40, b=1500, nrhs=2), dict(n=90, b=600, nrhs=1, flags=T128),
                dict(n=33, b=2100, nrhs=1, flags=T128, kind=hmv.TOEPLITZ), dict(n=20, b=300, nrhs=1)]
    hs, xs = [], []
    for i, pr in enumerate(problems):
        hs.append(uniform_vec(97 + i, 0, 2 * pr["n"] - 1, pr["b"]))
        xs.append(uniform_vec(97 + i, 1, pr["n"] * pr["nrhs"], pr["b"]))
    with hmv.Batch(problems) as bt:
        for i, h in enumerate(hs):
            bt.load_matrix(i, h)
        ys = bt.matvec(xs)
    for pr, h, x, y in zip(problems, hs, xs, ys):
        want, _ = run(pr["n"], pr["b"], h, x, kind=pr.get("kind", hmv.HANKEL), nrhs=pr["nrhs"])
        assert_same(y, want)
    # hmv_matvec_many: one product per plan, the two widths in one step
    import torch
    dev = torch.device("cuda", 0)
    plans, xp, yp, keep, exps = [], [], [], [], []
    singles = [pr for pr in problems if pr["nrhs"] == 1]
    for i, pr in enumerate(problems):
        if pr["nrhs"] != 1:
            continue
        p = hmv.Plan(pr["n"], pr["b"], kind=pr.get("kind", hmv.HANKEL), method=hmv.KARATSUBA,
                     flags=pr.get("flags", 0))
        p.load_matrix(hs[i])
        xl = torch.from_numpy(xs[i].limbs.view(np.int32)).to(dev)
        xn = torch.from_numpy(xs[i].neg).to(dev)
        yl, yn = torch.empty_like(xl), torch.empty_like(xn)
        keep.append((i, xl, xn, yl, yn))
        plans.append(p)
        xp.append((xl.data_ptr(), xn.data_ptr()))
        yp.append((yl.data_ptr(), yn.data_ptr()))
        exps.append(xs[i].exponent)
    out = hmv.matvec_many_device(plans, xp, yp, exps)
    torch.cuda.synchronize()
    assert len(singles) == len(plans)
    for (i, xl, xn, yl, yn), e in zip(keep, out):
        y = FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), problems[i]["b"], e)
        assert_same(y, ys[i])
    for p in plans:
        p.close()


def test_tile128_large_workload_matches_default():
    n, b, h, x = workload("large")
    y0, st0 = run(n, b, h, x, flags=hmv.FLAG_TILE256, method=hmv.AUTO)
    y, st = run(n, b, h, x, flags=T128, method=hmv.AUTO)
    assert st0["leaf_tile_digits"] == 256 and st["leaf_tile_digits"] == 128
    assert_same(y, y0)
    sampled_parity(oracle.HANKEL, n, h, x, y, 3, 11)


@pytest.mark.parametrize("n,b,levels,want", [(300, 256, -1, 128), (300, 64, -1, 128), (200, 4096, -1, 128),
                                              (120, 33220, 1, 256), (64, 33220, 0, 256)])
def test_auto_chooses_tile_width_and_stays_exact(n, b, levels, want):
    """HMV_AUTO weighs the padded product digits of each width against the
    MMA rates: 128-wide tiles (two issuing threads) for all but the widest
    unsplit products; either way the result is exact."""
    h = uniform_vec(99 + b, 0, 2 * n - 1, b, 1)
    x = uniform_vec(99 + b, 1, n, b, 2)
    y, st = run(n, b, h, x, method=hmv.AUTO, levels=levels)
    assert st["leaf_tile_digits"] == want
    assert_same(y, oracle_matvec(oracle.HANKEL, n, h, x))


def test_auto_benchmark_size_takes_toom8_on_128_wide_tiles():
    """At n = 8000, b = 33220 the cost model picks Toom-8 on 128-wide tiles; a
    caller-fixed split still gets the cost model's tile width."""
    n, b = 8000, 33220
    with hmv.Plan(n, b, method=hmv.AUTO) as p:
        st = p.stats()
    assert st["digit_products"] == 15 and st["leaf_tile_digits"] == 128
    with hmv.Plan(n, b, method=hmv.AUTO, flags=hmv.FLAG_DIGIT_TOOM6) as p:
        st = p.stats()
    assert st["digit_products"] == 11 and st["leaf_tile_digits"] == 128
