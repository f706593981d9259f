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
