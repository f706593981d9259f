"""The tensor-core leaf kernel's failure path: bounded waits -> HMV_ETIMEOUT.

No fault is provoked.  Through the library's test hook, one epilogue warp
holds back one release of an accumulator, so an MMA-issuing thread's bounded
wait for it runs out (with a 20 ms limit).  The kernel then records the
timeout, lets its own MMAs and its TMA loads in flight complete, frees its
tensor memory and returns.  The call must return HMV_ETIMEOUT without
writing y, and the next product on the same plan must be exact again.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec
from test_gpu_parity import THREADS, assert_same

pytestmark = pytest.mark.gpu

ETIMEOUT = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()
    yield
    hmv.arm_leaf_stall(0)


@pytest.mark.parametrize("n,b,levels,flags", [
    (200, 2048, 0, hmv.FLAG_TILE256),   # one MMA issuer, 256-digit tiles
    (200, 2048, 0, hmv.FLAG_TILE128),   # two MMA issuers, 128-digit tiles
    (600, 1024, 2, hmv.FLAG_TILE128),   # several leaves and CTAs
    (300, 4096, -1, hmv.FLAG_DIGIT_TOOM4),  # a split plan: seven products in one leaf launch
])
def test_leaf_timeout_is_reported_and_the_plan_recovers(n, b, levels, flags):
    torch = pytest.importorskip("torch")
    h = uniform_vec(8100 + n, 0, 2 * n - 1, b, 1)
    x = uniform_vec(8100 + n, 1, n, b, 0)
    zl, zn, e = oracle.matvec(oracle.HANKEL, n, h, x, THREADS)
    want = FixedVec(zl, zn, b, e)
    method = hmv.AUTO if levels < 0 else hmv.KARATSUBA
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    with hmv.Plan(n, b, method=method, levels=levels, flags=flags, stream=stream.cuda_stream) as p:
        p.load_matrix(h)
        with torch.cuda.stream(stream):
            xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
            xn = torch.from_numpy(x.neg).to(dev)
            yl = torch.full_like(xl, -1)
            yn = torch.full_like(xn, 7)
        stream.synchronize()
        # device buffers: the failed call leaves y as it was
        hmv.arm_leaf_stall(1, 20_000_000)
        t0 = time.perf_counter()
        with pytest.raises(hmv.HmvError) as ei:
            p.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
        waited = time.perf_counter() - t0
        assert ei.value.status == ETIMEOUT
        assert waited < 1.5, f"the abort took {waited:.2f} s"  # the hook's limit, not the 2 s default
        stream.synchronize()
        assert (yl.cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all() and (yn.cpu().numpy() == 7).all()
        # host buffers: the same through the synchronous path
        hmv.arm_leaf_stall(1, 20_000_000)
        with pytest.raises(hmv.HmvError) as ei:
            p.matvec(x)
        assert ei.value.status == ETIMEOUT
        # the hook is spent: the same plan gives the exact product again, twice
        assert_same(p.matvec(x), want)
        e2 = p.matvec_device(xl.data_ptr(), xn.data_ptr(), x.exponent, yl.data_ptr(), yn.data_ptr())
        stream.synchronize()
        got = FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), b, e2)
        assert_same(got, want)

