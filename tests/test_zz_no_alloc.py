"""The scratch-free entry point (hmv_schoolbook_noalloc) gives, bit for bit,
what the plan-based schoolbook product gives.

It serves callers that cannot allocate device memory while they run; it
works from the caller's buffers and one scratch array compiled into the
library.  Two calls in a row (different sizes and kinds) check that the
shared scratch carries nothing from one call into the next.  This file is
collected last so that a stop-at-first-failure run has run every other test.
"""
import numpy as np
import pytest

import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec

pytestmark = pytest.mark.gpu


def plan_schoolbook(n, b, kind, h, x):
    with hmv.Plan(n, b, kind=kind, method=hmv.SCHOOLBOOK) as p:
        p.load_matrix(h)
        return p.matvec(x)


def noalloc_call(n, b, kind, h, x, stream=None):
    """Calls the entry point on device copies of h and x with y preset to a
    fill pattern; returns (status, E_y or None, y limbs, y signs)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    hl = torch.from_numpy(h.limbs.view(np.int32)).to(dev)
    hn = torch.from_numpy(h.neg).to(dev)
    xl = torch.from_numpy(x.limbs.view(np.int32)).to(dev)
    xn = torch.from_numpy(x.neg).to(dev)
    yl = torch.full_like(xl, -1)
    yn = torch.full_like(xn, 7)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    try:
        e = hmv.schoolbook_noalloc(n, b, kind, (hl.data_ptr(), hn.data_ptr()), h.exponent,
                                   (xl.data_ptr(), xn.data_ptr()), x.exponent, (yl.data_ptr(), yn.data_ptr()), s)
        status = 0
    except hmv.HmvError as err:
        e, status = None, err.status
    torch.cuda.synchronize()
    return status, e, yl.cpu().numpy().view(np.uint32), yn.cpu().numpy()


def noalloc(n, b, kind, h, x):
    status, e, yl, yn = noalloc_call(n, b, kind, h, x)
    if status:
        raise hmv.HmvError(status, "hmv_schoolbook_noalloc")
    return FixedVec(yl, yn, b, e)


def same(a, b):
    return a.exponent == b.exponent and np.array_equal(a.limbs, b.limbs) and np.array_equal(a.neg, b.neg)


def test_noalloc_matches_plan_schoolbook_two_calls_in_a_row():
    pkg.build()
    cases = [(96, 2048, hmv.HANKEL, 0), (40, 700, hmv.TOEPLITZ, 1), (33, 33220, hmv.CIRCULANT, 2)]
    for n, b, kind, seed in cases:
        hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
        h = uniform_vec(500 + seed, 0, hlen, b, 1)
        x = uniform_vec(500 + seed, 1, n, b, -1)
        want = plan_schoolbook(n, b, kind, h, x)
        got = noalloc(n, b, kind, h, x)
        assert same(got, want), (n, b, kind)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    pkg.build()
    n, b = 101, 33220  # needs more than HMV_NOALLOC_SCRATCH_BYTES
    h = uniform_vec(9, 0, 2 * n - 1, b)
    x = uniform_vec(9, 1, n, b)
    with pytest.raises(hmv.HmvError) as ei:
        noalloc(n, b, hmv.HANKEL, h, x)
    assert ei.value.status == 1
    # and the entry point still works afterwards
    n, b = 12, 300
    h = uniform_vec(10, 0, 2 * n - 1, b)
    x = uniform_vec(10, 1, n, b)
    assert same(noalloc(n, b, hmv.HANKEL, h, x), plan_schoolbook(n, b, hmv.HANKEL, h, x))


def test_noalloc_rejects_bits_at_or_above_b_and_writes_nothing():
    pkg.build()
    n, b = 20, 300
    h = uniform_vec(11, 0, 2 * n - 1, b)
    x = uniform_vec(11, 1, n, b)
    bad = FixedVec(x.limbs.copy(), x.neg, b, 0)
    bad.limbs[7, -1] |= np.uint32(1 << (b % 32))  # bit b of entry 7
    status, e, yl, yn = noalloc_call(n, b, hmv.HANKEL, h, bad)
    assert status == 1 and e is None
    assert (yl == 0xFFFFFFFF).all() and (yn == 7).all()
    badh = FixedVec(h.limbs.copy(), h.neg, b, 0)
    badh.limbs[2 * n - 2, -1] |= np.uint32(1 << 31)
    status, e, yl, yn = noalloc_call(n, b, hmv.TOEPLITZ, badh, x)
    assert status == 1 and (yl == 0xFFFFFFFF).all() and (yn == 7).all()
    assert same(noalloc(n, b, hmv.HANKEL, h, x), plan_schoolbook(n, b, hmv.HANKEL, h, x))


def test_noalloc_rejects_rows_beyond_shared_memory():
    """b = 2^20 with n = 1 fits the scratch array, but one row's operands
    (8 * 32768 bytes) exceed the 227 KB of shared memory a block may use."""
    pkg.build()
    n, b = 1, 1 << 20
    h = uniform_vec(12, 0, 1, b)
    x = uniform_vec(12, 1, 1, b)
    status, e, yl, yn = noalloc_call(n, b, hmv.HANKEL, h, x)
    assert status == 1 and (yl == 0xFFFFFFFF).all() and (yn == 7).all()
