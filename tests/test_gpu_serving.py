"""Continuous batching: hmv_matvec_many equals separate products, and every
served request's result is the same alone and in any mix (exact)."""
import numpy as np
import pytest

import paper_1402_5287_gb300 as pkg
from paper_1402_5287_gb300 import hmv
from paper_1402_5287_gb300.inputs import FixedVec, uniform_vec

from test_gpu_parity import assert_same

pytestmark = pytest.mark.gpu

SPECS = [(40, 256, hmv.HANKEL), (150, 1024, hmv.TOEPLITZ), (64, 2048, hmv.HANKEL), (9, 100, hmv.CIRCULANT),
         (200, 700, hmv.HANKEL), (120, 16384, hmv.HANKEL)]


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    hmv.load_library()


def make(seed):
    out = []
    for i, (n, b, kind) in enumerate(SPECS):
        hlen = n if kind == hmv.CIRCULANT else 2 * n - 1
        out.append((n, b, kind, uniform_vec(seed + i, 0, hlen, b, 1), uniform_vec(seed + i, 1, n, b, 0)))
    return out


def test_matvec_many_equals_separate_products():
    torch = pytest.importorskip("torch")
    probs = make(300)
    stream = torch.cuda.Stream()
    plans, xs, ys, want = [], [], [], []
    for n, b, kind, h, x in probs:
        with hmv.Plan(n, b, kind=kind) as p1:
            p1.load_matrix(h)
            want.append(p1.matvec(x))
        p = hmv.Plan(n, b, kind=kind, stream=stream.cuda_stream)
        p.load_matrix(h)
        plans.append(p)
        xs.append((torch.from_numpy(x.limbs.view(np.int32)).cuda(), torch.from_numpy(x.neg).cuda()))
        ys.append((torch.zeros_like(xs[-1][0]), torch.zeros_like(xs[-1][1])))
    torch.cuda.synchronize()
    exps = hmv.matvec_many_device(plans, [(a.data_ptr(), b2.data_ptr()) for a, b2 in xs],
                                  [(a.data_ptr(), b2.data_ptr()) for a, b2 in ys], [x.exponent for *_, x in probs])
    for (n, b, kind, h, x), (yl, yn), e, w in zip(probs, ys, exps, want):
        assert_same(FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), b, e), w)
    for p in plans:
        p.close()


def chain_alone(n, b, kind, h, x, k):
    with hmv.Plan(n, b, kind=kind) as p:
        p.load_matrix(h)
        for _ in range(k):
            x = p.matvec(x)
    return x


@pytest.mark.parametrize("tight", [False, True])
def test_served_results_same_alone_and_in_the_mix(tight):
    from paper_1402_5287_gb300.serving import Request, Server
    probs = make(400)
    k = 3
    # together: all at once, so that every step carries several requests
    reqs = [Request(i, n, b, h, x, k, arrival=0.0, kind=kind) for i, (n, b, kind, h, x) in enumerate(probs)]
    sizes = [hmv.plan_bytes(n, b, kind=kind) for n, b, kind, _, _ in probs]
    # tight: the largest plan fits, all of them together do not
    budget = max(max(sizes), sum(sizes) // 2) if tight else 100 * max(sizes)
    srv = Server(memory_budget=budget)
    stats = srv.run(reqs)
    assert stats["matvecs"] == k * len(probs)
    assert stats["peak_bytes"] <= budget
    if tight:
        assert stats["peak_active"] < len(probs)  # admission waited for memory
    else:
        assert stats["mean_step_batch"] > 1.0  # products of different requests shared steps
    for r, (n, b, kind, h, x) in zip(reqs, probs):
        assert len(r.latencies) == k
        assert_same(r.result, chain_alone(n, b, kind, h, x, k))


def test_served_lanczos_drivers_equal_solo_runs():
    """Lanczos requests in the continuous-batching loop: each request's alpha,
    beta and final vector equal the same driver run alone, and the oracle's."""
    torch = pytest.importorskip("torch")
    from oracle import lanczos as ol
    from paper_1402_5287_gb300.lanczos import Lanczos
    from paper_1402_5287_gb300.serving import Request, Server
    probs = make(500)
    k = 3
    reqs = [Request(i, n, b, h, x, k, arrival=0.0, kind=kind, lanczos=True)
            for i, (n, b, kind, h, x) in enumerate(probs) if kind == hmv.HANKEL]
    sizes = [hmv.plan_bytes(r.n, r.b) for r in reqs]
    stats = Server(memory_budget=max(max(sizes), sum(sizes) // 2)).run(reqs)
    assert stats["matvecs"] == sum(len(r.alphas) for r in reqs)
    for r in reqs:
        with hmv.Plan(r.n, r.b) as p:
            p.load_matrix(r.h)
            solo = Lanczos(p, r.x0)
            a, bt = solo.run(k)
            v = solo.vector()
        assert r.alphas == a and r.betas == bt
        assert r.result.exponent == v.exponent and np.array_equal(r.result.limbs, v.limbs)
        if r.n <= 64:  # the oracle's recurrence on the smaller ones
            oa, ob, _ = ol.lanczos(r.h, r.x0, k)
            assert r.alphas == oa and r.betas == ob


@pytest.mark.parametrize("ntt_every", [1, 2])
def test_matvec_many_with_ntt_plans_equals_separate_products(ntt_every):
    """NTT plans in a step: alone (ntt_every = 1: no leaf launch at all) or
    mixed with tensor-core plans; bit-identical to separate products."""
    torch = pytest.importorskip("torch")
    probs = make(600)
    stream = torch.cuda.Stream()
    plans, xs, ys, want = [], [], [], []
    for i, (n, b, kind, h, x) in enumerate(probs):
        with hmv.Plan(n, b, kind=kind) as p1:
            p1.load_matrix(h)
            want.append(p1.matvec(x))
        method = hmv.NTT if i % ntt_every == 0 else hmv.AUTO
        p = hmv.Plan(n, b, kind=kind, method=method, stream=stream.cuda_stream)
        p.load_matrix(h)
        plans.append(p)
        xs.append((torch.from_numpy(x.limbs.view(np.int32)).cuda(), torch.from_numpy(x.neg).cuda()))
        ys.append((torch.zeros_like(xs[-1][0]), torch.zeros_like(xs[-1][1])))
    torch.cuda.synchronize()
    for _ in range(2):  # the step's buffers are reused by the next call
        exps = hmv.matvec_many_device(plans, [(a.data_ptr(), b2.data_ptr()) for a, b2 in xs],
                                      [(a.data_ptr(), b2.data_ptr()) for a, b2 in ys],
                                      [x.exponent for *_, x in probs])
        for (n, b, kind, h, x), (yl, yn), e, w in zip(probs, ys, exps, want):
            assert_same(FixedVec(yl.cpu().numpy().view(np.uint32), yn.cpu().numpy(), b, e), w)
    for p in plans:
        p.close()


def test_served_on_the_ntt_path_same_alone_and_in_the_mix():
    """The server on the exact NTT path (Lanczos and chain requests, all at
    once; every request on its own stream and runner): the same results as
    the tensor-core path run alone, with the requests' products overlapping."""
    from paper_1402_5287_gb300.lanczos import Lanczos
    from paper_1402_5287_gb300.serving import Request, Server
    probs = make(700)
    k = 3
    reqs = [Request(i, n, b, h, x, k, arrival=0.0, kind=kind, lanczos=(kind == hmv.HANKEL and i % 2 == 0))
            for i, (n, b, kind, h, x) in enumerate(probs)]
    stats = Server(memory_budget=64 << 30, method=hmv.NTT).run(reqs)
    assert stats["peak_active"] > 1 and stats["matvecs"] == sum(r.done for r in reqs)
    for r, (n, b, kind, h, x) in zip(reqs, probs):
        assert r.method == hmv.NTT
        if r.lanczos:
            with hmv.Plan(n, b, kind=kind) as p:
                p.load_matrix(h)
                solo = Lanczos(p, x)
                a, bt = solo.run(k)
            assert r.alphas == a and r.betas == bt
        else:
            assert_same(r.result, chain_alone(n, b, kind, h, x, k))


def test_ntt_server_keeps_within_a_tight_memory_budget():
    """The NTT path's independent requests are admitted within the budget (the
    largest plan fits, all of them together do not) and still give the
    results of the requests alone."""
    from paper_1402_5287_gb300.serving import Request, Server
    probs = make(800)
    k = 2
    reqs = [Request(i, n, b, h, x, k, arrival=0.0, kind=kind) for i, (n, b, kind, h, x) in enumerate(probs)]
    sizes = [hmv.plan_bytes(n, b, kind=kind, method=hmv.NTT) for n, b, kind, _, _ in probs]
    budget = max(max(sizes), sum(sizes) // 2)
    stats = Server(memory_budget=budget, method=hmv.NTT).run(reqs)
    assert stats["peak_bytes"] <= budget and stats["peak_active"] < len(probs)
    for r, (n, b, kind, h, x) in zip(reqs, probs):
        assert_same(r.result, chain_alone(n, b, kind, h, x, k))
