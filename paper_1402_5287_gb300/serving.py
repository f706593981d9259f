"""Continuous-batching server for Lanczos clients of the exact Hankel product.

Each request brings a matrix (its h) and a start vector and asks for a
number of steps against its device-resident A: either Lanczos steps (the
driver of paper_1402_5287_gb300/lanczos.py: the product, two exact inner
products and the exact three-term update; the request keeps the alpha and
beta sequence) or a plain chain v_{k+1} = A v_k.  The eigenvalue stage of a
Lanczos run is the client's.  The server

  * admits each request at its arrival, in order, while the device memory
    its plans need (hmv_plan_bytes, computed without allocating) fits the
    budget: a dispatcher thread starts the admission while steps run; the
    plan is created and its matrix loaded on a worker thread, on a CUDA
    stream of the request's own (so the load does not queue behind the
    running step), and the request joins the first step that starts after
    that,
  * keeps every admitted matrix resident (one plan per request),
  * on the tensor-core path runs steps: each step advances EVERY active
    request by one product with one hmv_matvec_many call, whose leaf products
    share one persistent tensor-core launch; requests that arrive during a
    step join at the next one, finished requests leave (continuous batching);
    on the exact NTT path (no leaf launch to share) every request instead
    advances on its own stream from a runner thread, the GPU interleaving the
    requests' kernels; either way finished plans are released on the worker
    thread, before any admission that follows, so that nothing waits for the
    device memory to be freed,
  * records, per product, the time from when it became ready (arrival for
    the first, the previous product's completion otherwise) to completion.

Every step is exact, so each request's results are identical whether it runs
alone or in any mix.
"""
from __future__ import annotations

import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import hmv
from .inputs import FixedVec


@dataclass
class Request:
    rid: int
    n: int
    b: int
    h: FixedVec
    x0: FixedVec
    matvecs: int
    arrival: float = 0.0
    kind: int = hmv.HANKEL
    lanczos: bool = False            # Lanczos steps instead of a plain chain
    # filled by the server
    method: int = hmv.AUTO           # the plan's method (the server's, or AUTO where that cannot take it)
    admitted: float | None = None
    finished: float | None = None
    latencies: list = field(default_factory=list)
    result: FixedVec | None = None   # the last vector (chain: A^k x; Lanczos: v_k)
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)
    footprint: int = 0


def plan_choice(n: int, b: int, kind: int, method: int) -> tuple[int, int]:
    """The method a request's plan gets and the device bytes it needs: the
    server's method, or AUTO where the NTT path cannot take the size."""
    try:
        return method, hmv.plan_bytes(n, b, kind=kind, method=method)
    except hmv.HmvError as err:
        if method == hmv.AUTO or err.status != hmv.EUNSUPPORTED:
            raise
    return hmv.AUTO, hmv.plan_bytes(n, b, kind=kind)


def percentile(values, q):
    if not values:
        return None
    return float(np.percentile(np.asarray(values, dtype=np.float64), q))


class Server:
    """method: hmv.AUTO (the tensor-core Karatsuba path) or hmv.NTT (the exact
    NTT path; a request whose size it cannot take gets AUTO)."""

    def __init__(self, memory_budget: int, max_active: int = 128, device: int = 0, clock=time.perf_counter,
                 method: int = hmv.AUTO):
        import torch
        if method not in (hmv.AUTO, hmv.NTT):
            raise ValueError("the server runs the tensor-core path (AUTO) or the exact NTT path (NTT)")
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.budget = memory_budget
        self.max_active = max_active
        self.clock = clock
        self.method = method
        self._warm_up()

    def _warm_up(self):
        # one exact inner product large enough for the tensor-core path: the
        # library's GEMM handle and kernels are made before the first request,
        # not inside its first product
        torch = self.torch
        n, b = 64, 33220
        x = FixedVec(np.ones((n, (b + 31) // 32), dtype=np.uint32), np.zeros(n, dtype=np.uint8), b, 0)
        with hmv.Plan(n, b, method=hmv.SCHOOLBOOK) as p:
            xl = torch.from_numpy(x.limbs.view(np.int32)).to(self.dev)
            xn = torch.from_numpy(x.neg).to(self.dev)
            torch.cuda.synchronize(self.dev)
            hmv.dot_device(p, (xl.data_ptr(), xn.data_ptr()), (xl.data_ptr(), xn.data_ptr()))

    def _admit(self, r: Request, now: float):
        # runs on the admission thread: the plan's load and the vectors'
        # copies go to the request's own stream, synchronised before the
        # request can join a step (a step then runs every active plan on its
        # lead plan's stream and synchronises it)
        torch = self.torch
        torch.cuda.set_device(self.dev)
        r.stream = torch.cuda.Stream(device=self.dev)
        with torch.cuda.stream(r.stream):
            r.plan = hmv.Plan(r.n, r.b, kind=r.kind, method=r.method, stream=r.stream.cuda_stream)
            r.plan.load_matrix(r.h)
            r.done = 0
            r.admitted = now
            if r.lanczos:
                from .lanczos import Lanczos
                r.lz = Lanczos(r.plan, r.x0, device=self.dev)
            else:
                r.xl = torch.from_numpy(r.x0.limbs.view(np.int32)).to(self.dev)
                r.xn = torch.from_numpy(r.x0.neg).to(self.dev)
                r.yl = torch.empty_like(r.xl)
                r.yn = torch.empty_like(r.xn)
                r.x_exp = r.x0.exponent
        r.stream.synchronize()

    def _finish(self, r: Request, now: float, pool):
        r.stream.synchronize()  # the request's last vector work (a step ends with its stream synchronised)
        if r.lanczos:
            r.result = r.lz.vector()
        else:
            r.result = FixedVec(r.xl.cpu().numpy().view(np.uint32), r.xn.cpu().numpy(), r.b, r.x_exp)
        r.finished = now
        r.retired = pool.submit(self._retire, r)

    def _retire(self, r: Request):
        # on the worker thread, in order with the admissions (the memory it
        # frees is counted free from now on)
        if r.lanczos:
            del r.lz
        else:
            del r.xl, r.xn, r.yl, r.yn
        r.plan.close()
        r.plan = None
        r.stream = None

    def run(self, requests: list[Request]) -> dict:
        if self.method == hmv.NTT:
            return self._run_independent(requests)
        return self._run_steps(requests)

    def _run_independent(self, requests: list[Request]) -> dict:
        """The NTT path's server: there is no shared leaf launch to batch, so
        every admitted request advances on its own, product after product on
        its own stream, from a runner thread; the GPU interleaves the
        requests' short kernels, and a request neither waits for a step
        boundary to start nor for the other requests' products.  Admission at
        arrival, in order, within the memory budget, as in the stepped loop."""
        import threading
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            r.method, r.footprint = plan_choice(r.n, r.b, r.kind, self.method)
            if r.footprint > self.budget:
                raise ValueError(f"request {r.rid} needs {r.footprint} bytes, more than the whole budget")
        cv = threading.Condition()
        shared = {"used": 0, "peak_used": 0, "inflight": 0, "running": 0, "peak_running": 0}
        pool = ThreadPoolExecutor(max_workers=1)  # admissions and releases, in order
        runners = ThreadPoolExecutor(max_workers=self.max_active)
        t0 = self.clock()

        def serve(r: Request):
            try:
                r.admission.result()  # an admission's error ends the run
                with cv:
                    shared["running"] += 1
                    shared["peak_running"] = max(shared["peak_running"], shared["running"])
                r.ready = r.arrival
                t_end = r.ready
                for _ in range(r.matvecs):
                    if r.lanczos:
                        a, bt = r.lz.step()
                        r.alphas.append(a)
                        r.betas.append(bt)
                    else:
                        e = r.plan.matvec_device(r.xl.data_ptr(), r.xn.data_ptr(), r.x_exp, r.yl.data_ptr(),
                                                 r.yn.data_ptr())
                        r.xl, r.yl = r.yl, r.xl
                        r.xn, r.yn = r.yn, r.xn
                        r.x_exp = e
                    t_end = self.clock() - t0
                    r.latencies.append(t_end - r.ready)
                    r.ready = t_end
                    r.done += 1
                    if r.lanczos and r.betas[-1][0] == 0:
                        break
                self._finish(r, t_end, pool)
            finally:
                with cv:
                    shared["running"] -= 1
                    shared["inflight"] -= 1
                    shared["used"] -= r.footprint
                    cv.notify_all()

        futures = []
        try:
            for r in pending:  # dispatch at arrival, in order, within the budget
                with cv:
                    while True:
                        delay = r.arrival - (self.clock() - t0)
                        if (delay <= 0 and shared["used"] + r.footprint <= self.budget
                                and shared["inflight"] < self.max_active):
                            break
                        cv.wait(timeout=delay if delay > 0 else 0.05)
                    shared["used"] += r.footprint
                    shared["peak_used"] = max(shared["peak_used"], shared["used"])
                    shared["inflight"] += 1
                r.admission = pool.submit(self._admit, r, self.clock() - t0)
                futures.append(runners.submit(serve, r))
            for f in futures:
                f.result()
        finally:
            runners.shutdown(wait=True)
        total = self.clock() - t0
        pool.shutdown(wait=True)
        for r in requests:
            r.retired.result()
        lat = [v for r in requests for v in r.latencies]
        req_lat = [r.finished - r.arrival for r in requests]
        nmv = sum(r.done for r in requests)
        return {"matvecs": nmv, "seconds": total, "matvecs_per_s": nmv / total if total > 0 else None,
                "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
                "request_p50_s": percentile(req_lat, 50), "request_p99_s": percentile(req_lat, 99),
                "steps": nmv, "mean_step_batch": 1.0, "peak_active": shared["peak_running"],
                "peak_bytes": shared["peak_used"], "mode": "independent requests"}

    def _run_steps(self, requests: list[Request]) -> dict:
        import threading
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            r.method, r.footprint = plan_choice(r.n, r.b, r.kind, self.method)
            if r.footprint > self.budget:
                raise ValueError(f"request {r.rid} needs {r.footprint} bytes, more than the whole budget")
        # shared with the dispatcher thread, under cv: device bytes of the
        # admitted plans, the number of active requests, the admissions in
        # flight, and whether every request has been dispatched
        cv = threading.Condition()
        shared = {"used": 0, "peak_used": 0, "active": 0, "admitting": [], "dispatched": False, "stop": False}
        pool = ThreadPoolExecutor(max_workers=1)
        t0 = self.clock()

        def dispatch():
            # each request's admission starts at its arrival (in order), as
            # soon as its plan fits the memory budget, while steps run
            try:
                for r in pending:
                    with cv:
                        while not shared["stop"]:
                            delay = r.arrival - (self.clock() - t0)
                            if (delay <= 0 and shared["used"] + r.footprint <= self.budget
                                    and shared["active"] + len(shared["admitting"]) < self.max_active):
                                break
                            cv.wait(timeout=delay if delay > 0 else 0.05)
                        if shared["stop"]:
                            return
                        shared["used"] += r.footprint
                        shared["peak_used"] = max(shared["peak_used"], shared["used"])
                        r.admission = pool.submit(self._admit, r, self.clock() - t0)
                        shared["admitting"].append(r)
                        cv.notify_all()
            finally:
                with cv:
                    shared["dispatched"] = True
                    cv.notify_all()

        dispatcher = threading.Thread(target=dispatch, daemon=True)
        dispatcher.start()
        active: list[Request] = []
        steps, step_sizes, peak_active = 0, [], 0
        try:
            while True:
                with cv:  # admitted requests join this step (one look at each admission)
                    joined, rest = [], []
                    for r in shared["admitting"]:
                        (joined if r.admission.done() else rest).append(r)
                    shared["admitting"] = rest
                for r in joined:
                    r.admission.result()  # an admission's error ends the run here
                    r.ready = r.arrival
                    active.append(r)
                with cv:
                    shared["active"] = len(active)
                    waiting = list(shared["admitting"])
                    if not active and not waiting and shared["dispatched"]:
                        break
                    if not active and not waiting:
                        cv.wait(timeout=0.05)  # until the next admission starts
                peak_active = max(peak_active, len(active))
                if not active:
                    if waiting:
                        waiting[0].admission.result()
                    continue
                xs, es, ys = [], [], []
                for r in active:
                    if r.lanczos:
                        vp, ev, wp = r.lz.operands()
                    else:
                        vp, ev, wp = (r.xl.data_ptr(), r.xn.data_ptr()), r.x_exp, (r.yl.data_ptr(), r.yn.data_ptr())
                    xs.append(vp)
                    es.append(ev)
                    ys.append(wp)
                exps = hmv.matvec_many_device([r.plan for r in active], xs, ys, es)
                for r, e in zip(active, exps):  # the rest of each Lanczos step
                    if r.lanczos:
                        a, bt = r.lz.finish(e)
                        r.alphas.append(a)
                        r.betas.append(bt)
                t_end = self.clock() - t0
                steps += 1
                step_sizes.append(len(active))
                still = []
                for r, e in zip(active, exps):
                    r.latencies.append(t_end - r.ready)
                    r.ready = t_end
                    if not r.lanczos:
                        r.xl, r.yl = r.yl, r.xl
                        r.xn, r.yn = r.yn, r.xn
                        r.x_exp = e
                    r.done += 1
                    if r.done == r.matvecs or (r.lanczos and r.betas[-1][0] == 0):
                        self._finish(r, t_end, pool)
                        with cv:  # its memory counts as free for the admissions that follow its release
                            shared["used"] -= r.footprint
                            cv.notify_all()
                    else:
                        still.append(r)
                active = still
        finally:
            with cv:
                shared["stop"] = True
                cv.notify_all()
            dispatcher.join()
        peak_used = shared["peak_used"]
        total = self.clock() - t0
        pool.shutdown(wait=True)
        for r in requests:
            r.retired.result()  # a release's error ends the run here
        lat = [v for r in requests for v in r.latencies]
        req_lat = [r.finished - r.arrival for r in requests]
        nmv = sum(r.done for r in requests)  # a Lanczos run that breaks down stops early
        return {"matvecs": nmv, "seconds": total, "matvecs_per_s": nmv / total if total > 0 else None,
                "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
                "request_p50_s": percentile(req_lat, 50), "request_p99_s": percentile(req_lat, 99),
                "steps": steps, "mean_step_batch": float(np.mean(step_sizes)) if step_sizes else 0.0,
                "peak_active": peak_active, "peak_bytes": peak_used, "mode": "continuous batching"}
