"""Lanczos driver on a device-resident Hankel matrix.

The paper's introduction motivates fast multiprecision Hankel products by
Lanczos-type iterations on these matrices; this module runs that iteration on
top of a loaded plan.  It uses the unnormalised three-term recurrence for the
symmetric A = A_H (no square roots):

    w            = A v_k
    alpha_k      = <v_k, w> / <v_k, v_k>
    w            = w - alpha_k v_k - beta_k v_{k-1}
    beta_{k+1}   = <w, w> / <v_k, v_k>
    v_{k+1}      = w

with v_{-1} = 0 and beta_0 = 0.  The symmetric tridiagonal matrix with
diagonal alpha and off-diagonal sqrt(beta_{k+1}) is the Lanczos matrix; its
eigenvalues (the Ritz values) are the caller's business.

Arithmetic: every vector is b-bit block fixed point; A v and the update of w
are exact and then rounded once (hmv_matvec, hmv_lincomb: least shared
exponent, ties to even); the inner products are exact (hmv_dot); alpha and
beta are the exact ratios rounded to b-bit floating point, ties to even, on
the host.  Every step is deterministic, so a run is reproducible bit for bit.
"""
from __future__ import annotations

import numpy as np

from . import hmv
from .inputs import FixedVec


def _round_ratio_exact(n: int, d: int, b: int) -> tuple[int, int]:
    """(q, t) with q = RNE(n 2^t / d), 2^(b-1) <= q < 2^b, for n, d > 0."""
    t = b - 1 - (n.bit_length() - d.bit_length())  # n 2^t / d in [2^(b-2), 2^b)
    while True:
        q, r = divmod(n << t, d) if t >= 0 else divmod(n, d << -t)
        dd = d if t >= 0 else d << -t
        if q >= 1 << (b - 1):
            break
        t += 1
    if 2 * r > dd or (2 * r == dd and q & 1):
        q += 1
        if q == 1 << b:
            q >>= 1
            t -= 1
    return q, t


_GUARD = 64  # guard bits of the truncated quotient


def _round_ratio_fast(n: int, d: int, b: int):
    """(q, t) as _round_ratio_exact from the leading b + 2G bits of n and d
    (G guard bits), or None when the truncated quotient cannot decide the
    rounding.  With N' = floor(n / 2^kn) and D' = floor(d / 2^kd) both at
    least 2^(b+2G-1) (or exact), the quotient Q = floor(N' 2^E / D') of the
    scaled ratio y = n 2^(t+G) / d satisfies |y - N' 2^E / D'| < 2^(2-G), so
    floor(y) is Q - 1, Q or Q + 1; the rounding at b bits is decided unless
    the G low bits of Q lie within 3 of one half (or Q within 3 of the
    normalisation boundary)."""
    G = _GUARD
    keep = b + 2 * G
    kn = max(0, n.bit_length() - keep)
    kd = max(0, d.bit_length() - keep)
    N, D = n >> kn, d >> kd
    t = b - (n.bit_length() - d.bit_length())  # n 2^t / d in [2^(b-1), 2^(b+1))
    E = t + G + kn - kd
    Q = (N << E) // D if E >= 0 else N // (D << -E)
    top = 1 << (b + G)
    if abs(Q - top) <= 4 or Q < (top >> 1) + 4:
        return None
    if Q > top:  # the value at t is above 2^b: one bit less
        Q >>= 1
        t -= 1
        if abs(Q - top) <= 4 or Q < (top >> 1) + 4:
            return None
    half = 1 << (G - 1)
    frac = Q & ((1 << G) - 1)
    if abs(frac - half) <= 3:
        return None
    q = (Q >> G) + (1 if frac > half else 0)
    if q == 1 << b:
        q >>= 1
        t -= 1
    return q, t


def round_ratio(num: int, den: int, shift: int, b: int) -> tuple[int, int]:
    """(m, e) with m * 2^e = RNE_b(num / den * 2^shift), 2^(b-1) <= |m| < 2^b
    (m = 0, e = 0 for a zero numerator).  Decided from the leading bits of
    num and den when that is enough, else by the exact division."""
    if den == 0:
        raise ZeroDivisionError("zero denominator")
    if num == 0:
        return 0, 0
    neg = (num < 0) != (den < 0)
    n, d = abs(num), abs(den)
    r = _round_ratio_fast(n, d, b)
    q, t = r if r is not None else _round_ratio_exact(n, d, b)
    return (-q if neg else q), shift - t


class Lanczos:
    """Runs the recurrence for the plan's matrix from a start vector; keeps
    v_{k-1}, v_k and w on the device (torch tensors on the plan's device)."""

    def __init__(self, plan: hmv.Plan, x0: FixedVec, device=None):
        import torch
        self.torch = torch
        self.plan = plan
        self.b = plan.b
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.dev = dev

        def buf(v=None):
            if v is None:
                limbs = torch.zeros((plan.n, plan.L32), dtype=torch.int32, device=dev)
                neg = torch.zeros(plan.n, dtype=torch.uint8, device=dev)
            else:
                limbs = torch.from_numpy(v.limbs.view(np.int32)).to(dev)
                neg = torch.from_numpy(v.neg).to(dev)
            return [limbs, neg]

        self.v, self.ev = buf(x0), x0.exponent
        self.u, self.eu = buf(), 0
        self.w = buf()
        torch.cuda.current_stream(dev).synchronize()  # the copies land before the plan's stream reads them
        self.beta = (0, 0)
        self.dvv = None
        self.k = 0

    @staticmethod
    def _ptrs(t):
        return t[0].data_ptr(), t[1].data_ptr()

    def operands(self):
        """The next product w = A v_k as ((v limbs, v sign), E_v, (w limbs, w sign))
        device pointers, for a caller that runs it (hmv_matvec_many) itself."""
        p = self.plan
        # the previous step's device calls have finished on the plan's stream
        if self.dvv is None:
            self.dvv = hmv.dot_device(p, self._ptrs(self.v), self._ptrs(self.v))
        if self.dvv == 0:
            raise ArithmeticError("Lanczos breakdown: v_k = 0")
        return self._ptrs(self.v), self.ev, self._ptrs(self.w)

    def finish(self, ew: int) -> tuple[tuple[int, int], tuple[int, int]]:
        """The rest of the step once w = A v_k (exponent ew) is in place:
        returns alpha_k and beta_{k+1} as (mantissa, exponent)."""
        p, b = self.plan, self.b
        P = self._ptrs
        dvw = hmv.dot_device(p, P(self.v), P(self.w))
        alpha = round_ratio(dvw, self.dvv, ew - self.ev, b)
        terms = [(1, 0, P(self.w), ew), (-alpha[0], alpha[1], P(self.v), self.ev)]
        if self.k > 0 and self.beta[0] != 0:
            terms.append((-self.beta[0], self.beta[1], P(self.u), self.eu))
        ew2 = hmv.lincomb_device(p, terms, P(self.w))  # w is read before it is written
        dww = hmv.dot_device(p, P(self.w), P(self.w))
        beta = round_ratio(dww, self.dvv, 2 * ew2 - 2 * self.ev, b) if dww else (0, 0)
        # rotate: u <- v, v <- w, w <- the old u's storage
        self.u, self.v, self.w = self.v, self.w, self.u
        self.eu, self.ev = self.ev, ew2
        self.beta = beta
        self.dvv = dww
        self.k += 1
        return alpha, beta

    def step(self) -> tuple[tuple[int, int], tuple[int, int]]:
        """One iteration: returns alpha_k and beta_{k+1} as (mantissa, exponent)."""
        vp, ev, wp = self.operands()
        return self.finish(self.plan.matvec_device(*vp, ev, *wp))

    def run(self, steps: int):
        """Up to `steps` iterations (fewer if the recurrence breaks down):
        lists of alpha_k and beta_{k+1}."""
        alphas, betas = [], []
        for _ in range(steps):
            if self.dvv == 0:
                break
            a, bt = self.step()
            alphas.append(a)
            betas.append(bt)
            if bt[0] == 0:
                break
        return alphas, betas

    def vector(self) -> FixedVec:
        """The current v_k as a host FixedVec."""
        self.torch.cuda.synchronize()
        return FixedVec(self.v[0].cpu().numpy().view(np.uint32), self.v[1].cpu().numpy(), self.b, self.ev)
