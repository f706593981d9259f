"""CPU replica of the NTT path's pass schedule (no GPU): the register-blocked
passes' assignment of points to threads (layouts A and B with one transpose),
their four-step twiddles (inner twiddles per stage, one column factor per
point at the end of a forward pass and the start of an inverse one) and the
split of the K stages into passes must reproduce a textbook radix-2
transform.  Forward: decimation in
frequency, natural order in, bit-reversed out; inverse: decimation in time,
back to natural order, times N.  Arithmetic modulo the path's first prime.
"""
import numpy as np
import pytest

P1 = 2013265921  # 15 * 2^27 + 1
ROOT1 = 31


def root(K):
    return pow(ROOT1, (P1 - 1) >> K, P1)


def passes(K):
    """The library's split of stages K .. 1 into ceil(K / 9) passes, as even
    as possible, the longer ones first."""
    nr = -(-K // 9)
    out, s_hi = [], K
    for i in range(nr):
        r = K // nr + (1 if i < K % nr else 0)
        out.append((s_hi, r))
        s_hi -= r
    return out


def shape(r):
    """Points a thread NP and log2 of the threads a column LG for a pass of r
    stages: 32 x 16, 16 x 16, 16 x 8, 8 x 8 for r = 9, 8, 7, 6."""
    LG = 4 if r >= 8 else 3
    return 1 << (r - LG), LG


def geo(bx, s_hi, r):
    s_lo = s_hi - r + 1
    lst = s_lo - 1
    lC = min(4, lst)
    if lst >= 4:
        blk0, low0 = bx >> (lst - 4), (bx & ((1 << (lst - 4)) - 1)) << 4
    else:
        blk0, low0 = bx << (4 - lC), 0
    cmask = (1 << lC) - 1
    return dict(s_lo=s_lo, lst=lst, lC=lC, blk0=blk0, low0=low0, cmask=cmask, s_hi=s_hi)


def gidx(g, t, q):
    return ((g["blk0"] + (q >> g["lC"])) << g["s_hi"]) + g["low0"] + (q & g["cmask"]) + (t << g["lst"])


def wpow(K, m, inverse):
    w = root(K)
    return pow(w, (-m) % (1 << K) if inverse else m, P1)


def rev(v, bits):
    return int(format(v, "0%db" % bits)[::-1], 2) if bits else 0


def reg_stage(xs, r, I, A, inverse, NP, LG):
    """One stage (span 2^I points of the column) on every thread's registers,
    as ntt_a_stage / ntt_b_stage: inner twiddles only, from the w_{2^r} table
    (layout A) or as powers of w_16 (layout B), checked against
    w_{2^(I+1)}^(t mod 2^I)."""
    G = 1 << LG
    HK = (1 << (I - LG)) if A else (1 << I)
    for tid in range(16 * G):
        gq = tid >> 4
        x = xs[tid]
        for i in range(NP):
            if i & HK:
                continue
            if A:
                w = wpow(r, (gq + G * (i & (HK - 1))) << (r - 1 - I), inverse)
            else:
                w = wpow(4, (i & (HK - 1)) << (3 - I), inverse)
            t = (gq + G * i) if A else (NP * gq + i)
            assert w == wpow(I + 1, t % (1 << I), inverse)
            u, v = x[i], x[i + HK]
            if not inverse:
                x[i], x[i + HK] = (u + v) % P1, (u - v) * w % P1
            else:
                tv = v * w % P1
                x[i], x[i + HK] = (u + tv) % P1, (u - tv) % P1


def column_factors(xs, g, K, inverse, NP, LG):
    """ntt_column_factors: point t = NP g + k of column c times
    (w_{2^s_hi}^c)^rev_r(t), the powers stepped through in the order of
    rev(k) from V^rev(g) by V^G."""
    lnp = NP.bit_length() - 1
    r = lnp + LG
    sh = K - g["s_hi"]
    for tid in range(16 << LG):
        q, gq = tid & 15, tid >> 4
        col = g["low0"] + (q & g["cmask"])
        f = wpow(K, (col * rev(gq, LG)) << sh, inverse)
        z = wpow(K, col << (sh + LG), inverse)
        for j in range(NP):
            k = rev(j, lnp)
            assert f == wpow(K, (col * rev(NP * gq + k, r)) << sh, inverse)
            xs[tid][k] = xs[tid][k] * f % P1
            f = f * z % P1


def run_rpass(d, K, s_hi, r, inverse, spectrum=None):
    """k_ntt_rpass (spectrum None) or k_ntt_rmid (with the pointwise product)
    as the library launches them: 16 columns a block, G threads a column, NP
    points a thread (shape(r)); inner stages, then the column factors
    (forward), or the factors first (inverse)."""
    NP, LG = shape(r)
    G = 1 << LG
    T = 16 * G
    N = len(d)

    def pa(gq, k):
        return gq + G * k

    def pb(gq, k):
        return NP * gq + k

    for bx in range((N >> r) // 16):
        g = geo(bx, s_hi, r)
        load_b = inverse and spectrum is None
        xs = [[d[gidx(g, (pb if load_b else pa)(tid >> 4, k), tid & 15)] for k in range(NP)] for tid in range(T)]

        def transpose(to_b):
            tile = {}
            for tid in range(T):
                q, gq = tid & 15, tid >> 4
                for k in range(NP):
                    tile[((pa if to_b else pb)(gq, k), q)] = xs[tid][k]
            for tid in range(T):
                q, gq = tid & 15, tid >> 4
                xs[tid] = [tile[((pb if to_b else pa)(gq, k), q)] for k in range(NP)]

        def forward():
            for I in range(r - 1, LG - 1, -1):
                reg_stage(xs, r, I, True, False, NP, LG)
            transpose(True)
            for I in range(LG - 1, -1, -1):
                reg_stage(xs, r, I, False, False, NP, LG)
            if g["lst"] > 0:
                column_factors(xs, g, K, False, NP, LG)

        def inverse_stages():
            if g["lst"] > 0:
                column_factors(xs, g, K, True, NP, LG)
            for I in range(0, LG):
                reg_stage(xs, r, I, False, True, NP, LG)
            transpose(False)
            for I in range(LG, r):
                reg_stage(xs, r, I, True, True, NP, LG)

        if spectrum is not None:
            forward()
            for tid in range(T):
                q, gq = tid & 15, tid >> 4
                xs[tid] = [xs[tid][k] * spectrum[gidx(g, pb(gq, k), q)] % P1 for k in range(NP)]
            inverse_stages()
            store_a = True
        elif not inverse:
            forward()
            store_a = False
        else:
            inverse_stages()
            store_a = True
        for tid in range(T):
            q, gq = tid & 15, tid >> 4
            for k in range(NP):
                d[gidx(g, (pa if store_a else pb)(gq, k), q)] = xs[tid][k]


def dif_reference(a, K):
    a = np.array(a, dtype=object)
    N = 1 << K
    for s in range(K, 0, -1):
        half = 1 << (s - 1)
        wj = [wpow(K, j << (K - s), False) for j in range(half)]
        for b0 in range(0, N, 2 * half):
            for j in range(half):
                u, v = a[b0 + j], a[b0 + j + half]
                a[b0 + j] = (u + v) % P1
                a[b0 + j + half] = (u - v) * wj[j] % P1
    return list(a)


@pytest.mark.parametrize("K", [13, 14, 16, 17])
def test_register_passes_equal_radix2_transform(K):
    """Passes 7 + 6, 7 + 7, 8 + 8 and 9 + 8: every register kernel shape."""
    rng = np.random.default_rng(K)
    N = 1 << K
    x = [int(v) for v in rng.integers(0, P1, N)]
    plan = passes(K)
    assert all(6 <= r <= 9 for _, r in plan)  # the register kernels cover every size
    d = list(x)
    for s_hi, r in plan:
        run_rpass(d, K, s_hi, r, False)
    assert d == dif_reference(x, K)
    # the inverse passes (last pass first) bring it back, times N
    for s_hi, r in reversed(plan):
        run_rpass(d, K, s_hi, r, True)
    assert d == [v * N % P1 for v in x]


@pytest.mark.parametrize("K", [13, 16])
def test_middle_pass_is_forward_product_inverse(K):
    """k_ntt_rmid: the last forward pass, the pointwise product and the first
    inverse pass in one, equal to the three done apart (last pass 6 and 8
    stages)."""
    rng = np.random.default_rng(5)
    N = 1 << K
    x = [int(v) for v in rng.integers(0, P1, N)]
    spec = [int(v) for v in rng.integers(0, P1, N)]
    (s0, r0), (s1, r1) = passes(K)
    a = list(x)
    run_rpass(a, K, s0, r0, False)
    b = list(a)
    run_rpass(a, K, s1, r1, False, spectrum=spec)
    run_rpass(b, K, s1, r1, False)
    b = [u * v % P1 for u, v in zip(b, spec)]
    run_rpass(b, K, s1, r1, True)
    assert a == b


def test_pass_split():
    assert passes(26) == [(26, 9), (17, 9), (8, 8)]
    assert passes(24) == [(24, 8), (16, 8), (8, 8)]
    assert passes(23) == [(23, 8), (15, 8), (7, 7)]
    assert passes(21) == [(21, 7), (14, 7), (7, 7)]
    assert passes(13) == [(13, 7), (6, 6)]
    for K in range(13, 27):
        rs = [r for _, r in passes(K)]
        assert sum(rs) == K and passes(K)[-1][0] == rs[-1]
        assert all(6 <= r <= 9 for r in rs) and max(rs) - min(rs) <= 1
        NP, LG = shape(rs[-1])
        assert NP >= (1 << LG) and NP << LG == 1 << rs[-1]  # both layouts hold; 16 G threads cover 2^r points
        assert (1 << (K - rs[0])) >= 16  # the first pass has 16 columns a block


@pytest.mark.parametrize("r", [6, 7, 8, 9])
def test_spectrum_permutation_matches_middle_kernel_reads(r):
    """k_ntt_scale_perm stores the matrix spectrum so that thread tid of the
    middle kernel's block bx finds point NP (tid >> 4) + k of its column
    tid & 15 at (bx NP + k) 16 G + tid: the store is a permutation of the N
    points, and each of those reads lands on the point the lowest pass's
    geometry names."""
    NP, LG = shape(r)
    lnp, lt = NP.bit_length() - 1, 4 + LG
    K = r + 5  # two blocks of 16 columns
    N = 1 << K
    src = []
    for o in range(N):  # the kernel's index arithmetic, entry by entry
        bx, rem = o >> (lnp + lt), o & ((1 << (lnp + lt)) - 1)
        k, tid = rem >> lt, rem & ((1 << lt) - 1)
        q, gq = tid & 15, tid >> 4
        src.append(((bx * 16 + q) << r) + (gq << lnp) + k)
    assert sorted(src) == list(range(N))
    for bx in range((N >> r) // 16):
        g = geo(bx, r, r)
        for tid in range(16 << LG):
            q, gq = tid & 15, tid >> 4
            for k in range(NP):
                assert src[((bx * NP) << lt) + tid + (k << lt)] == gidx(g, NP * gq + k, q)
