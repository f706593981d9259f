// Exact number-theoretic-transform path (the decomposition of Beliakov,
// arXiv:1402.5287, Secs. 1-2: the multiprecision numbers split into standard
// precision pieces and the Hankel product done as ONE cyclic convolution),
// with the floating-point FFT replaced by transforms modulo two primes, so
// that the convolution is exact with no error bound to check.
//
// Packing (Kronecker substitution, as in the split-FP64 path): every entry is
// cut into P = ceil(b / 16) pieces of 16 bits carrying the entry's sign,
// v = sum_p v_p 2^(16 p), |v_p| < 2^16.  With slot stride S = 2P - 1,
//     a[k S + p] = piece p of h_k,          k = 0..2n-2
//     c[(n-1-j) S + q] = piece q of x_j,    j = 0..n-1
// and the cyclic convolution of length N = 2^K >= (2n-1) S holds in slot
// n-1+i the sums z_i[t] = sum_j sum_{p+q=t} h_{i+j}[p] x_j[q], t < 2P-1, of
// y_i = sum_t z_i[t] 2^(16 t); no wrapped term reaches those slots.
//
// Exactness: |z_i[t]| < n P 2^32 <= 2^57 (N <= 2^26 bounds n P), below half
// the product of the primes p1 = 15 2^27 + 1 and p2 = 27 2^26 + 1 (about
// 2^61.7), so the Chinese remainder of the two residues, taken in
// (-p1 p2 / 2, p1 p2 / 2), is the coefficient itself.  Both primes have
// 2^26 | p - 1, which bounds N to 2^26.
//
// Arithmetic: Montgomery multiplication modulo each prime with R = 2^32
// (p < 2^31, so sums of two residues fit 32 bits); twiddles are kept in
// Montgomery form in two small tables per prime (w^m = T_hi[m >> 13] T_lo[m
// & 8191]), data in normal form.  Radix-2 transforms, forward by decimation
// in frequency (natural order in, bit-reversed out), inverse by decimation
// in time (bit-reversed in, natural out), so no permutation pass; passes of
// 6 to 9 stages with the points in registers (one transpose through shared
// memory a pass), both primes in one pass (a uint2 per point).  The matrix's
// spectrum is kept per plan, scaled by 1/N.
#include <cstring>
#include <utility>
#include <vector>

#include "hmv_internal.h"

namespace hmv {

constexpr uint32_t kNttP0 = 2013265921u, kNttP1 = 1811939329u;  // 15 2^27 + 1, 27 2^26 + 1
constexpr uint32_t kNttP[2] = {kNttP0, kNttP1};
constexpr uint32_t kNttRoot[2] = {31u, 13u};                // primitive roots
constexpr int kNttMaxK = 26;
constexpr int kNttPieceBits = 16;
constexpr int kTwLoBits = 13;
constexpr int kNttRootWords = 2 * 256 * 2;  // w_512^(+-j), j < 256, both primes

namespace {

constexpr int kNttMaxR = 9;   // radix-2 stages per pass
constexpr int kNttCols = 16;  // sub-transforms per block (16 x 8 bytes: 128-byte rows)
static_assert(kNttCols == 16, "the pass indexes columns with e & 15 and e >> 4");

struct NttConst {
    uint32_t p[2], pinv[2];  // pinv = -p^-1 mod 2^32
    const uint32_t *tlo[2], *thi[2];
    // w_16^e (w16[0]) and w_16^-e (w16[1]), Montgomery form, [direction][prime][e]:
    // the register passes' twiddles of span 1, 2, 4 and 8, read as
    // kernel-parameter constants
    uint32_t w16[2][2][8];
    // w_512^j and w_512^-j, j < 256, as (prime 0, prime 1) pairs in Montgomery
    // form, [direction][j]: the register passes' wider spans
    const uint2 *rt;
};

// a b / 2^32 mod p for a < 2p, b < p: t + m p < 2 p^2 + 2^32 p < 2^64 and
// (t + m p) / 2^32 < 2p, one conditional subtraction (the unsigned minimum
// of u and u - p: u - p wraps above u when u < p).
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
    const uint64_t t = static_cast<uint64_t>(a) * b;
    const uint32_t m = static_cast<uint32_t>(t) * pinv;
    const uint32_t u = static_cast<uint32_t>((t + static_cast<uint64_t>(m) * p) >> 32);
    return umin(u, u - p);
}
__device__ __forceinline__ uint32_t mod_add(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t s = a + b;  // < 2p < 2^32
    return umin(s, s - p);
}
__device__ __forceinline__ uint32_t mod_sub(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t d = a - b;  // a - b, or a - b + 2^32 when a < b, where d + p wraps to a - b + p < p
    return umin(d, d + p);
}

// w_N^m (forward) or w_N^-m (inverse) in Montgomery form, 0 <= m < N/2;
// w^-m = -w^(N/2 - m) for m > 0
__device__ __forceinline__ uint32_t table_power(const NttConst &c, int k, int m) {
    return mont_mul(__ldg(c.thi[k] + (m >> kTwLoBits)), __ldg(c.tlo[k] + (m & ((1 << kTwLoBits) - 1))), c.p[k],
                    c.pinv[k]);
}

// 16-bit pieces of sign-magnitude rows as residues modulo both primes, piece
// p of row k at slot(k) S + p; slot(k) = k (matrix side) or n-1-k (vector
// side); circ_n > 0 maps row k to entry (circ_n-1-k) mod circ_n.  One thread
// per limb (two pieces).
__global__ void k_ntt_pieces(const uint32_t *__restrict__ limbs, const uint8_t *__restrict__ neg, int rows, int L32,
                             int P, int S, int reverse_n, int circ_n, uint2 *__restrict__ out, int32_t *dstat) {
    const long long id = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (id >= static_cast<long long>(rows) * L32) return;
    const int k = static_cast<int>(id / L32), q = static_cast<int>(id % L32);
    int src = k;
    if (circ_n > 0) src = ((circ_n - 1 - k) % circ_n + circ_n) % circ_n;
    const uint32_t limb = limbs[static_cast<size_t>(src) * L32 + q];
    const bool sg = neg[src] != 0;
    const long long slot = reverse_n > 0 ? (reverse_n - 1 - k) : k;
    uint2 *o = out + slot * S;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int pc = 2 * q + h;
        const uint32_t v = (limb >> (16 * h)) & 0xFFFFu;
        if (pc >= P) {
            if (v) set_status(dstat, DEV_BADINPUT);  // bits beyond the pieces (cannot happen for valid input)
            continue;
        }
        o[pc] = (sg && v) ? make_uint2(kNttP0 - v, kNttP1 - v) : make_uint2(v, v);
    }
}

// One pass of radix-2 stages on sub-transforms of 2^r points spaced
// st = 2^(s_lo-1) apart inside blocks of 2^s_hi points:
//   forward (decimation in frequency), stages s_hi down to s_lo:
//     (u, v) -> (u + v, (u - v) w_{2^s}^j)
//   inverse (decimation in time), stages s_lo up to s_hi:
//     (u, v) -> (u + w_{2^s}^-j v, u - w_{2^s}^-j v)
// with j = (index of u) mod 2^(s-1) and w_{2^s}^j = w_N^(j 2^(K-s)).
// A block holds 16 sub-transforms (16 x 8 bytes: every row of its tile is
// one 128-byte line of d).
struct PassGeo {
    int s_hi, s_lo, lst, lC, cmask, blk0, low0;
    __device__ PassGeo(int s_hi_, int r) : s_hi(s_hi_) {
        // every index fits 32 bits (N <= 2^26) and every span is a power of two:
        // shifts and masks only
        s_lo = s_hi - r + 1;
        lst = s_lo - 1;  // log2 of the point spacing st
        lC = lst >= 4 ? 4 : lst;  // log2 of C, the columns of one block of 2^s_hi points
        if (lst >= 4) {
            const int lgroups = lst - 4;
            blk0 = static_cast<int>(blockIdx.x) >> lgroups;
            low0 = (static_cast<int>(blockIdx.x) & ((1 << lgroups) - 1)) << 4;
        } else {
            blk0 = static_cast<int>(blockIdx.x) << (4 - lC);
            low0 = 0;
        }
        cmask = (1 << lC) - 1;
    }
    __device__ int gidx(int t, int q) const { return ((blk0 + (q >> lC)) << s_hi) + low0 + (q & cmask) + (t << lst); }
};

// ---------------------------------------------------------------- register-blocked passes
// The same passes with the points in registers.  A block holds 16 columns
// of 2^r points; thread (q, g) = (tid & 15, tid >> 4), g < G = 2^LG
// threads per column, owns NP = 2^r / G points of column q, in one of two
// layouts:
//   A: points g + G k (k < NP): the stages of span G .. 2^(r-1) points pair
//      k with k + span/G, inside the thread;
//   B: points NP g + k: the stages of span 1 .. G/2 pair k with k + span.
// A pass runs its stages of one layout, transposes the tile once through
// shared memory, and runs the rest: one shared-memory round trip and one
// barrier per pass instead of one per stage.
//
// Twiddles, in the four-step form of a pass.  Point t of column c (c the
// offset below the point spacing 2^lst) meets at stage s = s_lo + i (span
// 2^i points of the column) the twiddle w_{2^s}^(c + (t mod 2^i) 2^lst), the
// product of
//   an inner twiddle  w_{2^(i+1)}^(t mod 2^i), the same for every column, and
//   a column factor   w_{2^s}^c, on the lower output of every butterfly.
// The column factor of stage i multiplies exactly the points with bit i of
// t set, and the later stages combine only points that agree in that bit,
// so the factors commute to the end of a forward pass (to the start of an
// inverse one), where point t is multiplied once by
//   Phi_c(t) = prod_{i : bit i of t} w_{2^(s_lo+i)}^c = (w_{2^s_hi}^c)^rev_r(t)
// (rev_r: the r bits of t reversed).  Inner twiddles of spans 1..8 are
// powers of w_16 fixed at compile time once the loops over the registers
// are unrolled (kernel-parameter constants; the first butterfly of every
// span has twiddle 1 and no product); those of wider spans are powers of
// w_{2^r}, read from a 2^(r-1)-entry table in shared memory (one broadcast
// load per butterfly).  The lowest pass has c = 0 and no column factors.

// Both primes: DIF (u, v) -> (u + v, (u - v) w), DIT (u, v) -> (u + w v, u - w v).
template <bool INV>
__device__ __forceinline__ void ntt_bfly(uint2 &u, uint2 &v, uint2 w, const NttConst &c) {
    if (!INV) {
        const uint2 a = make_uint2(mod_add(u.x, v.x, c.p[0]), mod_add(u.y, v.y, c.p[1]));
        // u - v + p < 2p: mont_mul's range
        v = make_uint2(mont_mul(u.x + c.p[0] - v.x, w.x, c.p[0], c.pinv[0]),
                       mont_mul(u.y + c.p[1] - v.y, w.y, c.p[1], c.pinv[1]));
        u = a;
    } else {
        const uint2 t = make_uint2(mont_mul(v.x, w.x, c.p[0], c.pinv[0]), mont_mul(v.y, w.y, c.p[1], c.pinv[1]));
        v = make_uint2(mod_sub(u.x, t.x, c.p[0]), mod_sub(u.y, t.y, c.p[1]));
        u = make_uint2(mod_add(u.x, t.x, c.p[0]), mod_add(u.y, t.y, c.p[1]));
    }
}
// Either direction with twiddle 1.
__device__ __forceinline__ void ntt_bfly1(uint2 &u, uint2 &v, const NttConst &c) {
    const uint2 a = make_uint2(mod_add(u.x, v.x, c.p[0]), mod_add(u.y, v.y, c.p[1]));
    v = make_uint2(mod_sub(u.x, v.x, c.p[0]), mod_sub(u.y, v.y, c.p[1]));
    u = a;
}
// Layout B, span 2^I (I < LG <= 4): pairs (k, k + 2^I), t mod 2^I = k mod 2^I
// (NP g is a multiple of 2^I), twiddle w_{2^(I+1)}^(k mod 2^I) = w_16^e.
template <int NP, int I, bool INV>
__device__ __forceinline__ void ntt_b_stage(uint2 (&x)[NP], const NttConst &c) {
    constexpr int HK = 1 << I;
    static_assert(I <= 3 && 2 * HK <= NP, "spans 1..8 inside the thread (NP a multiple of 2^(I+1))");
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (i & HK) continue;
        const int e = (i & (HK - 1)) << (3 - I);
        if (e == 0) ntt_bfly1(x[i], x[i + HK], c);
        else ntt_bfly<INV>(x[i], x[i + HK], make_uint2(c.w16[INV][0][e], c.w16[INV][1][e]), c);
    }
}
// Layout A, span G 2^(I-LG) (I >= LG): pairs (k, k + 2^(I-LG)), t mod 2^I =
// g + G (k mod 2^(I-LG)), twiddle w_{2^(I+1)}^m = rt[m 2^(r-1-I)].
template <int NP, int LG, int I, bool INV>
__device__ __forceinline__ void ntt_a_stage(uint2 (&x)[NP], const uint2 *rt, const NttConst &c, int gq) {
    constexpr int R = __builtin_ctz(NP) + LG;
    constexpr int HK = 1 << (I - LG);
    constexpr int SH = R - 1 - I;
    static_assert(I >= LG && I < R, "spans G .. 2^(r-1)");
    const uint2 *tb = rt + (gq << SH);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (i & HK) continue;
        ntt_bfly<INV>(x[i], x[i + HK], tb[(i & (HK - 1)) << (LG + SH)], c);
    }
}
// Stages I, I + STEP, ..., LAST of one layout.
template <int NP, int LG, int I, int LAST, int STEP, bool INV>
__device__ __forceinline__ void ntt_a_stages(uint2 (&x)[NP], const uint2 *rt, const NttConst &c, int gq) {
    ntt_a_stage<NP, LG, I, INV>(x, rt, c, gq);
    if constexpr (I != LAST) ntt_a_stages<NP, LG, I + STEP, LAST, STEP, INV>(x, rt, c, gq);
}
template <int NP, int I, int LAST, int STEP, bool INV>
__device__ __forceinline__ void ntt_b_stages(uint2 (&x)[NP], const NttConst &c) {
    ntt_b_stage<NP, I, INV>(x, c);
    if constexpr (I != LAST) ntt_b_stages<NP, I + STEP, LAST, STEP, INV>(x, c);
}
// w_N^m (or w_N^-m with inv), 0 <= m < N: w^(N/2) = -1, w^-m = w^(N-m).
__device__ __forceinline__ uint32_t root_power(const NttConst &c, int k, int m, bool inv, int K) {
    const int half = 1 << (K - 1);
    if (inv && m != 0) m = 2 * half - m;
    return m < half ? table_power(c, k, m) : c.p[k] - table_power(c, k, m - half);
}
constexpr int bit_reverse(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
// x[k] *= Phi_c(t) (or its inverse) for the thread's points t = NP g + k of
// layout B.  rev_r(t) = rev(k) G + rev(g), so Phi_c(t) = V^rev(g) (V^G)^rev(k)
// with V = w_{2^s_hi}^c = w_N^(c 2^(K - s_hi)): the powers are stepped
// through in the order of rev(k), one product per point, and applied, one
// more.
template <int NP, int LG, bool INV>
__device__ __forceinline__ void ntt_column_factors(uint2 (&x)[NP], const NttConst &c, const PassGeo &g, int K) {
    constexpr int LNP = __builtin_ctz(NP);
    const int q = threadIdx.x & 15, gq = threadIdx.x >> 4;
    const int col = g.low0 + (q & g.cmask);
    const int sh = K - g.s_hi;
    const int e0 = (col * static_cast<int>(__brev(static_cast<unsigned>(gq)) >> (32 - LG))) << sh;  // < 2^(K-LNP)
    const int ez = col << (sh + LG);
    uint32_t f[2], z[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        f[k] = root_power(c, k, e0, INV, K);
        z[k] = root_power(c, k, ez, INV, K);
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int k = bit_reverse(j, LNP);
        x[k] = make_uint2(mont_mul(x[k].x, f[0], c.p[0], c.pinv[0]), mont_mul(x[k].y, f[1], c.p[1], c.pinv[1]));
        if (j + 1 < NP) {
            f[0] = mont_mul(f[0], z[0], c.p[0], c.pinv[0]);
            f[1] = mont_mul(f[1], z[1], c.p[1], c.pinv[1]);
        }
    }
}
// The inner twiddles w_{2^r}^j (or w_{2^r}^-j), j < 2^(r-1): entries j 2^(9-r)
// of the w_512 table.  The caller synchronises before the first use.
template <int R>
__device__ __forceinline__ void ntt_load_roots(uint2 *rt, const NttConst &c, int inv) {
    static_assert(R <= 9, "the table holds powers of w_512");
    for (int j = threadIdx.x; j < (1 << (R - 1)); j += blockDim.x) rt[j] = c.rt[inv * 256 + (j << (9 - R))];
}

// The register passes' tile in shared memory: point t of column q at
// t * kTilePitch + q; the padding makes both a column-major and a row-major
// sweep conflict-free.
constexpr int kTilePitch = 17;
// A -> B (toB) or B -> A through the tile.
template <int NP, int LG>
__device__ __forceinline__ void ntt_reg_transpose(uint2 (&x)[NP], uint2 *tile, bool toB) {
    const int q = threadIdx.x & 15, gq = threadIdx.x >> 4;
#pragma unroll
    for (int k = 0; k < NP; ++k) tile[(toB ? gq + (k << LG) : NP * gq + k) * kTilePitch + q] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = tile[(toB ? NP * gq + k : gq + (k << LG)) * kTilePitch + q];
    __syncthreads();
}
// Loads and stores of a pass's points in layout A (layoutA) or B.  Where the
// 16 columns are 16 consecutive runs of 2^r points (the lowest pass, st = 1)
// a warp's points would fall in 16 separate pieces of memory: there the
// block copies its whole contiguous range through the tile instead.
template <int NP, int LG>
__device__ __forceinline__ void ntt_reg_load(uint2 (&x)[NP], const uint2 *__restrict__ d, uint2 *tile, const PassGeo &g,
                                             bool layoutA) {
    constexpr int r = __builtin_ctz(NP) + LG;
    const int q = threadIdx.x & 15, gq = threadIdx.x >> 4;
    if (g.lst == 0) {
        const uint2 *src = d + (static_cast<size_t>(g.blk0) << r);
        for (int e = threadIdx.x; e < (16 << r); e += blockDim.x) tile[(e & ((1 << r) - 1)) * kTilePitch + (e >> r)] = src[e];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NP; ++k) x[k] = tile[(layoutA ? gq + (k << LG) : NP * gq + k) * kTilePitch + q];
        __syncthreads();
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) x[k] = d[g.gidx(layoutA ? gq + (k << LG) : NP * gq + k, q)];
    }
}
template <int NP, int LG>
__device__ __forceinline__ void ntt_reg_store(const uint2 (&x)[NP], uint2 *__restrict__ d, uint2 *tile,
                                              const PassGeo &g, bool layoutA) {
    constexpr int r = __builtin_ctz(NP) + LG;
    const int q = threadIdx.x & 15, gq = threadIdx.x >> 4;
    if (g.lst == 0) {
#pragma unroll
        for (int k = 0; k < NP; ++k) tile[(layoutA ? gq + (k << LG) : NP * gq + k) * kTilePitch + q] = x[k];
        __syncthreads();
        uint2 *dst = d + (static_cast<size_t>(g.blk0) << r);
        for (int e = threadIdx.x; e < (16 << r); e += blockDim.x) dst[e] = tile[(e & ((1 << r) - 1)) * kTilePitch + (e >> r)];
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) d[g.gidx(layoutA ? gq + (k << LG) : NP * gq + k, q)] = x[k];
    }
}
template <int NP, int LG>
__device__ __forceinline__ void ntt_reg_forward(uint2 (&x)[NP], uint2 *tile, const uint2 *rt, const NttConst &c,
                                                const PassGeo &g, int K) {
    constexpr int R = __builtin_ctz(NP) + LG;
    const int gq = threadIdx.x >> 4;
    ntt_a_stages<NP, LG, R - 1, LG, -1, false>(x, rt, c, gq);  // spans 2^(R-1) .. G, layout A
    ntt_reg_transpose<NP, LG>(x, tile, true);
    ntt_b_stages<NP, LG - 1, 0, -1, false>(x, c);  // spans G/2 .. 1, layout B
    if (g.lst > 0) ntt_column_factors<NP, LG, false>(x, c, g, K);
}
template <int NP, int LG>
__device__ __forceinline__ void ntt_reg_inverse(uint2 (&x)[NP], uint2 *tile, const uint2 *rt, const NttConst &c,
                                                const PassGeo &g, int K) {
    constexpr int R = __builtin_ctz(NP) + LG;
    const int gq = threadIdx.x >> 4;
    if (g.lst > 0) ntt_column_factors<NP, LG, true>(x, c, g, K);
    ntt_b_stages<NP, 0, LG - 1, 1, true>(x, c);  // spans 1 .. G/2, layout B
    ntt_reg_transpose<NP, LG>(x, tile, false);
    ntt_a_stages<NP, LG, LG, R - 1, 1, true>(x, rt, c, gq);  // spans G .. 2^(R-1), layout A
}

// A pass of r = log2(NP G) stages with 16 G threads; forward passes load in
// layout A and store in layout B, inverse passes the other way round.  At
// most 128 registers a thread for 32 points (two 256-thread blocks per SM):
// measured 3.58 instead of 4.14 ms per matvec at one block per SM.
template <int NP, int LG>
__global__ void __launch_bounds__(16 << LG, NP == 32 ? 2 : 3) k_ntt_rpass(uint2 *__restrict__ d, NttConst c, int K,
                                                                             int s_hi, int inverse) {
    extern __shared__ uint2 tile[];  // [NP G][kTilePitch], then the 2^(r-1) inner twiddles
    constexpr int r = __builtin_ctz(NP) + LG;
    uint2 *rt = tile + (NP << LG) * kTilePitch;
    ntt_load_roots<r>(rt, c, inverse);
    __syncthreads();
    const PassGeo g(s_hi, r);
    uint2 x[NP];
    ntt_reg_load<NP, LG>(x, d, tile, g, !inverse);
    if (!inverse) ntt_reg_forward<NP, LG>(x, tile, rt, c, g, K);
    else ntt_reg_inverse<NP, LG>(x, tile, rt, c, g, K);
    ntt_reg_store<NP, LG>(x, d, tile, g, inverse);
}

// The lowest forward stages, the product with the matrix spectrum and the
// lowest inverse stages in one pass, with the points in registers: blocks of
// 2^r consecutive points stay on chip (both transforms visit them in the same
// bit-reversed order).
template <int NP, int LG>
__global__ void __launch_bounds__(16 << LG, NP == 32 ? 2 : 3) k_ntt_rmid(uint2 *__restrict__ d,
                                                                            const uint2 *__restrict__ a, NttConst c,
                                                                            int K) {
    extern __shared__ uint2 tile[];  // [NP G][kTilePitch], then the forward and inverse inner twiddles
    constexpr int r = __builtin_ctz(NP) + LG;
    uint2 *rtf = tile + (NP << LG) * kTilePitch, *rti = rtf + (1 << (r - 1));
    ntt_load_roots<r>(rtf, c, 0);
    ntt_load_roots<r>(rti, c, 1);
    __syncthreads();
    const PassGeo g(r, r);
    uint2 x[NP];
    ntt_reg_load<NP, LG>(x, d, tile, g, true);
    ntt_reg_forward<NP, LG>(x, tile, rtf, c, g, K);
    // layout B; the spectrum is stored in this kernel's register order
    // (point k of thread tid of block bx at (bx NP + k) 16 G + tid), so the
    // reads are coalesced
    const uint2 *ab = a + (static_cast<size_t>(blockIdx.x) * NP << (4 + LG)) + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const uint2 v = ab[k << (4 + LG)];
        x[k] = make_uint2(mont_mul(x[k].x, v.x, c.p[0], c.pinv[0]), mont_mul(x[k].y, v.y, c.p[1], c.pinv[1]));
    }
    ntt_reg_inverse<NP, LG>(x, tile, rti, c, g, K);
    ntt_reg_store<NP, LG>(x, d, tile, g, true);
}

// Shared memory of the register passes: the tile and the inner twiddles
// (one direction for k_ntt_rpass, both for k_ntt_rmid).
constexpr size_t ntt_rsmem(int r, bool mid) {
    return (static_cast<size_t>(kTilePitch) * (1u << r) + (mid ? (1u << r) : (1u << (r - 1)))) * sizeof(uint2);
}

// dst <- src * f in the register order of k_ntt_rmid<NP, LG> for a last pass
// of r stages (lnp = log2 NP, lt = 4 + LG the log2 of its threads): entry
// (bx NP + k) 2^lt + tid holds point NP (tid >> 4) + k of column tid & 15 of
// that kernel's block bx.
__global__ void k_ntt_scale_perm(const uint2 *__restrict__ src, uint2 *__restrict__ dst, long long N, int r, int lnp,
                                 int lt, NttConst c, uint32_t f0, uint32_t f1) {
    for (long long o = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; o < N;
         o += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long bx = o >> (lnp + lt);
        const int rem = static_cast<int>(o & ((1LL << (lnp + lt)) - 1));
        const int k = rem >> lt, tid = rem & ((1 << lt) - 1);
        const int q = tid & 15, gq = tid >> 4;
        const uint2 u = src[((bx * 16 + q) << r) + (static_cast<long long>(gq) << lnp) + k];
        dst[o] = make_uint2(mont_mul(u.x, f0, c.p[0], c.pinv[0]), mont_mul(u.y, f1, c.p[1], c.pinv[1]));
    }
}

// Row i of the product: the coefficients z[t] = c[(i+n-1) S + t], t < 2P-1,
// each the Chinese remainder of its two residues taken in (-p1 p2/2,
// p1 p2/2), then Z_i = sum_t z[t] 2^(16 t) as |Z| limbs, sign and bit length
// (as the other paths).  One warp per row, a window of 512 positions at a
// time: the residues are read coalesced (lane l: positions l + 32 k) and
// their coefficients parked in shared memory, from where every lane takes
// 16 consecutive positions; a carry chain base 2^16 per lane, then the
// carries passed up one lane per round among the lanes that hold positions
// of the row until none is left; two positions make a limb.  A final carry
// of -1 means Z < 0: the limbs hold its two's complement and are negated in
// place.
__device__ __forceinline__ long long ntt_crt(uint2 r, const NttConst &c, uint32_t inv1R) {
    const uint32_t p1 = c.p[0], p2 = c.p[1];
    const uint32_t r1m = r.x >= p2 ? r.x - p2 : r.x;  // r1 < p1 < 2 p2
    const uint32_t x = mont_mul(mod_sub(r.y, r1m, p2), inv1R, p2, c.pinv[1]);  // (r2 - r1) / p1 mod p2
    const unsigned long long M = static_cast<unsigned long long>(p1) * p2;
    const unsigned long long v = r.x + static_cast<unsigned long long>(p1) * x;  // in [0, p1 p2)
    return v > M / 2 ? static_cast<long long>(v) - static_cast<long long>(M) : static_cast<long long>(v);
}
constexpr int kExPos = 16;               // consecutive positions a lane
constexpr int kExWin = 32 * kExPos;      // positions a window
constexpr int kExPitch = kExPos + 1;     // shared-memory words a lane (the padding spreads the banks)
constexpr int kExWarps = 8;              // rows a block
// digits base 2^16 of v + carry-in, in place; returns the carry out (floor)
__device__ __forceinline__ long long ntt_chain(long long (&v)[kExPos], long long cy) {
#pragma unroll
    for (int k = 0; k < kExPos; ++k) {
        const long long s = v[k] + cy;
        v[k] = s & 0xFFFF;
        cy = s >> 16;  // arithmetic: floor
    }
    return cy;
}
__global__ void __launch_bounds__(32 * kExWarps) k_ntt_extract(const uint2 *__restrict__ cvec, int n, int S, int T,
                                                              NttConst c, uint32_t inv1R, uint32_t *__restrict__ zmag,
                                                              uint8_t *__restrict__ zneg, int32_t *__restrict__ zbits,
                                                              int ZW, int32_t *dstat, int row_offset) {
    __shared__ long long win[kExWarps][32 * kExPitch];
    const int lane = threadIdx.x & 31;
    const int i = static_cast<int>(blockIdx.x) * kExWarps + static_cast<int>(threadIdx.x >> 5);
    if (i >= n) return;  // warp-uniform; the warps share no data
    long long *ws = win[threadIdx.x >> 5];
    const uint2 *row = cvec + static_cast<long long>(i + n - 1) * S;
    uint32_t *z = zmag + static_cast<size_t>(row_offset + i) * ZW;
    const int span = max(T, 2 * ZW);  // every limb of the row is written
    long long wc = 0;
    bool above_nonzero = false, above_not_ones = false;
    for (int t0 = 0; t0 < span; t0 += kExWin) {
#pragma unroll
        for (int k = 0; k < kExPos; ++k) {
            const int e = lane + 32 * k;  // position t0 + e, kept by lane e / 16
            const int t = t0 + e;
            ws[(e >> 4) * kExPitch + (e & 15)] = t < T ? ntt_crt(row[t], c, inv1R) : 0;
        }
        __syncwarp();
        long long v[kExPos];
#pragma unroll
        for (int k = 0; k < kExPos; ++k) v[k] = ws[lane * kExPitch + k];
        __syncwarp();  // the next window's writes come after every lane's reads
        const int tb = t0 + kExPos * lane;
        const int last = min(31, (span - 1 - t0) / kExPos);  // the last lane with positions of the row
        long long pending = ntt_chain(v, lane == 0 ? wc : 0), out = 0;
        for (int round = 0; round <= 32; ++round) {
            out += __shfl_sync(0xffffffffu, pending, last);
            long long incoming = __shfl_up_sync(0xffffffffu, pending, 1);
            if (lane == 0 || lane > last) incoming = 0;
            if (!__any_sync(0xffffffffu, incoming != 0)) break;
            pending = ntt_chain(v, incoming);
        }
        wc = out;
#pragma unroll
        for (int k = 0; k < kExPos / 2; ++k) {
            const uint32_t limb = static_cast<uint32_t>(v[2 * k]) | (static_cast<uint32_t>(v[2 * k + 1]) << 16);
            const int li = tb / 2 + k;
            if (li < ZW) {
                z[li] = limb;
            } else if (lane <= last) {
                above_nonzero |= limb != 0u;
                above_not_ones |= limb != 0xFFFFFFFFu;
            }
        }
    }
    // wc: 0 (Z >= 0) or -1 (the limbs are 2^(32 ZW) + Z); otherwise Z does not fit
    const bool negative = wc == -1;
    bool bad = (wc != 0 && wc != -1) || (negative ? above_not_ones : above_nonzero);
    __syncwarp();
    if (negative) {
        int k0 = ZW;  // lowest non-zero limb
        for (int w = lane; w < ZW; w += 32)
            if (z[w]) { k0 = w; break; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) k0 = min(k0, __shfl_xor_sync(0xffffffffu, k0, off));
        if (k0 == ZW) bad = true;
        // four limbs a lane per round, loaded before any is stored: with the
        // loads and stores of z interleaved, each load waited for the one
        // before (at n = 64 the matvec took 158.5 instead of 143 us)
        for (int w0 = lane; w0 < ZW; w0 += 4 * 32) {
            uint32_t v4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = w0 + 32 * q;
                v4[q] = w < ZW ? z[w] : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = w0 + 32 * q;
                if (w >= ZW) break;
                if (w == k0) z[w] = ~v4[q] + 1u;
                else if (w > k0) z[w] = ~v4[q];
            }
        }
        __syncwarp();
    }
    int bits = 0;
    for (int w = lane; w < ZW; w += 32)
        if (z[w]) bits = 32 * w + (32 - __clz(z[w]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(dstat, DEV_OVERFLOW);
    if (lane == 0) {
        zbits[row_offset + i] = bits;
        zneg[row_offset + i] = (bits > 0 && negative) ? 1 : 0;
        atomicMax(dstat + 1, bits);
    }
}

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (a * b) % p; }  // a, b < p < 2^31
uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1;
    for (a %= p; e; e >>= 1, a = mulmod(a, a, p))
        if (e & 1) r = mulmod(r, a, p);
    return r;
}

NttConst ntt_const(const hmv_plan_s *p) {
    NttConst c;
    for (int k = 0; k < 2; ++k) {
        c.p[k] = kNttP[k];
        uint32_t inv = 1;  // p^-1 mod 2^32 by Newton's iteration (p odd)
        for (int it = 0; it < 5; ++it) inv *= 2u - kNttP[k] * inv;
        c.pinv[k] = 0u - inv;
        c.tlo[k] = p->ntt_tw + (2 * k) * (1 << kTwLoBits);
        c.thi[k] = p->ntt_tw + (2 * k + 1) * (1 << kTwLoBits);
        const uint64_t P = kNttP[k];
        const uint64_t w16 = powmod(kNttRoot[k], (P - 1) / 16, P);
        const uint64_t R = (uint64_t(1) << 32) % P;
        for (int e = 0; e < 8; ++e) {
            c.w16[0][k][e] = static_cast<uint32_t>(mulmod(powmod(w16, e, P), R, P));
            c.w16[1][k][e] = static_cast<uint32_t>(mulmod(powmod(w16, (16 - e) % 16, P), R, P));
        }
    }
    c.rt = reinterpret_cast<const uint2 *>(p->ntt_tw + 4 * (1 << kTwLoBits));
    return c;
}

int grid_for(long long work, int threads = 256) {
    const long long g = (work + threads - 1) / threads;
    return static_cast<int>(g < 65535LL * 32 ? g : 65535LL * 32);
}

// Pass boundaries, from the top stage down; the last pass ends with stage 1.
// K >= 13 is cut into ceil(K / 9) passes as even as possible, the longer ones
// first (26 = 9 + 9 + 8, 24 = 8 + 8 + 8, 23 = 8 + 8 + 7, 21 = 7 + 7 + 7,
// 13 = 7 + 6): every pass has 6 to 9 stages and runs with the points in
// registers.  (Splits into 9s with a short last pass ran the middle kernel
// from shared memory, at up to five times the time per point and stage.)
int ntt_passes(int K, int (&bounds)[8][2]) {
    const int nr = (K + kNttMaxR - 1) / kNttMaxR;
    int s_hi = K;
    for (int i = 0; i < nr; ++i) {
        const int r = K / nr + (i < K % nr ? 1 : 0);
        bounds[i][0] = s_hi;
        bounds[i][1] = r;
        s_hi -= r;
    }
    return nr;
}
// The register kernels' shape for a pass of r stages: NP points a thread,
// G = 2^LG threads a column (NP >= G: the two layouts), 16 G threads a block.
constexpr int ntt_lg(int r) { return r >= 8 ? 4 : 3; }
constexpr int ntt_lnp(int r) { return r - ntt_lg(r); }

cudaError_t ntt_attrs() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    // (the smaller passes stay under the default 48 KB)
    cudaError_t e = cudaFuncSetAttribute(k_ntt_rpass<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(ntt_rsmem(9, false)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ntt_rmid<32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(ntt_rsmem(9, true)));
    if (e == cudaSuccess) attr = true;
    return e;
}

cudaError_t launch_pass(hmv_plan_s *p, uint2 *data, const NttConst &c, int s_hi, int r, int inverse) {
    const unsigned blocks = static_cast<unsigned>((p->ntt_N >> r) / kNttCols);
    const size_t smem = ntt_rsmem(r, false);
    const int threads = 16 << ntt_lg(r);
    switch (r) {  // points in registers: NP a thread, G threads a column (8 threads a column for the
                  // 8-stage pass measured slower: 3.87 vs 3.58 ms per matvec); ntt_passes gives 6..9
        case 9: k_ntt_rpass<32, 4><<<blocks, threads, smem, p->stream>>>(data, c, p->ntt_K, s_hi, inverse); break;
        case 8: k_ntt_rpass<16, 4><<<blocks, threads, smem, p->stream>>>(data, c, p->ntt_K, s_hi, inverse); break;
        case 7: k_ntt_rpass<16, 3><<<blocks, threads, smem, p->stream>>>(data, c, p->ntt_K, s_hi, inverse); break;
        case 6: k_ntt_rpass<8, 3><<<blocks, threads, smem, p->stream>>>(data, c, p->ntt_K, s_hi, inverse); break;
        default: return cudaErrorInvalidValue;
    }
    p->launches_total++;
    return cudaGetLastError();
}

// Forward transform (matrix side).
cudaError_t run_ntt_forward(hmv_plan_s *p, uint2 *data) {
    cudaError_t e = ntt_attrs();
    const NttConst c = ntt_const(p);
    int bounds[8][2];
    const int np = ntt_passes(p->ntt_K, bounds);
    for (int k = 0; k < np && e == cudaSuccess; ++k) e = launch_pass(p, data, c, bounds[k][0], bounds[k][1], 0);
    return e;
}

// Forward transform, product with the matrix spectrum and inverse transform
// (vector side): the last forward pass, the product and the first inverse
// pass share one kernel.
cudaError_t run_ntt_product(hmv_plan_s *p, uint2 *data) {
    cudaError_t e = ntt_attrs();
    const NttConst c = ntt_const(p);
    int bounds[8][2];
    const int np = ntt_passes(p->ntt_K, bounds);
    for (int k = 0; k + 1 < np && e == cudaSuccess; ++k) e = launch_pass(p, data, c, bounds[k][0], bounds[k][1], 0);
    if (e == cudaSuccess) {
        const int r = bounds[np - 1][1];  // s_hi = r: blocks of 2^r consecutive points
        const unsigned blocks = static_cast<unsigned>((p->ntt_N >> r) / kNttCols);
        const size_t smem = ntt_rsmem(r, true);
        const int threads = 16 << ntt_lg(r);
        switch (r) {
            case 9: k_ntt_rmid<32, 4><<<blocks, threads, smem, p->stream>>>(data, p->ntt_a, c, p->ntt_K); break;
            case 8: k_ntt_rmid<16, 4><<<blocks, threads, smem, p->stream>>>(data, p->ntt_a, c, p->ntt_K); break;
            case 7: k_ntt_rmid<16, 3><<<blocks, threads, smem, p->stream>>>(data, p->ntt_a, c, p->ntt_K); break;
            case 6: k_ntt_rmid<8, 3><<<blocks, threads, smem, p->stream>>>(data, p->ntt_a, c, p->ntt_K); break;
            default: return cudaErrorInvalidValue;
        }
        p->launches_total++;
        e = cudaGetLastError();
    }
    for (int k = np - 2; k >= 0 && e == cudaSuccess; --k) e = launch_pass(p, data, c, bounds[k][0], bounds[k][1], 1);
    return e;
}

}  // namespace

// Geometry of the NTT path: P pieces of 16 bits, slot stride S = 2P - 1,
// N = 2^K >= (2n - 1) S; false when N would exceed 2^26.
bool ntt_geometry(int n, int b, int &P, int &S, int &K) {
    P = (b + kNttPieceBits - 1) / kNttPieceBits;
    S = 2 * P - 1;
    const long long need = static_cast<long long>(2 * n - 1) * S;
    K = 13;  // two passes of 6 or more stages (the register kernels' shapes), 16 columns a block
    while ((1LL << K) < need) ++K;
    return K <= kNttMaxK;
}

size_t ntt_table_words() { return 4 * (size_t(1) << kTwLoBits) + kNttRootWords; }

// Twiddle tables (Montgomery form, R = 2^32) for both primes: T_lo[i] =
// w^i, T_hi[i] = w^(i 2^13), w a primitive 2^K-th root of unity; then the
// register passes' w_512 table.
cudaError_t ntt_init(hmv_plan_s *p) {
    const int TS = 1 << kTwLoBits;
    std::vector<uint32_t> tab(ntt_table_words());
    for (int k = 0; k < 2; ++k) {
        const uint64_t P = kNttP[k];
        const uint64_t w = powmod(kNttRoot[k], (P - 1) >> p->ntt_K, P);
        const uint64_t R = (uint64_t(1) << 32) % P;
        uint64_t lo = R, hi = R;  // w^0 R
        const uint64_t wstep = powmod(w, TS, P);
        for (int i = 0; i < TS; ++i) {
            tab[(2 * k) * TS + i] = static_cast<uint32_t>(lo);
            tab[(2 * k + 1) * TS + i] = static_cast<uint32_t>(hi);
            lo = mulmod(lo, w, P);
            hi = mulmod(hi, wstep, P);
        }
    }
    // the register passes' inner twiddles: w_512^j and w_512^-j, j < 256, as
    // (prime 0, prime 1) pairs, forward table first
    for (int k = 0; k < 2; ++k) {
        const uint64_t P = kNttP[k];
        const uint64_t w512 = powmod(kNttRoot[k], (P - 1) / 512, P);
        const uint64_t R = (uint64_t(1) << 32) % P;
        for (int j = 0; j < 256; ++j) {
            tab[4 * static_cast<size_t>(TS) + 2 * j + k] = static_cast<uint32_t>(mulmod(powmod(w512, j, P), R, P));
            tab[4 * static_cast<size_t>(TS) + 512 + 2 * j + k] =
                static_cast<uint32_t>(mulmod(powmod(w512, (512 - j) % 512, P), R, P));
        }
    }
    return cudaMemcpyAsync(p->ntt_tw, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, p->stream);
}

// Matrix side: pieces of h, forward transform, scaling to Montgomery form / N.
cudaError_t ntt_load_matrix(hmv_plan_s *p) {
    const NttConst c = ntt_const(p);
    cudaError_t e = cudaMemsetAsync(p->ntt_a, 0, p->ntt_N * sizeof(uint2), p->stream);
    if (e != cudaSuccess) return e;
    const int rows = 2 * p->n - 1;
    k_ntt_pieces<<<grid_for(static_cast<long long>(rows) * p->L32), 256, 0, p->stream>>>(
        p->h_limbs_d, p->h_neg_d, rows, p->L32, p->ntt_P, p->ntt_S, 0, p->kind == HMV_CIRCULANT ? p->n : 0, p->ntt_a,
        p->dstat);
    p->launches_total++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = run_ntt_forward(p, p->ntt_a);
    if (e != cudaSuccess) return e;
    uint32_t f[2];
    for (int k = 0; k < 2; ++k) {  // R^2 / N mod p: mont_mul(A, f) = A R / N, the Montgomery form of A / N
        const uint64_t P = kNttP[k];
        const uint64_t R = (uint64_t(1) << 32) % P;
        f[k] = static_cast<uint32_t>(mulmod(mulmod(R, R, P), powmod(p->ntt_N % P, P - 2, P), P));
    }
    int bounds[8][2];
    const int last_r = bounds[ntt_passes(p->ntt_K, bounds) - 1][1];
    // the middle pass reads the spectrum (in Montgomery form, times 1/N: f = R^2 / N mod p) in its own
    // register order
    k_ntt_scale_perm<<<grid_for(p->ntt_N), 256, 0, p->stream>>>(p->ntt_a, p->ntt_x, p->ntt_N, last_r,
                                                                ntt_lnp(last_r), 4 + ntt_lg(last_r), c, f[0], f[1]);
    std::swap(p->ntt_a, p->ntt_x);  // the vector side's work array is free until the next matvec
    p->launches_total++;
    return cudaGetLastError();
}

// Vector side for right-hand side rhs: pieces, forward transform, pointwise
// product, inverse transform, exact rows into zmag/zneg/zbits.
cudaError_t ntt_vector_product(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn, int rhs) {
    const NttConst c = ntt_const(p);
    cudaError_t e = cudaMemsetAsync(p->ntt_x, 0, p->ntt_N * sizeof(uint2), p->stream);
    if (e != cudaSuccess) return e;
    k_ntt_pieces<<<grid_for(static_cast<long long>(p->n) * p->L32), 256, 0, p->stream>>>(
        xl, xn, p->n, p->L32, p->ntt_P, p->ntt_S, p->n, 0, p->ntt_x, p->dstat);
    p->launches_total++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = run_ntt_product(p, p->ntt_x);
    if (e != cudaSuccess) return e;
    const uint64_t P2 = kNttP[1];
    const uint32_t inv1R =
        static_cast<uint32_t>(mulmod(powmod(kNttP[0] % P2, P2 - 2, P2), (uint64_t(1) << 32) % P2, P2));
    k_ntt_extract<<<static_cast<unsigned>((p->n + kExWarps - 1) / kExWarps), 32 * kExWarps, 0, p->stream>>>(
        p->ntt_x, p->n, p->ntt_S, 2 * p->ntt_P - 1, c, inv1R, p->zmag, p->zneg, p->zbits, p->ZW, p->dstat, rhs * p->n);
    p->launches_total++;
    return cudaGetLastError();
}

}  // namespace hmv

// ---------------------------------------------------------------- measurement
namespace hmv {
namespace {
// Chains of independent Montgomery products modulo the first prime: the
// rate that bounds the transform stages.
__global__ void k_mont_rate(uint32_t *out, int iters, uint32_t w) {
    constexpr int ILP = 8;
    uint32_t pinv = 1;
    for (int i = 0; i < 5; ++i) pinv *= 2u - kNttP0 * pinv;
    pinv = 0u - pinv;
    uint32_t x[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = (threadIdx.x * 7919u + blockIdx.x * 104729u + i) % kNttP0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < ILP; ++i) x[i] = mont_mul(x[i], w, kNttP0, pinv);
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s ^= x[i];
    out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}
}  // namespace
}  // namespace hmv

extern "C" hmv_status hmv_measure_montgomery_rate(void *stream, double *products_per_s) {
    if (!products_per_s) return HMV_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return HMV_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * blocks * threads) != cudaSuccess) return HMV_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        hmv::k_mont_rate<<<blocks, threads, 0, st>>>(out, iters, 12345u);  // warm-up, then timed
        e = cudaEventRecord(e0, st);
        hmv::k_mont_rate<<<blocks, threads, 0, st>>>(out, iters, 12345u);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0 || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || best <= 0) return HMV_ECUDA;
    *products_per_s = static_cast<double>(blocks) * threads * iters * 8 / (best * 1e-3);
    return HMV_OK;
}
