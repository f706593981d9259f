// Split-FP64 FFT path (Beliakov, arXiv:1402.5287, Sec. 1 "FFT-based
// multiplication" and Sec. 2 "Decomposition approach"): the multiprecision
// numbers are split into standard-precision pieces and the Hankel product
// becomes one cyclic convolution done with one double-precision FFT.
//
// Packing (Kronecker substitution, unscaled integer pieces): every entry is
// split into P balanced pieces of w bits, v = sum_p v_p 2^(w p) with
// |v_p| <= 2^(w-1).  With slot stride S >= 2P-1,
//     a[k S + p] = piece p of h_k,         k = 0..2n-2
//     c[(n-1-j) S + q] = piece q of x_j,   j = 0..n-1
// and the cyclic convolution of length N = 2^K >= (2n-1) S holds, in slot
// n-1+i, the digit sums sum_j sum_{p+q=t} h_{i+j}[p] x_j[q] of y_i (no
// wrap-around reaches those slots).  The spectrum of a is computed once per
// matrix.
//
// The FFTs are radix-2 (forward decimation in frequency: natural order in,
// bit-reversed out; inverse decimation in time: bit-reversed in, natural
// out), so no permutation pass is needed; up to 8 stages run per pass in
// shared memory.  Twiddles come from a table filled with sincospi.
//
// Rounding to integers is exact when every computed coefficient is within
// 1/2 of the true one.  The path proves that before it rounds, with the
// L2-norm bound for floating-point FFT convolution of C. Percival, "Rapid
// multiplication modulo the sum and difference of highly composite numbers"
// (Math. Comp. 72, 2003; also Brent and Zimmermann, "Modern Computer
// Arithmetic", Sec. 3.3):
//   |z' - z|_inf < ||a||_2 ||c||_2 ((1+e)^(3K) (1+e sqrt5)^(3K+1) (1+b)^(3K) - 1)
// for radix-2 transforms of length 2^K with unit roundoff e = 2^-53 and
// twiddle error b.  b = 2^-52 follows from the documented 1-ulp accuracy of
// double-precision sincospi.  The norms are exact integer sums of squares of
// the pieces actually used.
#include <cmath>

#include "hmv_internal.h"

namespace hmv {
namespace {

constexpr int kMaxR = 8;   // radix-2 stages per pass
constexpr int kCols = 16;  // sub-transforms per block

__global__ void k_twiddles(double2 *tw, int K) {
    const long long half = 1LL << (K - 1);
    for (long long m = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; m < half;
         m += static_cast<long long>(gridDim.x) * blockDim.x) {
        double s, c;
        // omega_N^m = exp(-2 pi i m / N): 2m/N is exact (N a power of two)
        sincospi(ldexp(static_cast<double>(m), 1 - K), &s, &c);
        tw[m] = make_double2(c, -s);
    }
}

// Balanced w-bit pieces of the rows of a sign-magnitude vector, placed at
// slot(k) * S + p; slot(k) = k (matrix side) or n-1-k (vector side).
// circ_n > 0 maps row k to entry (circ_n-1-k) mod circ_n.  Adds the exact
// sum of squares of the pieces to *sumsq.
__global__ void k_pieces(const uint32_t *__restrict__ limbs, const uint8_t *__restrict__ neg, int rows, int L32,
                         int w, int P, int S, int reverse_n, int circ_n, double2 *__restrict__ out,
                         unsigned long long *sumsq, int32_t *dstat) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long sq = 0;
    if (k < rows) {
        int src = k;
        if (circ_n > 0) src = ((circ_n - 1 - k) % circ_n + circ_n) % circ_n;
        const uint32_t *m = limbs + static_cast<size_t>(src) * L32;
        const int sgn = neg[src] ? -1 : 1;
        const long long slot = reverse_n > 0 ? (reverse_n - 1 - k) : k;
        double2 *o = out + slot * S;
        const long long half = 1LL << (w - 1), full = 1LL << w;
        long long carry = 0;
        for (int p = 0; p < P; ++p) {
            const long long bit = static_cast<long long>(w) * p;
            const int li = static_cast<int>(bit >> 5), off = static_cast<int>(bit & 31);
            unsigned long long chunk = 0;
            if (li < L32) chunk = m[li] >> off;
            if (off + w > 32 && li + 1 < L32) chunk |= static_cast<unsigned long long>(m[li + 1]) << (32 - off);
            chunk &= static_cast<unsigned long long>(full - 1);
            long long t = sgn * static_cast<long long>(chunk) + carry;
            carry = 0;
            if (t >= half) { t -= full; carry = 1; }
            else if (t < -half) { t += full; carry = -1; }
            o[p] = make_double2(static_cast<double>(t), 0.0);
            sq += static_cast<unsigned long long>(t * t);
        }
        if (carry != 0) set_status(dstat, DEV_OVERFLOW);
    }
    // warp sum, one atomic per warp
    for (int d = 16; d > 0; d >>= 1) sq += __shfl_down_sync(0xFFFFFFFFu, sq, d);
    if ((threadIdx.x & 31) == 0 && sq) atomicAdd(sumsq, sq);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One pass of radix-2 stages on sub-transforms of 2^r points spaced
// st = 2^(s_lo-1) apart inside blocks of 2^s_hi points.
// forward (decimation in frequency): stages s_hi down to s_lo,
//   (u, v) -> (u + v, (u - v) w_{2^s}^j)
// inverse (decimation in time): stages s_lo up to s_hi,
//   (u, v) -> (u + conj(w) v, u - conj(w) v)
// with j = (index of u) mod 2^s.
__global__ void __launch_bounds__(256) k_fft_pass(double2 *__restrict__ d, const double2 *__restrict__ tw, int K,
                                                  int s_hi, int r, int inverse) {
    extern __shared__ double2 sm[];  // [2^r][kCols]
    const int s_lo = s_hi - r + 1;
    const long long st = 1LL << (s_lo - 1);
    const int C = st >= kCols ? kCols : static_cast<int>(st);
    const int B = kCols / C;
    long long blk0, low0;
    if (st >= kCols) {
        const long long groups = st / kCols;
        blk0 = blockIdx.x / groups;
        low0 = (blockIdx.x % groups) * kCols;
    } else {
        blk0 = static_cast<long long>(blockIdx.x) * B;
        low0 = 0;
    }
    const int pts = 1 << r;
    auto gidx = [&](int t, int q) -> long long {
        return ((blk0 + q / C) << s_hi) + low0 + (q % C) + t * st;
    };
    for (int e = threadIdx.x; e < pts * kCols; e += blockDim.x) {
        const int t = e / kCols, q = e % kCols;
        sm[e] = d[gidx(t, q)];
    }
    __syncthreads();
    const int nbf = (pts / 2) * kCols;
    for (int st_i = 0; st_i < r; ++st_i) {
        const int s = inverse ? (s_lo + st_i) : (s_hi - st_i);
        const int ht = 1 << (s - s_lo);  // span in sub-transform units
        for (int e = threadIdx.x; e < nbf; e += blockDim.x) {
            const int q = e % kCols, bf = e / kCols;
            const int t = (bf / ht) * 2 * ht + (bf % ht);
            const long long j = low0 + (q % C) + static_cast<long long>(t % (2 * ht)) * st;
            double2 wv = tw[j << (K - s)];
            double2 u = sm[t * kCols + q], v = sm[(t + ht) * kCols + q];
            if (!inverse) {
                sm[t * kCols + q] = make_double2(u.x + v.x, u.y + v.y);
                sm[(t + ht) * kCols + q] = cmul(make_double2(u.x - v.x, u.y - v.y), wv);
            } else {
                wv.y = -wv.y;
                const double2 vw = cmul(v, wv);
                sm[t * kCols + q] = make_double2(u.x + vw.x, u.y + vw.y);
                sm[(t + ht) * kCols + q] = make_double2(u.x - vw.x, u.y - vw.y);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < pts * kCols; e += blockDim.x) {
        const int t = e / kCols, q = e % kCols;
        d[gidx(t, q)] = sm[e];
    }
}

// x <- (x * a) / N, exact power-of-two scaling
__global__ void k_pointwise(double2 *__restrict__ x, const double2 *__restrict__ a, long long N, double scale) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double2 p = cmul(x[i], a[i]);
        x[i] = make_double2(p.x * scale, p.y * scale);
    }
}

// Row i: coefficients c[(i+n-1) S + t], t < 2P-1, rounded to integers, then
// Z_i = sum_t c_t 2^(w t) -> |Z| limbs, sign, bit length (as the other paths).
__global__ void k_fft_extract(const double2 *__restrict__ c, int n, int S, int P, int w, uint32_t *__restrict__ zmag,
                              uint8_t *__restrict__ zneg, int32_t *__restrict__ zbits, int ZW, int32_t *dstat,
                              unsigned long long *maxdist, int row_offset) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 *row = c + static_cast<long long>(i + n - 1) * S;
    const int T = 2 * P - 1;
    double md = 0.0;
    __int128 carry = 0;
    for (int t = 0; t < T; ++t) {  // sign of Z: the final carry of the digit expansion
        const double v = row[t].x;
        const double rv = rint(v);
        md = fmax(md, fabs(v - rv));
        carry = (static_cast<__int128>(static_cast<long long>(rv)) + carry) >> w;
    }
    const int sgn = carry < 0 ? -1 : 1;
    uint32_t *z = zmag + static_cast<size_t>(row_offset + i) * ZW;
    for (int q = 0; q < ZW; ++q) z[q] = 0;
    carry = 0;
    const __int128 mask = (static_cast<__int128>(1) << w) - 1;
    long long bitpos = 0;
    for (int t = 0; t < T + 4; ++t, bitpos += w) {
        __int128 acc = carry + (t < T ? static_cast<__int128>(sgn * static_cast<long long>(rint(row[t].x))) : 0);
        const uint32_t dig = static_cast<uint32_t>(acc & mask);
        carry = acc >> w;
        const long long li = bitpos >> 5;
        const int off = static_cast<int>(bitpos & 31);
        if (li < ZW) z[li] |= dig << off;
        if (off + w > 32 && li + 1 < ZW) z[li + 1] |= dig >> (32 - off);
    }
    if (carry != 0) set_status(dstat, DEV_OVERFLOW);
    int top = -1;
    uint32_t topv = 0;
    for (int q = ZW - 1; q >= 0; --q)
        if (z[q]) { top = q; topv = z[q]; break; }
    const int bits = top < 0 ? 0 : 32 * top + (32 - __clz(topv));
    zbits[row_offset + i] = bits;
    zneg[row_offset + i] = (bits > 0 && sgn < 0) ? 1 : 0;
    atomicMax(dstat + 1, bits);
    atomicMax(maxdist, static_cast<unsigned long long>(__double_as_longlong(md)));
}

int grid_for(long long work, int threads = 256) {
    long long g = (work + threads - 1) / threads;
    return static_cast<int>(g < 65535LL * 32 ? g : 65535LL * 32);
}

cudaError_t run_fft(hmv_plan_s *p, double2 *data, bool inverse) {
    const int K = p->fft_K;
    // pass boundaries: from the top stage down in chunks of up to 8 stages
    int bounds[8][2];
    int np = 0;
    for (int s_hi = K; s_hi >= 1; s_hi -= kMaxR) {
        const int r = s_hi >= kMaxR ? kMaxR : s_hi;
        bounds[np][0] = s_hi;
        bounds[np][1] = r;
        ++np;
    }
    for (int k = 0; k < np; ++k) {
        const int idx = inverse ? (np - 1 - k) : k;
        const int s_hi = bounds[idx][0], r = bounds[idx][1];
        const long long blocks = (p->fft_N >> r) / kCols;
        const size_t smem = static_cast<size_t>(kCols) * (1u << r) * sizeof(double2);
        k_fft_pass<<<static_cast<unsigned>(blocks), 256, smem, p->stream>>>(data, p->fft_tw, K, s_hi, r,
                                                                            inverse ? 1 : 0);
        p->launches_total++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// Error bound of the FFT convolution for the given exact sums of squares.
double fft_error_bound(double sumsq_a, double sumsq_x, int K) {
    const double eps = std::ldexp(1.0, -53);
    const double beta = std::ldexp(1.0, -52);
    const double lg = 3.0 * K * std::log1p(eps) + (3.0 * K + 1.0) * std::log1p(eps * std::sqrt(5.0)) +
                      3.0 * K * std::log1p(beta);
    return std::sqrt(sumsq_a) * std::sqrt(sumsq_x) * std::expm1(lg) * (1.0 + 1e-9);
}

// Geometry for piece width w: pieces P, slot stride S, length exponent K.
void fft_geometry(int n, int b, int w, int &P, int &S, int &K) {
    P = (b + 2 + w - 1) / w;
    S = 2 * P - 1;
    const long long need = static_cast<long long>(2 * n - 1) * S;
    K = 12;
    while ((1LL << K) < need) ++K;
}

// Worst-case bound (every piece at full magnitude 2^(w-1)).
double fft_worst_bound(int n, int b, int w, int hlen) {
    int P, S, K;
    fft_geometry(n, b, w, P, S, K);
    const double m2 = std::ldexp(1.0, 2 * (w - 1));
    return fft_error_bound(static_cast<double>(hlen) * P * m2, static_cast<double>(n) * P * m2, K);
}

cudaError_t fft_init(hmv_plan_s *p) {
    k_twiddles<<<grid_for(p->fft_N / 2), 256, 0, p->stream>>>(p->fft_tw, p->fft_K);
    p->launches_total++;
    return cudaGetLastError();
}

cudaError_t set_fft_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fft_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kCols * (1u << kMaxR) * sizeof(double2)));
    if (e == cudaSuccess) done = true;
    return e;
}

// Matrix side: pieces of h into the spectrum buffer, then its forward FFT.
cudaError_t fft_load_matrix(hmv_plan_s *p) {
    cudaError_t e = set_fft_attrs();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->fft_a, 0, p->fft_N * sizeof(double2), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->fft_sumsq, 0, 2 * sizeof(unsigned long long), p->stream);
    if (e != cudaSuccess) return e;
    const int rows = 2 * p->n - 1;
    k_pieces<<<(rows + 127) / 128, 128, 0, p->stream>>>(p->h_limbs_d, p->h_neg_d, rows, p->L32, p->fft_w, p->fft_P,
                                                        p->fft_S, 0, p->kind == HMV_CIRCULANT ? p->n : 0, p->fft_a,
                                                        p->fft_sumsq, p->dstat);
    p->launches_total++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return run_fft(p, p->fft_a, false);
}

// Vector side, first half: pieces of x and their exact sum of squares.
cudaError_t fft_vector_pieces(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn) {
    cudaError_t e = cudaMemsetAsync(p->fft_x, 0, p->fft_N * sizeof(double2), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->fft_sumsq + 1, 0, sizeof(unsigned long long), p->stream);
    if (e != cudaSuccess) return e;
    k_pieces<<<(p->n + 127) / 128, 128, 0, p->stream>>>(xl, xn, p->n, p->L32, p->fft_w, p->fft_P, p->fft_S, p->n, 0,
                                                        p->fft_x, p->fft_sumsq + 1, p->dstat);
    p->launches_total++;
    return cudaGetLastError();
}

// Vector side, second half (after the bound has been checked): transform,
// pointwise product, inverse transform, exact rows.
cudaError_t fft_vector_product(hmv_plan_s *p, int rhs) {
    cudaError_t e = run_fft(p, p->fft_x, false);
    if (e != cudaSuccess) return e;
    k_pointwise<<<grid_for(p->fft_N), 256, 0, p->stream>>>(p->fft_x, p->fft_a, p->fft_N,
                                                           std::ldexp(1.0, -p->fft_K));
    p->launches_total++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = run_fft(p, p->fft_x, true);
    if (e != cudaSuccess) return e;
    k_fft_extract<<<(p->n + 127) / 128, 128, 0, p->stream>>>(p->fft_x, p->n, p->fft_S, p->fft_P, p->fft_w, p->zmag,
                                                            p->zneg, p->zbits, p->ZW, p->dstat, p->fft_maxdist,
                                                            rhs * p->n);
    p->launches_total++;
    return cudaGetLastError();
}

}  // namespace hmv
