// Plain schoolbook Hankel product on 32-bit limbs (Beliakov,
// arXiv:1402.5287, Sec. 1: y_i = sum_j a_{i+j} x_j), CUDA cores only.
// It is the comparison kernel for the tensor-core Karatsuba path.
//
// Block (w-block, row i): thread w accumulates the exact signed column sum
//     S_w = sum_j sign_j * sum_p A_{i+j}[p] * X_j[w-p]
// of 32-bit limb weight w in a 128-bit integer; the row value is
// sum_w S_w 2^(32 w), normalised afterwards.
#include "hmv_internal.h"

namespace hmv {
namespace {

constexpr int kT = 128;

__global__ void __launch_bounds__(kT) k_schoolbook(const uint32_t *__restrict__ hl, const uint8_t *__restrict__ hn,
                                                   const uint32_t *__restrict__ xl, const uint8_t *__restrict__ xn,
                                                   int n, int L32, int circ, __int128 *__restrict__ colsum) {
    extern __shared__ uint32_t sh[];
    uint32_t *As = sh;
    uint32_t *Xs = sh + L32;
    const int i = blockIdx.y;
    const int w0 = blockIdx.x * kT;
    const int w = w0 + threadIdx.x;
    const int ncols = 2 * L32;
    // limbs this block touches: p in [p_min, p_max], w-p in [q_min, q_max]
    const int p_min = max(0, w0 - (L32 - 1)), p_max = min(L32 - 1, w0 + kT - 1);
    const int q_min = max(0, w0 - (L32 - 1)), q_max = min(L32 - 1, w0 + kT - 1);
    const int p_lo = max(0, w - (L32 - 1)), p_hi = min(L32 - 1, w);
    __int128 acc = 0;
    for (int j = 0; j < n; ++j) {
        const int k = i + j;
        const int src = circ ? (((n - 1 - k) % n) + n) % n : k;
        __syncthreads();
        for (int q = p_min + threadIdx.x; q <= p_max; q += kT) As[q] = hl[static_cast<size_t>(src) * L32 + q];
        for (int q = q_min + threadIdx.x; q <= q_max; q += kT) Xs[q] = xl[static_cast<size_t>(j) * L32 + q];
        __syncthreads();
        unsigned __int128 s = 0;
        for (int p = p_lo; p <= p_hi; ++p) s += static_cast<unsigned long long>(As[p]) * Xs[w - p];
        const bool neg = (hn[src] != 0) != (xn[j] != 0);
        acc += neg ? -static_cast<__int128>(s) : static_cast<__int128>(s);
    }
    if (w < ncols) colsum[static_cast<size_t>(i) * ncols + w] = acc;
}

}  // namespace

cudaError_t launch_schoolbook(hmv_plan_s *p, const uint32_t *x_limbs, const uint8_t *x_neg, int rhs) {
    (void)rhs;
    const int ncols = 2 * p->L32;
    dim3 grid((ncols + kT - 1) / kT, p->n);
    const size_t smem = static_cast<size_t>(2) * p->L32 * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_schoolbook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_schoolbook<<<grid, kT, smem, p->stream>>>(p->h_limbs_d, p->h_neg_d, x_limbs, x_neg, p->n, p->L32,
                                                 p->kind == HMV_CIRCULANT ? 1 : 0, p->colsum);
    p->launches_total++;
    return cudaGetLastError();
}

// Whether the kernel's dynamic shared memory (both operands' limbs of one
// row, 2 L32 words) fits the current device's opt-in limit per block.
bool schoolbook_smem_fits(int L32) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return static_cast<size_t>(2) * L32 * sizeof(uint32_t) <= static_cast<size_t>(optin);
}

// Same kernel on caller-given buffers (used by the scratch-free entry point).
cudaError_t launch_schoolbook_raw(const uint32_t *hl, const uint8_t *hn, const uint32_t *xl, const uint8_t *xn, int n,
                                  int L32, int circ, __int128 *colsum, cudaStream_t stream) {
    const int ncols = 2 * L32;
    dim3 grid((ncols + kT - 1) / kT, n);
    const size_t smem = static_cast<size_t>(2) * L32 * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_schoolbook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_schoolbook<<<grid, kT, smem, stream>>>(hl, hn, xl, xn, n, L32, circ, colsum);
    return cudaGetLastError();
}

}  // namespace hmv
