// Exact vector operations for Krylov drivers on top of the resident-matrix
// products: the inner product of two b-bit block vectors and a short linear
// combination rounded once to b bits.  A Lanczos iteration on the Hankel
// matrix (the consumer of fast multiprecision Hankel products named in the
// introduction of Beliakov, arXiv:1402.5287) needs exactly these next to
// y = A x.
//
// Both are schoolbook sums of 32-bit limb products in signed 128-bit column
// sums (the same representation as the plain product kernel), normalised to
// limbs by k_colsum_normalize.  The inner product's products are
// register-blocked over operands staged in shared memory; the linear
// combination reads its scalars' limbs as broadcasts from the read-only cache.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "hmv_internal.h"

namespace hmv {
namespace {

constexpr int kDotRows = 8;  // rows summed by one thread of the inner product

// One limb product added into a 96-bit column sum (a0, a1, a2) with the carry
// chain of the integer multiply-add.
__device__ __forceinline__ void mac96(uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t u, uint32_t v) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2)
        : "r"(u), "r"(v));
}

// Four consecutive columns v0..v0+3 of the product of a limb string C (nl
// limbs) and a row X (L32 limbs), out[q] = sum_a C[a] X[v0 + q - a], with a
// sliding window of X limbs: one new X limb and one C limb per four products.
__device__ __forceinline__ void cols4(const uint32_t *__restrict__ cr, int nl, const uint32_t *__restrict__ xr,
                                      int L32, int v0, unsigned __int128 (&out)[4]) {
    const int a_lo = max(0, v0 - (L32 - 1)), a_hi = min(nl - 1, v0 + 3);
    uint32_t s0[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0};
    uint32_t win[4];  // win[q] = X[v0 + q - a] (0 outside the row)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = v0 + q - a_lo;
        win[q] = (j >= 0 && j < L32) ? xr[j] : 0u;
    }
    for (int a = a_lo; a <= a_hi; ++a) {
        const uint32_t ca = __ldg(cr + a);
#pragma unroll
        for (int q = 0; q < 4; ++q) mac96(s0[q], s1[q], s2[q], ca, win[q]);
        win[3] = win[2];
        win[2] = win[1];
        win[1] = win[0];
        const int j = v0 - a - 1;
        win[0] = (j >= 0 && j < L32) ? xr[j] : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        out[q] = (static_cast<unsigned __int128>(s2[q]) << 64) |
                 (static_cast<unsigned __int128>(s1[q]) << 32) | s0[q];
}

// Column sums of limb-string products on the CUDA cores.  A warp owns 128
// consecutive columns w (4 a lane) and stages, in its own piece of shared
// memory, the first operand A 1024 limbs at a time and the window of the
// second operand B those columns meet (j = w - a), both zero-padded, so that
// a lane reads four limbs with one 16-byte shared load and makes a
// 4-column x 4-limb block of products per step, each added into a 96-bit
// column sum (a row's sums stay below 2^(64 + 15), b <= 2^20).  Warps
// synchronise only among their own lanes.
constexpr int kBlasWarps = 4;                        // warps of a block (independent tasks)
constexpr int kWarpCols = 128;                       // columns of one warp
constexpr int kBlasTA = 1024;                        // limbs of A staged at a time
constexpr int kBlasWin = kBlasTA + kWarpCols + 32;   // limbs of B's window
struct BlasWarpSmem {
    uint32_t A[kBlasTA + 4];
    uint32_t B[kBlasWin];
};
static_assert((kBlasTA + 4) % 4 == 0 && kBlasWin % 4 == 0, "16-byte rows");
// B'[j] sits at window index j + kBlasTA + 15 - c0 + a0: the index of
// j = w0 - a - 3 is then a multiple of 4 for w0, c0, a, a0 multiples of 4.
__device__ __forceinline__ int blas_win_off(int c0, int a0) { return kBlasTA + 15 - c0 + a0; }

// A[a0, a0 + kBlasTA) (zeros from lenA) and the window of B' (B'[j] = B[j -
// boff], zeros outside [boff, boff + lenB)) for the warp's columns from c0.
__device__ __forceinline__ void blas_stage(BlasWarpSmem &sm, const uint32_t *__restrict__ A, int lenA,
                                           const uint32_t *__restrict__ B, int lenB, int boff, int c0, int a0,
                                           int lane) {
    for (int e = lane; e < kBlasTA + 4; e += 32) {
        const int a = a0 + e;
        sm.A[e] = a < lenA ? A[a] : 0u;
    }
    const int jb = c0 - a0 - kBlasTA - 15 - boff;  // window entry e holds B[jb + e]
    for (int e = lane; e < kBlasWin; e += 32) {
        const int j = jb + e;
        sm.B[e] = (j >= 0 && j < lenB) ? B[j] : 0u;
    }
}

__device__ __forceinline__ uint4 lds4(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }

// acc[q] += sum_{a = a_lo}^{a_hi + 3} A[a] B'[w0 + q - a], q < 4 (a_lo a
// multiple of 4, a_hi <= a0 + kBlasTA - 1; products past the operands' ends
// meet the zero padding).  Window: win[k] = B'[w0 - a - 3 + k].
__device__ __forceinline__ void conv4x4(const uint32_t *A_s, const uint32_t *B_s, int w0, int c0, int a0, int a_lo,
                                        int a_hi, uint32_t (&acc)[4][3]) {
    int wb = w0 - a_lo - 3 + blas_win_off(c0, a0);
    const uint4 l4 = lds4(B_s + wb), h4 = lds4(B_s + wb + 4);
    uint32_t win[8] = {l4.x, l4.y, l4.z, l4.w, h4.x, h4.y, h4.z, h4.w};
    for (int a = a_lo; a <= a_hi; a += 4) {
        const uint4 av = lds4(A_s + (a - a0));
        const uint32_t ar[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) mac96(acc[q][0], acc[q][1], acc[q][2], ar[r], win[q - r + 3]);
        wb -= 4;
        const uint4 nw = lds4(B_s + wb);
        win[7] = win[3];
        win[6] = win[2];
        win[5] = win[1];
        win[4] = win[0];
        win[0] = nw.x;
        win[1] = nw.y;
        win[2] = nw.z;
        win[3] = nw.w;
    }
}
// The warp's columns of one product A * B' (every staging of A it meets).
__device__ __forceinline__ void warp_row_conv(BlasWarpSmem &sm, const uint32_t *__restrict__ A, int lenA,
                                              const uint32_t *__restrict__ B, int lenB, int boff, int c0, int W,
                                              int lane, uint32_t (&acc)[4][3]) {
    const int w0 = c0 + 4 * lane;
    const int LB = boff + lenB;
    for (int a0 = 0; a0 < lenA; a0 += kBlasTA) {
        if (a0 > c0 + kWarpCols - 1 || a0 + kBlasTA - 1 < c0 - (LB - 1)) continue;  // warp-uniform
        __syncwarp();  // the previous products' reads are done
        blas_stage(sm, A, lenA, B, lenB, boff, c0, a0, lane);
        __syncwarp();
        const int a_lo = max(a0, w0 - (LB - 1)) & ~3;
        const int a_hi = min(min(a0 + kBlasTA, lenA) - 1, w0 + 3);
        if (w0 < W && a_lo <= a_hi) conv4x4(sm.A, sm.B, w0, c0, a0, a_lo, a_hi, acc);
    }
}
__device__ __forceinline__ void add_signed(__int128 (&tot)[4], const uint32_t (&acc)[4][3], bool neg) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __int128 v = static_cast<__int128>((static_cast<unsigned __int128>(acc[q][2]) << 64) |
                                                 (static_cast<unsigned __int128>(acc[q][1]) << 32) | acc[q][0]);
        tot[q] += neg ? -v : v;
    }
}

// partial[c][w] = sum over rows i of chunk c of s_i * sum_a X_i[a] Y_i[w - a]
// (s_i = +-1 from the two signs), for limb columns w in [0, 2 L32): one warp
// per (chunk, slice of 128 columns).
__global__ void __launch_bounds__(32 * kBlasWarps) k_dot_partial(const uint32_t *__restrict__ x,
                                                                  const uint8_t *__restrict__ xn,
                                                                  const uint32_t *__restrict__ y,
                                                                  const uint8_t *__restrict__ yn, int n, int L32,
                                                                  int slices, int chunks,
                                                                  __int128 *__restrict__ partial) {
    __shared__ __align__(16) BlasWarpSmem sm[kBlasWarps];
    const int warp = static_cast<int>(threadIdx.x >> 5), lane = static_cast<int>(threadIdx.x & 31);
    const long long task = static_cast<long long>(blockIdx.x) * kBlasWarps + warp;
    if (task >= static_cast<long long>(chunks) * slices) return;  // the whole warp; no block barrier follows
    const int c = static_cast<int>(task / slices), c0 = static_cast<int>(task % slices) * kWarpCols;
    const int W = 2 * L32, w0 = c0 + 4 * lane;
    const int i0 = c * kDotRows, i1 = min(n, i0 + kDotRows);
    __int128 tot[4] = {0, 0, 0, 0};
    for (int i = i0; i < i1; ++i) {
        uint32_t acc[4][3] = {};
        warp_row_conv(sm[warp], x + static_cast<size_t>(i) * L32, L32, y + static_cast<size_t>(i) * L32, L32, 0, c0,
                      W, lane, acc);
        add_signed(tot, acc, xn[i] != yn[i]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (w0 + q < W) partial[static_cast<size_t>(c) * W + w0 + q] = tot[q];
}

// The inner product as one dense product on the tensor cores, for large
// n and b: every entry is cut into D >= ceil(32 L32 / 6) digits of 6 bits
// carrying its sign (|d| <= 63, exact in bf16), X and Y as n x D digit
// matrices, and C = X^T Y (D x D, C[s][t] = sum_i X_i[s] Y_i[t]) by cuBLAS in
// chunks of 4096 rows, so that every fp32 partial sum is an integer below
// 4096 * 63^2 < 2^24 and exact in any order (7-bit digits allow chunks of
// 1024 rows only: at n = 8000, b = 33220 eight GEMMs and eight D x D outputs
// instead of two, 1.00 against 0.75 ms).  The product's digit column u
// is the sum of C along the anti-diagonal s + t = u (int64), which becomes
// the 128-bit limb column sums of the schoolbook kernels.
constexpr int kDig = 6;               // bits of a digit
constexpr int kGemmRows = 4096;       // rows of one exact fp32 GEMM chunk
constexpr int kGemmMaxDigits = 8192;  // larger D: the CUDA-core kernel (C would pass 256 MB)
constexpr int kDigMax = (1 << kDig) - 1;
static_assert(static_cast<long long>(kGemmRows) * kDigMax * kDigMax < (1LL << 24), "exact fp32 chunk sums");

__global__ void k_digit_planes(const uint32_t *__restrict__ limbs, const uint8_t *__restrict__ neg, int n, int L32, int D,
                          __nv_bfloat16 *__restrict__ out) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(n) * D) return;
    const int i = static_cast<int>(idx / D), s = static_cast<int>(idx - static_cast<long long>(i) * D);
    const int bit = kDig * s, w = bit >> 5, r = bit & 31;
    int d = 0;  // the padding digits past the entry's 32 L32 bits are 0
    if (w < L32) {
        const uint32_t *row = limbs + static_cast<size_t>(i) * L32;
        uint64_t v = row[w];
        if (w + 1 < L32) v |= static_cast<uint64_t>(row[w + 1]) << 32;
        d = static_cast<int>((v >> r) & static_cast<uint64_t>(kDigMax));
    }
    out[idx] = __int2bfloat16_rn(neg[i] ? -d : d);
}

// z[u] += sum over a 32 x 32 tile of C (column-major, D x D, fp32 holding
// integers below 2^24) of the entries with s + t = u: the tile is written
// skewed into shared memory (entry (s, t) in row s + t, padded rows of 33:
// both passes conflict-free), one thread sums a row (32 entries: below 2^29,
// int32), one global 64-bit atomic per anti-diagonal of the tile.
__global__ void __launch_bounds__(256) k_antidiag(const float *__restrict__ C, int D, unsigned long long *__restrict__ z) {
    __shared__ int32_t sk[63 * 33];
    const int s0 = static_cast<int>(blockIdx.x) * 32, t0 = static_cast<int>(blockIdx.y) * 32;
    const int tx = static_cast<int>(threadIdx.x & 31), ty = static_cast<int>(threadIdx.x >> 5);
    for (int e = threadIdx.x; e < 63 * 33; e += blockDim.x) sk[e] = 0;
    __syncthreads();
    const int s = s0 + tx;
    for (int j = ty; j < 32; j += 8) {  // column t0 + j of the tile: tx + j is its anti-diagonal
        const int t = t0 + j;
        if (s < D && t < D) sk[(tx + j) * 33 + j] = static_cast<int32_t>(C[s + static_cast<size_t>(t) * D]);
    }
    __syncthreads();
    if (threadIdx.x < 63) {
        const int k = static_cast<int>(threadIdx.x);
        long long v = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) v += sk[k * 33 + j];
        if (v) atomicAdd(z + s0 + t0 + k, static_cast<unsigned long long>(v));  // two's complement: signed sum
    }
}

// cols[w] = sum of z[u] 2^(6u - 32w) over the digit columns u whose bit 6u
// lies in limb column w.
__global__ void k_digits_to_cols(const long long *__restrict__ z, int nz, int W, __int128 *__restrict__ cols) {
    const int w = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    if (w >= W) return;
    __int128 acc = 0;
    const int u_lo = (32 * w + kDig - 1) / kDig, u_hi = min(nz - 1, (32 * w + 31) / kDig);
    for (int u = u_lo; u <= u_hi; ++u) acc += static_cast<__int128>(z[u]) << (kDig * u - 32 * w);
    cols[w] = acc;
}

// The linear combination's large terms on the tensor cores: for scalar c (the
// host's shifted limbs, Dc digits) and all rows x_i, the products c x_i are
// the rows of T X^T with T the (Dc + D - 1) x D Toeplitz matrix of c's
// digits (T[u][s] = c_(u-s)), by cuBLAS in 4096-digit chunks of the inner
// dimension (exact fp32 sums, as the inner product's); each chunk's digit
// columns are folded into the 128-bit limb column sums of the rows, moved up
// by the term's limb offset.
__global__ void k_toeplitz(const uint32_t *__restrict__ c, int nl, int neg, int Dc, int D, int Up,
                           __nv_bfloat16 *__restrict__ T) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(Up) * D) return;
    const int sidx = static_cast<int>(idx / Up), u = static_cast<int>(idx - static_cast<long long>(sidx) * Up);
    const int v = u - sidx;  // digit of c at this entry
    int d = 0;
    if (v >= 0 && v < Dc) {
        const int bit = kDig * v, w = bit >> 5, r = bit & 31;
        if (w < nl) {
            uint64_t x = c[w];
            if (w + 1 < nl) x |= static_cast<uint64_t>(c[w + 1]) << 32;
            d = static_cast<int>((x >> r) & static_cast<uint64_t>(kDigMax));
        }
    }
    T[idx] = __int2bfloat16_rn(neg ? -d : d);
}
// cols[i][w] += sum of Cm[u][i] 2^(6u - 32 (w - off)) over the digit columns u
// (< U) of the term's own limb column w - off.
__global__ void k_term_cols(const float *__restrict__ Cm, int Up, int U, int n, int off, int W,
                            __int128 *__restrict__ cols) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(n) * W) return;
    const int i = static_cast<int>(idx / W), w = static_cast<int>(idx - static_cast<long long>(i) * W);
    const int wl = w - off;
    if (wl < 0) return;
    const int u_lo = (32 * wl + kDig - 1) / kDig, u_hi = min(U - 1, (32 * wl + 31) / kDig);
    if (u_lo > u_hi) return;
    const float *col = Cm + static_cast<size_t>(i) * Up;
    __int128 acc = 0;
    for (int u = u_lo; u <= u_hi; ++u)
        acc += static_cast<__int128>(static_cast<long long>(col[u])) << (kDig * u - 32 * wl);
    cols[idx] += acc;
}

// One cuBLAS handle per host thread and device (a handle is not shared
// between threads); made on first use and kept for the process.
cublasHandle_t blas_handle() {
    thread_local cublasHandle_t handles[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!handles[dev] && cublasCreate(&handles[dev]) != CUBLAS_STATUS_SUCCESS) handles[dev] = nullptr;
    return handles[dev];
}

// out[w] = sum_c partial[c][w]; a block of 32 x 8 threads covers 32 columns,
// the 8 lanes of a column take every 8th chunk and meet in shared memory.
__global__ void __launch_bounds__(256) k_dot_reduce(const __int128 *__restrict__ partial, int chunks, int W,
                                                    __int128 *__restrict__ out) {
    __shared__ __int128 red[8][32];
    const int w = blockIdx.x * 32 + threadIdx.x;
    __int128 s = 0;
    if (w < W)
        for (int c = threadIdx.y; c < chunks; c += 8) s += partial[static_cast<size_t>(c) * W + w];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && w < W) {
#pragma unroll
        for (int l = 1; l < 8; ++l) s += red[l][threadIdx.x];
        out[w] = s;
    }
}

// Up to three terms c_k x_k: scalar k has nl[k] limbs (already shifted left by
// its bit residue), sign sneg[k], and enters at limb offset off[k].
struct LinTerms {
    const uint32_t *x[3];
    const uint8_t *xn[3];
    const uint32_t *c[3];  // device copies of the scalar limbs
    int nl[3], off[3], sneg[3];
    int count;
};

// colsum[i][w] = sum_k sign * sum_a C_k[a] X_k,i[w - off_k - a]; grid (rows,
// column blocks), four consecutive columns per thread with a sliding window
// of X limbs (as the inner product); the scalar limbs are read by every
// thread of a block and stay in the read-only cache.
__global__ void k_lincomb_colsum(LinTerms t, int n, int L32, int W, __int128 *__restrict__ colsum) {
    const int i = blockIdx.x;
    const int w0 = 4 * (blockIdx.y * blockDim.x + threadIdx.x);
    if (i >= n || w0 >= W) return;
    __int128 tot[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k >= t.count) break;
        const int v0 = w0 - t.off[k];  // first column within C_k * X_k,i
        if (v0 + 3 < 0) continue;
        unsigned __int128 v[4];
        cols4(t.c[k], t.nl[k], t.x[k] + static_cast<size_t>(i) * L32, L32, v0, v);
        const bool neg = (t.xn[k][i] != 0) != (t.sneg[k] != 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) tot[q] += neg ? -static_cast<__int128>(v[q]) : static_cast<__int128>(v[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (w0 + q < W) colsum[static_cast<size_t>(i) * W + w0 + q] = tot[q];
}

// Consecutive 256-byte aligned pieces of one buffer.
struct Carve {
    size_t off = 0;
    template <class T>
    T *take(void *base, size_t count) {
        T *p = base ? reinterpret_cast<T *>(static_cast<char *>(base) + off) : nullptr;
        off += (count * sizeof(T) + 255) / 256 * 256;
        return p;
    }
};

bool device_vec(const hmv_vec *v, int n, int b) {
    return v && v->len == n && v->nrhs == 1 && v->b == b && v->limbs && v->neg && v->on_device == 1 && !v->reserved;
}

}  // namespace
}  // namespace hmv

using namespace hmv;

extern "C" hmv_status hmv_dot(hmv_plan_t *p, const hmv_vec *x, const hmv_vec *y, uint32_t *z, int32_t zl,
                              uint8_t *z_neg) {
    if (!p || !z || !z_neg) return HMV_EINVAL;
    const int n = p->n, L32 = p->L32, W = 2 * L32;
    if (!device_vec(x, n, p->b) || !device_vec(y, n, p->b) || zl < W + 2) return HMV_EINVAL;
    const int chunks = (n + kDotRows - 1) / kDotRows;
    // digits of an entry, padded with zero digits to a multiple of 32 (16-byte
    // aligned leading dimensions for the tensor-core GEMM kernels)
    const int D = ((32 * L32 + kDig - 1) / kDig + 31) / 32 * 32;
    // the dense product pays for its D x D matrix from about 2^26 limb products on
    const bool dense = D <= kGemmMaxDigits && static_cast<double>(n) * L32 * L32 >= 67108864.0;
    const bool same = x->limbs == y->limbs && x->neg == y->neg;
    cudaStream_t s = p->stream;
    __int128 *partial = nullptr, *cols = nullptr;
    __nv_bfloat16 *xd = nullptr, *yd = nullptr;
    float *cm = nullptr;
    long long *zd = nullptr;
    uint32_t *mag = nullptr;
    uint8_t *zn = nullptr;
    int32_t *zb = nullptr, *st = nullptr;
    const int ZW = W + 2;
    const int NZ = 2 * D + 64;  // digit columns (2D - 1) and the tiles' overhang
    // working memory from the plan (allocated by the first call, reused after)
    auto carve = [&](void *base) {
        Carve c;
        if (dense) {
            xd = c.take<__nv_bfloat16>(base, static_cast<size_t>(n) * D);
            yd = same ? xd : c.take<__nv_bfloat16>(base, static_cast<size_t>(n) * D);
            cm = c.take<float>(base, static_cast<size_t>(D) * D);
            zd = c.take<long long>(base, NZ);
        } else {
            partial = c.take<__int128>(base, static_cast<size_t>(chunks) * W);
        }
        cols = c.take<__int128>(base, W);
        mag = c.take<uint32_t>(base, ZW);
        zn = c.take<uint8_t>(base, 16);
        zb = c.take<int32_t>(base, 4);
        st = c.take<int32_t>(base, 8);
        return c.off;
    };
    cudaError_t e = grow(p->dot_buf, carve(nullptr), p->stream);
    if (e == cudaSuccess) {
        carve(p->dot_buf.ptr);
        e = cudaMemsetAsync(st, 0, 8 * sizeof(int32_t), s);
    }
    if (e == cudaSuccess && dense) {
        cublasHandle_t h = blas_handle();
        if (!h || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) e = cudaErrorUnknown;
        const long long nd = static_cast<long long>(n) * D;
        if (e == cudaSuccess) {
            k_digit_planes<<<static_cast<unsigned>((nd + 255) / 256), 256, 0, s>>>(x->limbs, x->neg, n, L32, D, xd);
            if (!same)
                k_digit_planes<<<static_cast<unsigned>((nd + 255) / 256), 256, 0, s>>>(y->limbs, y->neg, n, L32, D, yd);
            e = cudaMemsetAsync(zd, 0, NZ * sizeof(long long), s);
            p->launches_total += same ? 1 : 2;
        }
        const float one = 1.0f, zero = 0.0f;
        const dim3 tiles((D + 31) / 32, (D + 31) / 32);
        for (int c0 = 0; c0 < n && e == cudaSuccess; c0 += kGemmRows) {
            const int kc = std::min(kGemmRows, n - c0);
            // C (D x D, column-major) = Xc Yc^T over the chunk's rows (digit-major rows: column-major D x kc)
            if (cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_T, D, D, kc, &one, xd + static_cast<size_t>(c0) * D,
                             CUDA_R_16BF, D, yd + static_cast<size_t>(c0) * D, CUDA_R_16BF, D, &zero, cm, CUDA_R_32F,
                             D, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS) {
                e = cudaErrorUnknown;
                break;
            }
            k_antidiag<<<tiles, 256, 0, s>>>(cm, D, reinterpret_cast<unsigned long long *>(zd));
            p->launches_total += 1;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_digits_to_cols<<<(W + 127) / 128, 128, 0, s>>>(zd, 2 * D - 1, W, cols);
            e = launch_colsum_normalize_cols(cols, 1, W, mag, zn, zb, ZW, st, s);
            p->launches_total += 2;
        }
    } else if (e == cudaSuccess) {
        const int slices = (W + kWarpCols - 1) / kWarpCols;
        const long long tasks = static_cast<long long>(slices) * chunks;
        k_dot_partial<<<static_cast<unsigned>((tasks + kBlasWarps - 1) / kBlasWarps), 32 * kBlasWarps, 0, s>>>(
            x->limbs, x->neg, y->limbs, y->neg, n, L32, slices, chunks, partial);
        k_dot_reduce<<<(W + 31) / 32, dim3(32, 8), 0, s>>>(partial, chunks, W, cols);
        e = launch_colsum_normalize_cols(cols, 1, W, mag, zn, zb, ZW, st, s);
        p->launches_total += 3;
    }
    int32_t status[8] = {0};
    uint8_t sign = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, mag, static_cast<size_t>(ZW) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sign, zn, 1, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, st, sizeof status, cudaMemcpyDeviceToHost, s);
    const cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? HMV_ENOMEM : HMV_ECUDA; }
    if (status[0] != DEV_OK) return HMV_EINTERNAL;
    for (int w = ZW; w < zl; ++w) z[w] = 0;
    *z_neg = sign;
    return HMV_OK;
}

extern "C" hmv_status hmv_lincomb(hmv_plan_t *p, int32_t count, const hmv_scalar *c, const hmv_vec *xs, hmv_vec *y) {
    if (!p || !c || !xs || !y || count < 1 || count > 3) return HMV_EINVAL;
    const int n = p->n, b = p->b, L32 = p->L32;
    if (!device_vec(y, n, b)) return HMV_EINVAL;
    // term k: value C_k * M_k,i * 2^(s_k), s_k = c_k.exponent + x_k.exponent - b
    long long smin = 0;
    for (int k = 0; k < count; ++k) {
        if (!device_vec(&xs[k], n, b) || !c[k].limbs || c[k].nlimbs < 1 || c[k].nlimbs > L32 + 1) return HMV_EINVAL;
        const long long sk = static_cast<long long>(c[k].exponent) + xs[k].exponent - b;
        smin = (k == 0) ? sk : std::min(smin, sk);
    }
    LinTerms t;
    memset(&t, 0, sizeof t);
    t.count = count;
    std::vector<std::vector<uint32_t>> shifted(count);
    int W = 0;
    for (int k = 0; k < count; ++k) {
        const long long shift = static_cast<long long>(c[k].exponent) + xs[k].exponent - b - smin;
        if (shift > 4LL * 32 * L32) return HMV_EUNSUPPORTED;  // terms too far apart in scale
        const int off = static_cast<int>(shift / 32), r = static_cast<int>(shift % 32);
        std::vector<uint32_t> &v = shifted[k];  // C_k << r
        v.assign(c[k].nlimbs + 1, 0u);
        for (int q = 0; q < c[k].nlimbs; ++q) {
            const uint64_t wv = static_cast<uint64_t>(c[k].limbs[q]) << r;
            v[q] |= static_cast<uint32_t>(wv);
            v[q + 1] |= static_cast<uint32_t>(wv >> 32);
        }
        while (v.size() > 1 && v.back() == 0) v.pop_back();
        t.x[k] = xs[k].limbs;
        t.xn[k] = xs[k].neg;
        t.nl[k] = static_cast<int>(v.size());
        t.off[k] = off;
        t.sneg[k] = c[k].neg ? 1 : 0;
        W = std::max(W, off + t.nl[k] + L32);
    }
    W += 1;
    const int ZW = W + 3;
    cudaStream_t s = p->stream;
    // terms with large scalars on large problems go to the tensor cores (as
    // the inner product's dense path), the others to the CUDA-core kernel
    const int D = ((32 * L32 + kDig - 1) / kDig + 31) / 32 * 32;
    bool dense[3] = {false, false, false};
    int Upmax = 0;
    for (int k = 0; k < count; ++k) {
        dense[k] = D <= kGemmMaxDigits && t.nl[k] >= 64 &&
                   static_cast<double>(n) * L32 * t.nl[k] >= 67108864.0;
        if (dense[k]) Upmax = std::max(Upmax, ((32 * t.nl[k] + kDig - 1) / kDig + D - 1 + 31) / 32 * 32);
    }
    const bool any_dense = Upmax > 0;
    uint32_t *dc = nullptr, *mag = nullptr;
    __int128 *cols = nullptr;
    uint8_t *zn = nullptr;
    int32_t *zb = nullptr, *st = nullptr;
    __nv_bfloat16 *xd = nullptr, *tm = nullptr;
    float *cm = nullptr;
    int total = 0;
    for (int k = 0; k < count; ++k) total += t.nl[k];
    // working memory from the plan (grown when a call needs more, reused after)
    auto carve = [&](void *base) {
        Carve c;
        dc = c.take<uint32_t>(base, total);
        cols = c.take<__int128>(base, static_cast<size_t>(n) * W);
        mag = c.take<uint32_t>(base, static_cast<size_t>(n) * ZW);
        zn = c.take<uint8_t>(base, n);
        zb = c.take<int32_t>(base, n);
        st = c.take<int32_t>(base, 8);
        if (any_dense) {
            xd = c.take<__nv_bfloat16>(base, static_cast<size_t>(n) * D);
            tm = c.take<__nv_bfloat16>(base, static_cast<size_t>(Upmax) * D);
            cm = c.take<float>(base, static_cast<size_t>(Upmax) * n);
        }
        return c.off;
    };
    cudaError_t e = grow(p->lin_buf, carve(nullptr), p->stream);
    if (e == cudaSuccess) carve(p->lin_buf.ptr);
    std::vector<uint32_t> flat;
    for (int k = 0; k < count; ++k) flat.insert(flat.end(), shifted[k].begin(), shifted[k].end());
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, flat.data(), flat.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, 8 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        int o = 0;
        for (int k = 0; k < count; ++k) {
            t.c[k] = dc + o;
            o += t.nl[k];
        }
        // the small terms write every column sum (all zero without them) ...
        LinTerms ts;
        memset(&ts, 0, sizeof ts);
        for (int k = 0; k < count; ++k) {
            if (dense[k]) continue;
            const int j = ts.count++;
            ts.x[j] = t.x[k];
            ts.xn[j] = t.xn[k];
            ts.c[j] = t.c[k];
            ts.nl[j] = t.nl[k];
            ts.off[j] = t.off[k];
            ts.sneg[j] = t.sneg[k];
        }
        if (ts.count > 0) {
            k_lincomb_colsum<<<dim3(n, (W / 4 + 127) / 128 + 1), 128, 0, s>>>(ts, n, L32, W, cols);  // 4 columns/thread
            p->launches_total++;
            e = cudaGetLastError();
        } else {
            e = cudaMemsetAsync(cols, 0, static_cast<size_t>(n) * W * sizeof(__int128), s);
        }
        // ... and the large ones add theirs
        cublasHandle_t h = any_dense ? blas_handle() : nullptr;
        if (e == cudaSuccess && any_dense && (!h || cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS)) e = cudaErrorUnknown;
        const float one = 1.0f, zero = 0.0f;
        const long long nd = static_cast<long long>(n) * D;
        for (int k = 0; k < count && e == cudaSuccess; ++k) {
            if (!dense[k]) continue;
            const int Dc = (32 * t.nl[k] + kDig - 1) / kDig, U = Dc + D - 1, Up = (U + 31) / 32 * 32;
            k_digit_planes<<<static_cast<unsigned>((nd + 255) / 256), 256, 0, s>>>(t.x[k], t.xn[k], n, L32, D, xd);
            const long long nt = static_cast<long long>(Up) * D;
            k_toeplitz<<<static_cast<unsigned>((nt + 255) / 256), 256, 0, s>>>(t.c[k], t.nl[k], t.sneg[k], Dc, D, Up,
                                                                              tm);
            p->launches_total += 2;
            for (int k0 = 0; k0 < D && e == cudaSuccess; k0 += kGemmRows) {
                const int kc = std::min(kGemmRows, D - k0);
                // Cm (Up x n, column-major) = T[:, k0:k0+kc] X[:, k0:k0+kc]^T
                if (cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, Up, n, kc, &one, tm + static_cast<size_t>(k0) * Up,
                                 CUDA_R_16BF, Up, xd + k0, CUDA_R_16BF, D, &zero, cm, CUDA_R_32F, Up,
                                 CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS) {
                    e = cudaErrorUnknown;
                    break;
                }
                const long long nw = static_cast<long long>(n) * W;
                k_term_cols<<<static_cast<unsigned>((nw + 255) / 256), 256, 0, s>>>(cm, Up, U, n, t.off[k], W, cols);
                p->launches_total++;
                e = cudaGetLastError();
            }
        }
        // value = S * 2^smin = S * 2^(e_in - 2b)
        if (e == cudaSuccess)
            e = launch_colsum_round_cols(cols, n, W, L32, mag, zn, zb, ZW, st, b, static_cast<int>(smin + 2LL * b),
                                         y->limbs, y->neg, s);
        p->launches_total += 3;
    }
    int32_t status[8] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, st, sizeof status, cudaMemcpyDeviceToHost, s);
    const cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? HMV_ENOMEM : HMV_ECUDA; }
    if (status[0] != DEV_OK) return HMV_EINTERNAL;
    y->exponent = status[3];
    return HMV_OK;
}
