// Digit-plane kernels of the Karatsuba-style Hankel product (Beliakov,
// arXiv:1402.5287, Sec. 3, Algorithm 1) and the final rounding.
//
// Representation: every operand in the recursion tree is a signed integer
// held as Dl balanced radix-2^8 digits d_u in [-128, 127] (value
// sum_u d_u 256^u), one int8 per digit, Dp (>= Dl, multiple of 16) digits per
// row.  Sums and differences of Algorithm 1 are formed digit-wise and
// renormalised with an exact carry chain, so every intermediate is exact.
#include <cuda_bf16.h>

#include <type_traits>

#include "hmv_carry.cuh"
#include "hmv_internal.h"

namespace hmv {

namespace {

constexpr int kThreads = 256;

// Per-plan buffers of a group of plans with the same geometry (the products
// of a digit split), one launch for all of them: blockIdx.y (z for
// pack_vector) selects the plan.  A single plan is a group of one.
constexpr int kMaxGroup = 16;  // plans per grouped launch (the 15 Toom-8 products)
struct PlanPtrs {
    const void *in[kMaxGroup];
    const void *in2[kMaxGroup];
    void *out[kMaxGroup];
};

inline int blocks_for(long long work, int threads = kThreads) {
    return static_cast<int>((work + threads - 1) / threads);
}


// Four balanced digits in one word, a little-endian byte each (two's
// complement, [-128, 127]): their value sum_i d_i 256^i is the unsigned
// reading U less 256^(i+1) for every negative digit, U - 2 (U & 0x80808080).
__device__ __forceinline__ long long word_value(uint32_t w) {
    return static_cast<long long>(w) - 2 * static_cast<long long>(w & 0x80808080u);
}
// v + carry (|v| < 2^33) written as four balanced digits and a new carry:
// adding 128 to every digit position makes each digit plus 128 a byte in
// [0, 255], so the low word of v + carry + 0x80808080 holds them (XOR 0x80
// takes each back to d_i) and the bits above it are the carry out.  The
// balanced representation is unique, so this is the digit-by-digit chain.
__device__ __forceinline__ uint32_t balanced_word(long long v, long long &carry) {
    const long long t = v + carry + 0x80808080LL;
    carry = t >> 32;  // arithmetic: floor
    return static_cast<uint32_t>(t) ^ 0x80808080u;
}

__device__ __forceinline__ uint16_t bf16_bits_of_small_int(int v) {
    // integers with |v| <= 256 are exact in bf16: the float has zero low bits
    return static_cast<uint16_t>(__float_as_uint(static_cast<float>(v)) >> 16);
}

__device__ __forceinline__ void warp_balance(int (&d)[kDigitsPerLane], int lane, int &wcarry) {
    warp_carry<true, int>(d, lane, wcarry);
}

// Store a lane's digits [ub, ub + kDigitsPerLane) of a Dp-digit int8 row;
// digits at or past Dp must be zero (else the row overflowed).
__device__ __forceinline__ void store_lane_digits(const int (&d)[kDigitsPerLane], int ub, int Dp, int8_t *o,
                                                  int32_t *dstat) {
#pragma unroll
    for (int q = 0; q < kDigitsPerLane; ++q)
        if (ub + q >= Dp && d[q] != 0) set_status(dstat, DEV_OVERFLOW);
#pragma unroll
    for (int h = 0; h < kDigitsPerLane / 16; ++h) {
        const int uh = ub + 16 * h;  // Dp is a multiple of 16
        if (uh >= Dp) break;
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            pk[q] = (static_cast<uint32_t>(d[16 * h + 4 * q]) & 0xFFu) |
                    ((static_cast<uint32_t>(d[16 * h + 4 * q + 1]) & 0xFFu) << 8) |
                    ((static_cast<uint32_t>(d[16 * h + 4 * q + 2]) & 0xFFu) << 16) |
                    ((static_cast<uint32_t>(d[16 * h + 4 * q + 3]) & 0xFFu) << 24);
        *reinterpret_cast<uint4 *>(o + uh) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// ------------------------------------------------------------------ encode
// Sign-magnitude limbs -> balanced digits (the number representation of
// Sec. 2, a = sum_k B^k a_k, with base B = 2^8 and signed digits).
// circ_n > 0: row k takes entry (circ_n - 1 - k) mod circ_n (circulant ->
// Toeplitz sequence); otherwise row k takes entry k.
// One warp per row, windows of 32 x kDigitsPerLane digits (8 limbs per lane).
__global__ void __launch_bounds__(256) k_encode(PlanPtrs g, int rows, int L32, int b, int circ_n, int Dp,
                                                int32_t *dstat) {
    const uint32_t *__restrict__ limbs = static_cast<const uint32_t *>(g.in[blockIdx.y]);
    const uint8_t *__restrict__ neg = static_cast<const uint8_t *>(g.in2[blockIdx.y]);
    int8_t *__restrict__ out = static_cast<int8_t *>(g.out[blockIdx.y]);
    const int lane = threadIdx.x & 31;
    const int k = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (k >= rows) return;  // warp-uniform
    int src = k;
    if (circ_n > 0) src = ((circ_n - 1 - k) % circ_n + circ_n) % circ_n;
    const uint32_t *m = limbs + static_cast<size_t>(src) * L32;
    const int topbits = b - 32 * (L32 - 1);
    if (lane == 0 && topbits < 32 && (m[L32 - 1] >> topbits) != 0) set_status(dstat, DEV_BADINPUT);
    const int sgn = neg[src] ? -1 : 1;
    int8_t *o = out + static_cast<size_t>(k) * Dp;
    int wcarry = 0;
    for (int u0 = 0; u0 < Dp; u0 += 32 * kDigitsPerLane) {
        const int ub = u0 + kDigitsPerLane * lane;
        int d[kDigitsPerLane];
#pragma unroll
        for (int q = 0; q < kDigitsPerLane / 4; ++q) {
            const int li = ub / 4 + q;
            const uint32_t w = (li < L32) ? m[li] : 0u;
#pragma unroll
            for (int by = 0; by < 4; ++by) d[4 * q + by] = sgn * static_cast<int>((w >> (8 * by)) & 0xFFu);
        }
        warp_balance(d, lane, wcarry);
        store_lane_digits(d, ub, Dp, o, dstat);
    }
    if (lane == 0 && wcarry != 0) set_status(dstat, DEV_OVERFLOW);
}

// ------------------------------------------------------------------ pre-pass
// One level of Algorithm 1, steps 3-6, for every node of a level.
// Node nu (order s) has children 3nu (c, h -> p), 3nu+1 (d, f -> q),
// 3nu+2 (e, g -> r).  0-based:
//   matrix side  c_k = a_{2k} + a_{2k+1},  d_k = a_{2k+1},  e_k = a_{2k}
//   vector side  h_k = x_{2k},  f_k = x_{2k} - x_{2k+1},  g_k = x_{2k-1} - x_{2k}
// with a_q = 0 for q >= 2s-1 and x_q = 0 for q < 0 or q >= s.
// A block of 128 threads makes 128 consecutive rows k0 .. k0 + 127 of one
// child, each thread one row, its carry chain running over words of four
// balanced digits (balanced_word).  Those rows read parent rows
// 2k0 - 1 .. 2k0 + 255 only, kept in shared memory as even rows E[a] = parent
// 2k0 + 2a and odd rows O[j] = parent 2k0 - 1 + 2j (so that thread a finds
// 2k at E[a], 2k + 1 at O[a + 1] and 2k - 1 at O[a], all conflict-free with an
// 80-byte pitch), 64 digits at a time, loaded coalesced with cp.async into two
// stages: the next 64 digits land while the current carry chains run.  Each
// thread's 64 output digits go to a shared tile that the block then stores
// coalesced.  Parent rows outside the node are zero.  Blocks are ordered
// row block first, so the three children of a parent row block are
// neighbours and share its rows in L2.
constexpr int kPreRows = 128;
constexpr int kPreDig = 64;                 // digits per stage
constexpr int kPrePitch = kPreDig + 16;     // bytes per staged row: an odd number of 16-byte units
constexpr int kPrePieces = kPreDig / 16;    // 16-byte pieces per staged row
constexpr int kPreStage = (kPreRows + kPreRows + 1) * kPrePitch;
constexpr int kPreSmem = 2 * kPreStage + kPreRows * kPrePitch;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int src_bytes = valid ? 16 : 0;  // 0: the 16 bytes are filled with zeros, nothing is read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(kPreRows) k_prepass_staged(PlanPtrs g, int in_rows, const int *__restrict__ in_size,
                                                            int out_rows, const int *__restrict__ out_size,
                                                            int nchildren, int Dp, int matrix_side, int32_t *dstat) {
    extern __shared__ __align__(16) uint8_t pre_smem[];
    const int8_t *__restrict__ in = static_cast<const int8_t *>(g.in[blockIdx.y]);
    int8_t *__restrict__ out = static_cast<int8_t *>(g.out[blockIdx.y]);
    const int child = blockIdx.x % nchildren, rb = blockIdx.x / nchildren;
    const int parent = child / 3, t = child % 3;
    const int s = in_size[parent];
    const int cs = out_size[child];
    const int cnt = matrix_side ? 2 * cs - 1 : cs;
    const int k0 = rb * kPreRows;
    if (k0 >= cnt) return;  // the whole block
    const int len = matrix_side ? 2 * s - 1 : s;
    // which parent rows the child reads: 2k (even set), 2k+1 and 2k-1 (odd set)
    const bool needE = !(matrix_side && t == 1);
    const bool needO = matrix_side ? (t != 2) : (t != 0);
    const int8_t *pbase = in + static_cast<size_t>(parent) * in_rows * Dp;
    const int tid = threadIdx.x;
    auto stage_in = [&](int st, int u0) {
        uint8_t *E = pre_smem + st * kPreStage;
        uint8_t *O = E + kPreRows * kPrePitch;
        // 16-byte pieces (row, piece), even rows first
        const int nE = needE ? kPreRows * kPrePieces : 0, nO = needO ? (kPreRows + 1) * kPrePieces : 0;
        for (int c = tid; c < nE + nO; c += kPreRows) {
            const bool even = c < nE;
            const int cc = even ? c : c - nE;
            const int r = cc / kPrePieces, pc = cc % kPrePieces;
            const int q = even ? 2 * k0 + 2 * r : 2 * k0 - 1 + 2 * r;  // parent row
            const int u = u0 + 16 * pc;
            const bool valid = q >= 0 && q < len && u < Dp;
            const int8_t *src = pbase + static_cast<size_t>(valid ? q : 0) * Dp + (valid ? u : 0);
            cp_async16((even ? E : O) + r * kPrePitch + 16 * pc, src, valid);
        }
        cp_async_commit();
    };
    int q1, q2, s1, s2;  // this thread's parent rows and signs, as in k_prepass
    const int k = k0 + tid;
    if (matrix_side) {
        if (t == 0) { q1 = 2 * k; s1 = 1; q2 = 2 * k + 1; s2 = 1; }
        else if (t == 1) { q1 = 2 * k + 1; s1 = 1; q2 = 0; s2 = 0; }
        else { q1 = 2 * k; s1 = 1; q2 = 0; s2 = 0; }
    } else {
        if (t == 0) { q1 = 2 * k; s1 = 1; q2 = 0; s2 = 0; }
        else if (t == 1) { q1 = 2 * k; s1 = 1; q2 = 2 * k + 1; s2 = -1; }
        else { q1 = 2 * k - 1; s1 = 1; q2 = 2 * k; s2 = -1; }
    }
    // staged row of parent q (rows outside the node are zero-filled in shared memory)
    auto srow = [&](int st, int q) -> const uint8_t * {
        const uint8_t *E = pre_smem + st * kPreStage;
        const uint8_t *O = E + kPreRows * kPrePitch;
        const int d = q - 2 * k0;  // -1 .. 255
        return (d & 1) ? O + ((d + 1) >> 1) * kPrePitch : E + (d >> 1) * kPrePitch;
    };
    uint8_t *T = pre_smem + 2 * kPreStage;  // output tile
    long long carry = 0;
    const int nst = (Dp + kPreDig - 1) / kPreDig;
    stage_in(0, 0);
    for (int c = 0; c < nst; ++c) {
        const int u0 = c * kPreDig;
        if (c + 1 < nst) {
            stage_in((c + 1) & 1, u0 + kPreDig);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int st = c & 1;
        const uint8_t *r1 = srow(st, s1 ? q1 : 2 * k0);
        const uint8_t *r2 = srow(st, s2 ? q2 : 2 * k0);
#pragma unroll
        for (int h = 0; h < kPrePieces; ++h) {
            if (u0 + 16 * h >= Dp) break;  // Dp is a multiple of 16: the carry out of digit Dp - 1 is checked
            const uint4 v1 = *reinterpret_cast<const uint4 *>(r1 + 16 * h);
            const uint4 v2 = *reinterpret_cast<const uint4 *>(r2 + 16 * h);
            const uint32_t a1[4] = {v1.x, v1.y, v1.z, v1.w};
            const uint32_t a2[4] = {v2.x, v2.y, v2.z, v2.w};
            uint32_t packed[4];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) packed[qq] = balanced_word(s1 * word_value(a1[qq]) + s2 * word_value(a2[qq]), carry);
            *reinterpret_cast<uint4 *>(T + tid * kPrePitch + 16 * h) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
        __syncthreads();  // the tile is complete, and stage st may be refilled
        for (int pcs = tid; pcs < kPreRows * kPrePieces; pcs += kPreRows) {
            const int r = pcs / kPrePieces, pc = pcs % kPrePieces;
            const int u = u0 + 16 * pc;
            if (k0 + r < cnt && u < Dp)
                *reinterpret_cast<uint4 *>(out + (static_cast<size_t>(child) * out_rows + k0 + r) * Dp + u) =
                    *reinterpret_cast<const uint4 *>(T + r * kPrePitch + 16 * pc);
        }
    }
    if (k < cnt && carry != 0) set_status(dstat, DEV_OVERFLOW);
}

// ------------------------------------------------------------------ packing
// Matrix-side leaves -> bf16 slabs, digits reversed (most significant first)
// and pre-tiled for the tensor cores: hrev[leaf][c][k][kk] holds digit
// (Dp-1-8c-kk) of a_k; rows k >= 2*size-1 are zero.  One 16-byte run per
// (chunk, row), rows adjacent, so any run of rows of one chunk is a block of
// 8-row x 16-byte core matrices.
__global__ void k_pack_matrix(const int8_t *__restrict__ leafd, int rowsA, const int *__restrict__ size,
                              uint16_t *__restrict__ hrev, int RA, int Dp, int nleaves) {
    long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int chunks = Dp / 8;
    long long per_leaf = static_cast<long long>(RA) * chunks;
    int leaf = static_cast<int>(idx / per_leaf);
    if (leaf >= nleaves) return;
    int rem = static_cast<int>(idx % per_leaf);
    int c = rem / RA, k = rem % RA;
    uint16_t v[8];
    if (k < 2 * size[leaf] - 1) {
        const int8_t *src = leafd + (static_cast<size_t>(leaf) * rowsA + k) * Dp + (Dp - 8 * c - 8);
        uint2 raw = *reinterpret_cast<const uint2 *>(src);
        const uint32_t w[2] = {raw.x, raw.y};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int sidx = 7 - i;  // reversed
            int d = static_cast<int8_t>((w[sidx / 4] >> (8 * (sidx % 4))) & 0xFFu);
            v[i] = bf16_bits_of_small_int(d);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0;
    }
    uint4 pk = make_uint4(v[0] | (uint32_t(v[1]) << 16), v[2] | (uint32_t(v[3]) << 16), v[4] | (uint32_t(v[5]) << 16),
                          v[6] | (uint32_t(v[7]) << 16));
    *reinterpret_cast<uint4 *>(hrev + ((static_cast<size_t>(leaf) * chunks + c) * RA + k) * 8) = pk;
}

// Vector-side leaves -> bf16 shifted copies, pre-tiled as 8x8 blocks:
// xg[leaf][j][e][r][kk] = digit (8e + r + kk - 7) of x_j, e in [0, Dp/8 + 1)
// (zero outside [0, Dp) and for j >= size).  Block e is the core matrix of
// every (n-group g, k-group c) with g + c = e - e0 of the digit-Toeplitz
// operand whose window starts at chunk e0.
// One block per (leaf, j, segment of at most kPackSeg chunks): the segment's
// digits are staged once in shared memory, and each thread builds 16-byte
// rows from two aligned 8-byte words (consecutive threads store consecutive
// rows).
constexpr int kPackSeg = 128;
__global__ void __launch_bounds__(128) k_pack_vector(PlanPtrs g, int rowsX, const int *__restrict__ size, int RX,
                                                     int Dp, int seg) {
    const int8_t *__restrict__ leafd = static_cast<const int8_t *>(g.in[blockIdx.z]);
    uint16_t *__restrict__ xg = static_cast<uint16_t *>(g.out[blockIdx.z]);
    __shared__ __align__(16) uint64_t s[kPackSeg + 2];
    const int leaf = blockIdx.x / RX, j = blockIdx.x % RX;
    const int chunks = Dp / 8 + 1;
    const int e0 = blockIdx.y * seg;
    const int ne = min(seg, chunks - e0);
    const bool live = j < size[leaf];
    const int8_t *row = leafd + (static_cast<size_t>(leaf) * rowsX + j) * Dp;
    // s word t holds digits base + 8t .. base + 8t + 7 (zero outside [0, Dp))
    const int base = 8 * e0 - 8;
    for (int t = threadIdx.x; t < ne + 2; t += blockDim.x) {
        const int u = base + 8 * t;  // Dp and u are multiples of 8
        s[t] = (live && u >= 0 && u < Dp) ? *reinterpret_cast<const uint64_t *>(row + u) : 0ull;
    }
    __syncthreads();
    uint4 *out = reinterpret_cast<uint4 *>(xg + ((static_cast<size_t>(leaf) * RX + j) * chunks + e0) * 64);
    for (int q = threadIdx.x; q < 8 * ne; q += blockDim.x) {
        const int el = q >> 3, r = q & 7;
        // digits 8(e0+el) + r - 7 + i (i = 0..7) are bytes r+1 .. r+8 of words el, el+1
        const uint64_t lo = s[el], hi = s[el + 1];
        const int sh = 8 * (r + 1);
        const uint64_t w = (sh == 64) ? hi : ((lo >> sh) | (hi << (64 - sh)));
        uint32_t pk[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int d0 = static_cast<int8_t>((w >> (16 * h)) & 0xFFu);
            const int d1 = static_cast<int8_t>((w >> (16 * h + 8)) & 0xFFu);
            pk[h] = bf16_bits_of_small_int(d0) | (static_cast<uint32_t>(bf16_bits_of_small_int(d1)) << 16);
        }
        out[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// ------------------------------------------------------------------ CUDA-core leaf
// Same output as the tensor-core leaf: for tile (leaf, i0, ub) and row
// i = i0 + blockIdx.y, the column sums Y[i][u] = sum_j sum_s a_{i+j}[s] x_j[u-s]
// for u in [ub*tn, ub*tn+tn), normalised to digits in [0, 256) plus the
// carry out of the block (floor of the block value / 256^tn), tn <= TN.
__global__ void k_leaf_simt(const int8_t *__restrict__ A, int rowsA, const int8_t *__restrict__ X, int rowsX,
                            const int *__restrict__ size, int Dp, int Dl, const Tile *__restrict__ tiles,
                            uint8_t *__restrict__ dig, int32_t *__restrict__ carry, int MT, int Uo, int NUB,
                            int32_t *dstat, int tn) {
    const Tile tl = tiles[blockIdx.x];
    const int m = size[tl.leaf];
    const int i = tl.i0 + blockIdx.y;
    if (i >= m) return;
    __shared__ long long col[TN];
    const int u = tl.ub * tn + threadIdx.x;
    long long acc = 0;
    const int s_lo = max(0, u - (Dl - 1)), s_hi = min(Dl - 1, u);
    for (int j = 0; j < m; ++j) {
        const int8_t *a = A + (static_cast<size_t>(tl.leaf) * rowsA + i + j) * Dp;
        const int8_t *x = X + (static_cast<size_t>(tl.leaf) * rowsX + j) * Dp;
        int part = 0;  // |part| <= Dl * 2^14 < 2^31 for Dl < 2^17
        for (int s = s_lo; s <= s_hi; ++s) part += static_cast<int>(a[s]) * static_cast<int>(x[u - s]);
        acc += part;
    }
    col[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long c = 0;
        uint8_t *o = dig + (static_cast<size_t>(tl.leaf) * MT * TM + i) * Uo + tl.ub * tn;
        for (int q = 0; q < tn; ++q) {
            long long t = col[q] + c;
            o[q] = static_cast<uint8_t>(t & 255);
            c = t >> 8;
        }
        if (c > INT32_MAX || c < INT32_MIN) set_status(dstat, DEV_OVERFLOW);
        carry[(static_cast<size_t>(tl.leaf) * MT * TM + i) * NUB + tl.ub] = static_cast<int32_t>(c);
    }
}

// ------------------------------------------------------------------ leaf normalise
// Joins the per-block digits and block carries of one leaf row into one
// carry-save digit vector with small digits, elementwise: out[u] = dig[u] for
// u < Uo, plus the carry out of block t (a signed 32-bit integer) spread over
// digits (t+1)*tn .. (t+1)*tn + 3 as three base-256 digits and a signed top
// part; out[Uo+4 .. Wo) = 0.  Every digit is then within [-128, 510], so L
// levels of the post-pass keep them within 510 * 2^L (int16 digits while
// L <= 6, else int32); the final normalise propagates all carries.  One block
// per leaf row.
template <class T>
__device__ __forceinline__ void store4(T *o, int g, int4 v);
template <>
__device__ __forceinline__ void store4<int32_t>(int32_t *o, int g, int4 v) {
    reinterpret_cast<int4 *>(o)[g] = v;
}
template <>
__device__ __forceinline__ void store4<int16_t>(int16_t *o, int g, int4 v) {
    reinterpret_cast<uint2 *>(o)[g] = make_uint2((static_cast<uint32_t>(v.x) & 0xFFFFu) | (static_cast<uint32_t>(v.y) << 16),
                                                 (static_cast<uint32_t>(v.z) & 0xFFFFu) | (static_cast<uint32_t>(v.w) << 16));
}
template <class T>
__global__ void k_leaf_normalize(PlanPtrs g, const int *__restrict__ size, int MT, int Uo, int NUB, int rowsX, int Wo,
                                 int tn) {
    const uint8_t *__restrict__ dig = static_cast<const uint8_t *>(g.in[blockIdx.y]);
    const int32_t *__restrict__ carry = static_cast<const int32_t *>(g.in2[blockIdx.y]);
    T *__restrict__ out = static_cast<T *>(g.out[blockIdx.y]);
    const int leaf = blockIdx.x / rowsX, row = blockIdx.x % rowsX;
    if (row >= size[leaf]) return;
    const size_t r = static_cast<size_t>(leaf) * MT * TM + row;
    const uint32_t *d = reinterpret_cast<const uint32_t *>(dig + r * Uo);
    const int32_t *cy = carry + r * NUB;
    T *o = out + (static_cast<size_t>(leaf) * rowsX + row) * Wo;
    for (int g8 = threadIdx.x; g8 < Wo / 8; g8 += blockDim.x) {  // 8 digits per step; Uo, Wo multiples of 8
        const int u0 = 8 * g8;
        const uint2 w = (u0 < Uo) ? reinterpret_cast<const uint2 *>(d)[g8] : make_uint2(0, 0);
        int4 v0 = make_int4(w.x & 0xFF, (w.x >> 8) & 0xFF, (w.x >> 16) & 0xFF, w.x >> 24);
        const int4 v1 = make_int4(w.y & 0xFF, (w.y >> 8) & 0xFF, (w.y >> 16) & 0xFF, w.y >> 24);
        if (u0 > 0 && u0 <= Uo && u0 % tn == 0) {
            const int32_t c = cy[u0 / tn - 1];
            v0.x += c & 0xFF;
            v0.y += (c >> 8) & 0xFF;
            v0.z += (c >> 16) & 0xFF;
            v0.w += c >> 24;  // arithmetic shift: the signed top part
        }
        store4<T>(o, 2 * g8, v0);
        store4<T>(o, 2 * g8 + 1, v1);
    }
}

// The leaf normalise fused into the deepest post-pass level: output rows
// 2k and 2k+1 of a level-(L-1) node are p_k - q_k and p_k + r_k, each leaf
// row read as its block digits plus its block carries spread as above, so
// the carry-save leaf rows are never written out.  Digits of the result are
// within [-638, 1020], as after the two separate kernels.  One block per
// pair of output rows (they share p_k: three leaf rows read, not four).
__device__ __forceinline__ void leaf_digits8(uint2 w, int (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = static_cast<int>((w.x >> (8 * q)) & 0xFF);
        v[4 + q] = static_cast<int>((w.y >> (8 * q)) & 0xFF);
    }
}
__device__ __forceinline__ void add_block_carry(int (&v)[8], int32_t c, int sg) {
    v[0] += sg * (c & 0xFF);
    v[1] += sg * ((c >> 8) & 0xFF);
    v[2] += sg * ((c >> 16) & 0xFF);
    v[3] += sg * (c >> 24);  // arithmetic shift: the signed top part
}
template <class T>
__global__ void k_leaf_post(PlanPtrs g, const int *__restrict__ parent_size, int MT, int Uo, int NUB, int rows_out,
                            int Wo, int tn) {
    const uint8_t *__restrict__ dig = static_cast<const uint8_t *>(g.in[blockIdx.y]);
    const int32_t *__restrict__ carry = static_cast<const int32_t *>(g.in2[blockIdx.y]);
    T *__restrict__ out = static_cast<T *>(g.out[blockIdx.y]);
    const int pairs = (rows_out + 1) / 2;
    const int nu = blockIdx.x / pairs, k = blockIdx.x % pairs;
    const int size = parent_size[nu];
    if (2 * k >= size) return;
    const bool odd = 2 * k + 1 < size;  // the node has output row 2k+1
    size_t r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = static_cast<size_t>(3 * nu + c) * MT * TM + k;  // p_k, q_k, r_k
    T *o0 = out + (static_cast<size_t>(nu) * rows_out + 2 * k) * Wo;
    T *o1 = o0 + Wo;
    for (int g8 = threadIdx.x; g8 < Wo / 8; g8 += blockDim.x) {  // 8 digits per step; Uo, Wo multiples of 8
        const int u0 = 8 * g8;
        const bool in = u0 < Uo;
        int vp[8], vq[8], vr[8];
        leaf_digits8(in ? reinterpret_cast<const uint2 *>(dig + r[0] * Uo)[g8] : make_uint2(0, 0), vp);
        leaf_digits8(in ? reinterpret_cast<const uint2 *>(dig + r[1] * Uo)[g8] : make_uint2(0, 0), vq);
        leaf_digits8(in && odd ? reinterpret_cast<const uint2 *>(dig + r[2] * Uo)[g8] : make_uint2(0, 0), vr);
        if (u0 > 0 && u0 <= Uo && u0 % tn == 0) {
            const int cb = u0 / tn - 1;
            add_block_carry(vp, carry[r[0] * NUB + cb], 1);
            add_block_carry(vq, carry[r[1] * NUB + cb], 1);
            if (odd) add_block_carry(vr, carry[r[2] * NUB + cb], 1);
        }
        store4<T>(o0, 2 * g8, make_int4(vp[0] - vq[0], vp[1] - vq[1], vp[2] - vq[2], vp[3] - vq[3]));
        store4<T>(o0, 2 * g8 + 1, make_int4(vp[4] - vq[4], vp[5] - vq[5], vp[6] - vq[6], vp[7] - vq[7]));
        if (odd) {
            store4<T>(o1, 2 * g8, make_int4(vp[0] + vr[0], vp[1] + vr[1], vp[2] + vr[2], vp[3] + vr[3]));
            store4<T>(o1, 2 * g8 + 1, make_int4(vp[4] + vr[4], vp[5] + vr[5], vp[6] + vr[6], vp[7] + vr[7]));
        }
    }
}

// ------------------------------------------------------------------ post-pass
// Algorithm 1, step 8 (0-based): y_{2k} = p_k - q_k, y_{2k+1} = p_k + r_k,
// digit-wise without carries (digits grow by at most one bit per level).
// One block per output row, 16 bytes of digits per thread and step.
template <class T>
__global__ void k_postpass(PlanPtrs g, int rows_in, int rows_out, const int *__restrict__ parent_size, int Wo) {
    const T *__restrict__ in = static_cast<const T *>(g.in[blockIdx.y]);
    T *__restrict__ out = static_cast<T *>(g.out[blockIdx.y]);
    const int nu = blockIdx.x / rows_out, i = blockIdx.x % rows_out;
    if (i >= parent_size[nu]) return;
    const int k = i >> 1;
    const int other = (i & 1) ? 2 : 1;
    const int4 *p = reinterpret_cast<const int4 *>(in + (static_cast<size_t>(3 * nu) * rows_in + k) * Wo);
    const int4 *o = reinterpret_cast<const int4 *>(in + (static_cast<size_t>(3 * nu + other) * rows_in + k) * Wo);
    int4 *y = reinterpret_cast<int4 *>(out + (static_cast<size_t>(nu) * rows_out + i) * Wo);
    const int groups = Wo * static_cast<int>(sizeof(T)) / 16;  // Wo is a multiple of 8
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int4 a = p[g], b = o[g];
        int4 r;
        if (sizeof(T) == 4) {
            r = (i & 1) ? make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w)
                        : make_int4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        } else {  // two int16 digits per word, no carries between halves
            const int av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
            int rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int alo = static_cast<int16_t>(av[q] & 0xFFFF), ahi = av[q] >> 16;
                const int blo = static_cast<int16_t>(bv[q] & 0xFFFF), bhi = bv[q] >> 16;
                const int lo = (i & 1) ? alo + blo : alo - blo;
                const int hi = (i & 1) ? ahi + bhi : ahi - bhi;
                rv[q] = static_cast<int>((static_cast<uint32_t>(lo) & 0xFFFFu) | (static_cast<uint32_t>(hi) << 16));
            }
            r = make_int4(rv[0], rv[1], rv[2], rv[3]);
        }
        y[g] = r;
    }
}

// Two levels of step 8 in one pass: rows 4m .. 4m+3 of a level-l node nu
// from row m of its nine grandchildren 9 nu + c (level l + 2), the middle
// level never written.  With A_c = grandchild 9 nu + c, row m (0-based, as
// in k_postpass: level-(l+1) row k of node mu is p - q (k even) or p + r
// (k odd) of mu's children):
//   y_4m   = (A_0 - A_1) - (A_3 - A_4)     y_4m+1 = (A_0 - A_1) + (A_6 - A_7)
//   y_4m+2 = (A_0 + A_2) - (A_3 + A_5)     y_4m+3 = (A_0 + A_2) + (A_6 + A_8)
// Only the rows of outputs inside the node are read (they lie inside the
// grandchildren's orders).  Digits stay carry-save; the two levels' growth is
// within the post-pass digit bound.  One block per group of four output
// rows, 16 bytes of digits per thread and step.
template <class T>
__device__ __forceinline__ void unpack16B(int4 w, int (&d)[16 / sizeof(T)]) {
    const int v[4] = {w.x, w.y, w.z, w.w};
    if (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = v[q];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            d[2 * q] = static_cast<int16_t>(v[q] & 0xFFFF);
            d[2 * q + 1] = v[q] >> 16;
        }
    }
}
template <class T>
__device__ __forceinline__ int4 pack16B(const int (&d)[16 / sizeof(T)]) {
    if (sizeof(T) == 4) return make_int4(d[0], d[1], d[2], d[3]);
    int v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        v[q] = static_cast<int>((static_cast<uint32_t>(d[2 * q]) & 0xFFFFu) | (static_cast<uint32_t>(d[2 * q + 1]) << 16));
    return make_int4(v[0], v[1], v[2], v[3]);
}
template <class T>
__global__ void k_postpass2(PlanPtrs g, int rows_in, int rows_out, const int *__restrict__ parent_size, int Wo) {
    constexpr int ND = 16 / sizeof(T);  // digits per 16 bytes
    const T *__restrict__ in = static_cast<const T *>(g.in[blockIdx.y]);
    T *__restrict__ out = static_cast<T *>(g.out[blockIdx.y]);
    const int quads = (rows_out + 3) / 4;
    const int nu = blockIdx.x / quads, m = blockIdx.x % quads;
    const int size = parent_size[nu];
    const int i0 = 4 * m;
    if (i0 >= size) return;
    bool has[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) has[j] = i0 + j < size;
    // grandchild c is read when one of its outputs exists
    const bool need[9] = {true, has[0] || has[1], has[2] || has[3], has[0] || has[2], has[0],
                          has[2], has[1] || has[3], has[1], has[3]};
    const int4 *a[9];
#pragma unroll
    for (int c = 0; c < 9; ++c)
        a[c] = reinterpret_cast<const int4 *>(in + (static_cast<size_t>(9 * nu + c) * rows_in + m) * Wo);
    int4 *y = reinterpret_cast<int4 *>(out + (static_cast<size_t>(nu) * rows_out + i0) * Wo);
    const int groups = Wo * static_cast<int>(sizeof(T)) / 16;  // Wo is a multiple of 8
    const size_t ystride = static_cast<size_t>(Wo) * sizeof(T) / 16;
    for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
        int d[9][ND];
#pragma unroll
        for (int c = 0; c < 9; ++c) unpack16B<T>(need[c] ? a[c][gi] : make_int4(0, 0, 0, 0), d[c]);
        int r[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) r[q] = (d[0][q] - d[1][q]) - (d[3][q] - d[4][q]);
        if (has[0]) y[gi] = pack16B<T>(r);
#pragma unroll
        for (int q = 0; q < ND; ++q) r[q] = (d[0][q] - d[1][q]) + (d[6][q] - d[7][q]);
        if (has[1]) y[ystride + gi] = pack16B<T>(r);
#pragma unroll
        for (int q = 0; q < ND; ++q) r[q] = (d[0][q] + d[2][q]) - (d[3][q] + d[5][q]);
        if (has[2]) y[2 * ystride + gi] = pack16B<T>(r);
#pragma unroll
        for (int q = 0; q < ND; ++q) r[q] = (d[0][q] + d[2][q]) + (d[6][q] + d[8][q]);
        if (has[3]) y[3 * ystride + gi] = pack16B<T>(r);
    }
}

// ------------------------------------------------------------------ final normalise
// Row digit vector (int32 digits, radix 256) -> |Z| as 32-bit limbs, sign, bit
// length.  One warp per row: a first pass of carry propagation gives the sign
// (the carry out of the top), a second one over sign * digits gives the
// magnitude's digits in [0, 256), four to a limb.
struct Digits4 {
    long long x, y, z, w;
};
__device__ __forceinline__ Digits4 load4(const int32_t *d, int u) {
    const int4 w = *reinterpret_cast<const int4 *>(d + u);
    return {w.x, w.y, w.z, w.w};
}
__device__ __forceinline__ Digits4 load4(const int16_t *d, int u) {
    const uint2 w = *reinterpret_cast<const uint2 *>(d + u);
    return {static_cast<int16_t>(w.x & 0xFFFFu), static_cast<int>(w.x) >> 16, static_cast<int16_t>(w.y & 0xFFFFu),
            static_cast<int>(w.y) >> 16};
}
__device__ __forceinline__ Digits4 load4(const int64_t *d, int u) {
    const longlong2 a = reinterpret_cast<const longlong2 *>(d + u)[0];
    const longlong2 b = reinterpret_cast<const longlong2 *>(d + u)[1];
    return {a.x, a.y, b.x, b.y};
}
template <class T, class D>
__device__ __forceinline__ void load_lane_digits(const T *d, int ub, int Wo, D (&v)[kDigitsPerLane], int sgn) {
#pragma unroll
    for (int g = 0; g < kDigitsPerLane / 4; ++g) {
        const int u = ub + 4 * g;  // Wo is a multiple of 4
        const Digits4 w = (u < Wo) ? load4(d, u) : Digits4{0, 0, 0, 0};
        v[4 * g] = static_cast<D>(sgn * w.x);
        v[4 * g + 1] = static_cast<D>(sgn * w.y);
        v[4 * g + 2] = static_cast<D>(sgn * w.z);
        v[4 * g + 3] = static_cast<D>(sgn * w.w);
    }
}
template <class T>
__global__ void __launch_bounds__(256) k_final_normalize(const T *__restrict__ in, int n, int Wo,
                                                         uint32_t *__restrict__ zmag, uint8_t *__restrict__ zneg,
                                                         int32_t *__restrict__ zbits, int ZW, int32_t *dstat,
                                                         int row_offset, int track_max) {
    const int lane = threadIdx.x & 31;
    const int i = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;  // warp-uniform
    using D = typename std::conditional<sizeof(T) == 8, long long, int>::type;  // int32 digits with carries fit int
    const T *d = in + static_cast<size_t>(i) * Wo;
    D v[kDigitsPerLane];
    D wc = 0;
    for (int u0 = 0; u0 < Wo; u0 += 32 * kDigitsPerLane) {
        load_lane_digits(d, u0 + kDigitsPerLane * lane, Wo, v, 1);
        warp_carry<false, D>(v, lane, wc);
    }
    const int sgn = (wc < 0) ? -1 : 1;  // digits in [0, 256) below the carry: the value is negative iff it is
    uint32_t *z = zmag + static_cast<size_t>(row_offset + i) * ZW;
    int bits = 0;
    bool bad = false;
    wc = 0;
    for (int u0 = 0; u0 < Wo; u0 += 32 * kDigitsPerLane) {
        const int ub = u0 + kDigitsPerLane * lane;
        load_lane_digits(d, ub, Wo, v, sgn);
        warp_carry<false, D>(v, lane, wc);
#pragma unroll
        for (int g = 0; g < kDigitsPerLane / 4; ++g) {
            const int u = ub + 4 * g;
            const uint32_t limb = static_cast<uint32_t>(v[4 * g]) | (static_cast<uint32_t>(v[4 * g + 1]) << 8) |
                                  (static_cast<uint32_t>(v[4 * g + 2]) << 16) |
                                  (static_cast<uint32_t>(v[4 * g + 3]) << 24);
            if (u < Wo) {
                z[u / 4] = limb;
                if (limb) bits = 32 * (u / 4) + (32 - __clz(limb));
            } else if (limb) {
                bad = true;  // |Z| does not fit the row
            }
        }
    }
    if (wc != 0) bad = true;
    for (int w = Wo / 4 + lane; w < ZW; w += 32) z[w] = 0u;  // limbs above the row's digits
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(dstat, DEV_OVERFLOW);
    if (lane == 0) {
        zbits[row_offset + i] = bits;
        zneg[row_offset + i] = (bits > 0 && sgn < 0) ? 1 : 0;
        if (track_max) atomicMax(dstat + 1, bits);
    }
}

// Signed 128-bit column sums of 32-bit limb weights -> |Z| limbs, sign, bits.
__global__ void k_colsum_normalize(const __int128 *__restrict__ cs, int n, int ncols, uint32_t *__restrict__ zmag,
                                   uint8_t *__restrict__ zneg, int32_t *__restrict__ zbits, int ZW, int32_t *dstat,
                                   int row_offset) {
    // one thread per row; the columns are read eight at a time, ahead of the
    // carry chain that consumes them, so the chain does not wait on each load
    constexpr int G = 8;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const __int128 *d = cs + static_cast<size_t>(i) * ncols;
    __int128 c = 0;
    for (int w0 = 0; w0 < ncols; w0 += G) {
        __int128 v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) v[q] = (w0 + q < ncols) ? d[w0 + q] : static_cast<__int128>(0);
#pragma unroll
        for (int q = 0; q < G; ++q) c = (v[q] + c) >> 32;
    }
    const int sgn = (c < 0) ? -1 : 1;
    c = 0;
    uint32_t *z = zmag + static_cast<size_t>(row_offset + i) * ZW;
    int top = -1;
    uint32_t topv = 0;
    for (int w0 = 0; w0 < ZW; w0 += G) {
        __int128 v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) v[q] = (w0 + q < ncols) ? d[w0 + q] : static_cast<__int128>(0);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int w = w0 + q;
            if (w >= ZW) break;
            const __int128 t = (sgn < 0 ? -v[q] : v[q]) + c;
            const uint32_t limb = static_cast<uint32_t>(static_cast<unsigned __int128>(t) & 0xFFFFFFFFu);
            c = t >> 32;
            z[w] = limb;
            if (limb) { top = w; topv = limb; }
        }
    }
    if (c != 0) set_status(dstat, DEV_OVERFLOW);
    int bits = (top < 0) ? 0 : 32 * top + (32 - __clz(topv));
    zbits[row_offset + i] = bits;
    zneg[row_offset + i] = (bits > 0 && sgn < 0) ? 1 : 0;
    atomicMax(dstat + 1, bits);
}

// ------------------------------------------------------------------ rounding
// bit pos of |Z| (0 outside)
__device__ __forceinline__ uint32_t zbit(const uint32_t *z, int ZW, long long pos) {
    if (pos < 0 || pos >= 32LL * ZW) return 0;
    return (z[pos >> 5] >> (pos & 31)) & 1u;
}
// 32 bits of |Z| starting at bit pos (pos may be negative: zeros shifted in)
__device__ __forceinline__ uint32_t zword(const uint32_t *z, int ZW, long long pos) {
    long long w = (pos >= 0) ? (pos >> 5) : -((-pos + 31) >> 5);
    int sh = static_cast<int>(pos - 32 * w);
    uint32_t lo = (w >= 0 && w < ZW) ? z[w] : 0u;
    uint32_t hi = (w + 1 >= 0 && w + 1 < ZW) ? z[w + 1] : 0u;
    return sh ? ((lo >> sh) | (hi << (32 - sh))) : lo;
}
// round bit and sticky of |Z| / 2^t (t > 0)
__device__ void round_bits(const uint32_t *z, int ZW, long long t, uint32_t &half, uint32_t &sticky) {
    half = zbit(z, ZW, t - 1);
    sticky = 0;
    long long below = t - 1;  // bits [0, below)
    long long full = below >> 5;
    for (long long w = 0; w < full && w < ZW; ++w) sticky |= z[w];
    int rem = static_cast<int>(below & 31);
    if (rem && full < ZW) sticky |= z[full] & ((1u << rem) - 1u);
    sticky = sticky ? 1u : 0u;
}

// dstat: [0] error, [1] max bit length, [2] round-up-to-2^b flag, [3] E_y
// A row can reach 2^b only if it has the maximum bit length.
__global__ void k_round_check(const uint32_t *__restrict__ zmag, const int32_t *__restrict__ zbits, int rows, int ZW,
                              int b, int32_t *dstat) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const int B = dstat[1];
    const long long t = static_cast<long long>(B) - b;
    if (B == 0 || t <= 0 || zbits[i] != B) return;
    const uint32_t *z = zmag + static_cast<size_t>(i) * ZW;
    // all b bits of |Z| >> t set?
    for (long long p = t; p < t + b; ++p)
        if (!zbit(z, ZW, p)) return;
    uint32_t half, sticky;
    round_bits(z, ZW, t, half, sticky);
    if (half) atomicExch(dstat + 2, 1);  // an all-ones mantissa is odd: a half rounds up
}

// One warp per output row: the lanes cut the b-bit mantissa limbs out of |Z|
// and OR the bits below the rounding position in parallel; the rare carry of
// a round-up runs through the limbs on lane 0.
__global__ void __launch_bounds__(256) k_round(const uint32_t *__restrict__ zmag, const uint8_t *__restrict__ zneg,
                                               int n, int nrhs, int ZW, int b, int L32, int e_in, int reverse,
                                               int32_t *dstat, uint32_t *__restrict__ y, uint8_t *__restrict__ yneg) {
    const int lane = threadIdx.x & 31;
    const int idx = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (idx >= n * nrhs) return;  // warp-uniform
    if (dstat[0] != DEV_OK) return;  // an earlier stage failed: write nothing
    const int rhs = idx / n, i = idx % n;
    const int orow = rhs * n + (reverse ? (n - 1 - i) : i);
    uint32_t *o = y + static_cast<size_t>(orow) * L32;
    const int B = dstat[1];
    if (B == 0) {
        for (int w = lane; w < L32; w += 32) o[w] = 0;
        if (lane == 0) {
            yneg[orow] = 0;
            if (idx == 0) dstat[3] = e_in;
        }
        return;
    }
    const long long t = static_cast<long long>(B) - b + dstat[2];
    const uint32_t *z = zmag + static_cast<size_t>(idx) * ZW;
    const int topbits = b - 32 * (L32 - 1);
    uint32_t first = 0;  // lane 0: limb 0 of the truncated mantissa
    for (int w = lane; w < L32; w += 32) {
        uint32_t v = zword(z, ZW, t + 32LL * w);
        if (w == L32 - 1 && topbits < 32) v &= (1u << topbits) - 1u;
        o[w] = v;
        if (w == 0) first = v;
    }
    if (t > 0) {
        const uint32_t half = zbit(z, ZW, t - 1);
        // sticky: any bit of |Z| below position t - 1
        const long long below = t - 1;
        const long long full = min(below >> 5, static_cast<long long>(ZW));
        uint32_t st = 0;
        for (long long w = lane; w < full; w += 32) st |= z[w];
        const int rem = static_cast<int>(below & 31);
        if (lane == 0 && rem && full < ZW) st |= z[full] & ((1u << rem) - 1u);
        const bool sticky = __any_sync(0xffffffffu, st != 0);
        const uint32_t lsb = __shfl_sync(0xffffffffu, first, 0) & 1u;
        __syncwarp();  // the lanes' limbs are in place before lane 0 carries through them
        if (lane == 0 && half && (sticky || lsb)) {
            for (int w = 0; w < L32; ++w) {
                o[w] += 1u;
                if (o[w] != 0) break;
            }
            if (topbits < 32 && (o[L32 - 1] >> topbits)) set_status(dstat, DEV_OVERFLOW);
        }
        __syncwarp();
    }
    uint32_t any = 0;
    for (int w = lane; w < L32; w += 32) any |= o[w];
    const bool nonzero = __any_sync(0xffffffffu, any != 0);
    if (lane == 0) {
        yneg[orow] = (nonzero && zneg[idx]) ? 1 : 0;
        if (idx == 0) dstat[3] = static_cast<int32_t>(e_in + t - b);
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
namespace {
cudaError_t encode_group(hmv_plan_s *p, const PlanPtrs &g, int G, int rows, int circulant_n) {
    k_encode<<<dim3(static_cast<unsigned>((rows + 7) / 8), G), 256, 0, p->stream>>>(  // a warp per row
        g, rows, p->L32, p->b, circulant_n, p->Dp, p->dstat);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t prepass_group(hmv_plan_s *p, const PlanPtrs &g, int G, int level, bool matrix_side) {
    const LevelGeom &pl = p->lv[level], &cl = p->lv[level + 1];
    const int in_rows = matrix_side ? pl.rowsA : pl.rowsX;
    const int out_rows = matrix_side ? cl.rowsA : cl.rowsX;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_prepass_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, kPreSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // a block per 128 rows of a child, row block major (siblings are neighbours)
    const long long blocks = static_cast<long long>((out_rows + kPreRows - 1) / kPreRows) * cl.nodes;
    k_prepass_staged<<<dim3(static_cast<unsigned>(blocks), G), kPreRows, kPreSmem, p->stream>>>(
        g, in_rows, pl.d_size, out_rows, cl.d_size, cl.nodes, p->Dp, matrix_side ? 1 : 0, p->dstat);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t pack_vector_group(hmv_plan_s *p, const PlanPtrs &g, int G) {
    const LevelGeom &ll = p->lv[p->L];
    const int chunks = p->Dp / 8 + 1;
    const int nseg = (chunks + kPackSeg - 1) / kPackSeg;
    const int seg = (chunks + nseg - 1) / nseg;  // balanced segments of at most kPackSeg chunks
    const dim3 grid(static_cast<unsigned>(ll.nodes) * p->RX, nseg, G);
    k_pack_vector<<<grid, 128, 0, p->stream>>>(g, ll.rowsX, ll.d_size, p->RX, p->Dp, seg);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t leaf_normalize_group(hmv_plan_s *p, const PlanPtrs &g, int G) {
    const LevelGeom &ll = p->lv[p->L];
    const dim3 grid(static_cast<unsigned>(ll.nodes) * ll.rowsX, G);  // one block per leaf row
    if (p->post16)
        k_leaf_normalize<int16_t><<<grid, 128, 0, p->stream>>>(g, ll.d_size, p->MT, p->Uo, p->NUB, ll.rowsX, p->Wo,
                                                               p->tn);
    else
        k_leaf_normalize<int32_t><<<grid, 128, 0, p->stream>>>(g, ll.d_size, p->MT, p->Uo, p->NUB, ll.rowsX, p->Wo,
                                                               p->tn);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t leaf_post_group(hmv_plan_s *p, const PlanPtrs &g, int G) {
    const LevelGeom &pl = p->lv[p->L - 1];
    const dim3 grid(static_cast<unsigned>(pl.nodes) * ((pl.rowsX + 1) / 2), G);  // one block per output row pair
    const int steps = (p->Wo / 8 + 31) / 32 * 32;  // threads: one step of 8 digits each, at most 256
    const int threads = steps < 256 ? steps : 256;
    if (p->post16)
        k_leaf_post<int16_t><<<grid, threads, 0, p->stream>>>(g, pl.d_size, p->MT, p->Uo, p->NUB, pl.rowsX, p->Wo,
                                                               p->tn);
    else
        k_leaf_post<int32_t><<<grid, threads, 0, p->stream>>>(g, pl.d_size, p->MT, p->Uo, p->NUB, pl.rowsX, p->Wo,
                                                               p->tn);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t postpass2_group(hmv_plan_s *p, const PlanPtrs &g, int G, int level) {
    const LevelGeom &pl = p->lv[level], &gl = p->lv[level + 2];
    const dim3 grid(static_cast<unsigned>(pl.nodes) * ((pl.rowsX + 3) / 4), G);  // one block per four output rows
    if (p->post16)
        k_postpass2<int16_t><<<grid, 128, 0, p->stream>>>(g, gl.rowsX, pl.rowsX, pl.d_size, p->Wo);
    else
        k_postpass2<int32_t><<<grid, 128, 0, p->stream>>>(g, gl.rowsX, pl.rowsX, pl.d_size, p->Wo);
    p->launches_total++;
    return cudaGetLastError();
}
cudaError_t postpass_group(hmv_plan_s *p, const PlanPtrs &g, int G, int level) {
    const LevelGeom &pl = p->lv[level], &cl = p->lv[level + 1];
    const dim3 grid(static_cast<unsigned>(pl.nodes) * pl.rowsX, G);  // one block per output row
    if (p->post16)
        k_postpass<int16_t><<<grid, 128, 0, p->stream>>>(g, cl.rowsX, pl.rowsX, pl.d_size, p->Wo);
    else
        k_postpass<int32_t><<<grid, 128, 0, p->stream>>>(g, cl.rowsX, pl.rowsX, pl.d_size, p->Wo);
    p->launches_total++;
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_encode(hmv_plan_s *p, const uint32_t *limbs, const uint8_t *neg, int rows, int circulant_n,
                          int8_t *out) {
    PlanPtrs g{};
    g.in[0] = limbs;
    g.in2[0] = neg;
    g.out[0] = out;
    return encode_group(p, g, 1, rows, circulant_n);
}

cudaError_t launch_prepass(hmv_plan_s *p, int level, bool matrix_side, const int8_t *in, int8_t *out) {
    PlanPtrs g{};
    g.in[0] = in;
    g.out[0] = out;
    return prepass_group(p, g, 1, level, matrix_side);
}

cudaError_t launch_pack_matrix(hmv_plan_s *p, const int8_t *leaf_digits) {
    const LevelGeom &ll = p->lv[p->L];
    long long work = static_cast<long long>(ll.nodes) * p->RA * (p->Dp / 8);
    k_pack_matrix<<<blocks_for(work), kThreads, 0, p->stream>>>(leaf_digits, ll.rowsA, ll.d_size, p->hrev, p->RA,
                                                                p->Dp, ll.nodes);
    p->launches_total++;
    return cudaGetLastError();
}

cudaError_t launch_pack_vector(hmv_plan_s *p, const int8_t *leaf_digits) {
    PlanPtrs g{};
    g.in[0] = leaf_digits;
    g.out[0] = p->xg;
    return pack_vector_group(p, g, 1);
}

cudaError_t launch_leaf_simt(hmv_plan_s *p, const int8_t *a_leaf, const int8_t *x_leaf) {
    const LevelGeom &ll = p->lv[p->L];
    dim3 grid(p->ntiles, TM);
    k_leaf_simt<<<grid, p->tn, 0, p->stream>>>(a_leaf, ll.rowsA, x_leaf, ll.rowsX, ll.d_size, p->Dp, p->Dl,
                                               p->d_tiles, p->leaf_dig, p->leaf_carry, p->MT, p->Uo, p->NUB, p->dstat,
                                               p->tn);
    p->launches_leaf++;
    p->launches_total++;
    return cudaGetLastError();
}

// The vector side (encode of each plan's staged x, every pre-pass level, the
// shifted bf16 copies) and the post side (leaf normalise, every post-pass
// level) of up to kMaxGroup plans with the same geometry, one launch per
// kernel and level for all of them, on ps[0]'s stream.
cudaError_t launch_vector_side_group(hmv_plan_s *const *ps, int G) {
    if (G < 1 || G > kMaxGroup) return cudaErrorInvalidValue;
    hmv_plan_s *p = ps[0];
    PlanPtrs g{};
    for (int k = 0; k < G; ++k) {
        g.in[k] = ps[k]->x_limbs_d;
        g.in2[k] = ps[k]->x_neg_d;
        g.out[k] = ps[k]->x_lvl[0];
    }
    cudaError_t e = encode_group(p, g, G, p->n, 0);
    for (int l = 0; l < p->L && e == cudaSuccess; ++l) {
        for (int k = 0; k < G; ++k) {
            g.in[k] = ps[k]->x_lvl[l % 2];
            g.out[k] = ps[k]->x_lvl[(l + 1) % 2];
        }
        e = prepass_group(p, g, G, l, false);
    }
    if (e == cudaSuccess) {
        for (int k = 0; k < G; ++k) {
            g.in[k] = ps[k]->x_lvl[p->L % 2];
            g.out[k] = ps[k]->xg;
        }
        e = pack_vector_group(p, g, G);
    }
    return e;
}

cudaError_t launch_post_group(hmv_plan_s *const *ps, int G) {
    if (G < 1 || G > kMaxGroup) return cudaErrorInvalidValue;
    hmv_plan_s *p = ps[0];
    PlanPtrs g{};
    // leaf normalise alone at depth 0, else fused into the deepest post-pass level
    for (int k = 0; k < G; ++k) {
        g.in[k] = ps[k]->leaf_dig;
        g.in2[k] = ps[k]->leaf_carry;
        g.out[k] = ps[k]->post[(p->L + 1) % 2];
    }
    if (p->L == 0) {
        for (int k = 0; k < G; ++k) g.out[k] = ps[k]->post[0];
        return leaf_normalize_group(p, g, G);
    }
    // levels L-1 .. 0: two at a time (k_postpass2) while two are left, then one;
    // the buffers alternate, and leaf_post starts in the one that makes level 0
    // land in post[0]
    int steps = 0;
    for (int c = p->L - 1; c > 0; c -= (c >= 2 ? 2 : 1)) ++steps;
    int cur = steps % 2;
    for (int k = 0; k < G; ++k) g.out[k] = ps[k]->post[cur];
    cudaError_t e = leaf_post_group(p, g, G);  // level L - 1
    for (int c = p->L - 1; c > 0 && e == cudaSuccess;) {
        const int l = c >= 2 ? c - 2 : c - 1;
        for (int k = 0; k < G; ++k) {
            g.in[k] = ps[k]->post[cur];
            g.out[k] = ps[k]->post[1 - cur];
        }
        e = (c - l == 2) ? postpass2_group(p, g, G, l) : postpass_group(p, g, G, l);
        cur = 1 - cur;
        c = l;
    }
    return e;
}

// Plans that one grouped launch can serve together.
bool same_geometry(hmv_plan_s *const *ps, int G) {
    if (G < 1 || G > kMaxGroup) return false;
    const hmv_plan_s *a = ps[0];
    if (!a->xg || a->L < 0 || static_cast<int>(a->lv.size()) != a->L + 1) return false;
    for (int k = 1; k < G; ++k) {
        const hmv_plan_s *c = ps[k];
        if (!c->xg || c->n != a->n || c->L != a->L || c->L32 != a->L32 || c->b != a->b || c->Dp != a->Dp ||
            c->RX != a->RX || c->MT != a->MT || c->Uo != a->Uo || c->NUB != a->NUB || c->Wo != a->Wo ||
            c->tn != a->tn || c->post16 != a->post16)
            return false;
    }
    return true;
}
cudaError_t launch_final_normalize(hmv_plan_s *p, const int32_t *in, int rhs, int digit_bytes, bool track_max) {
    const unsigned blocks = static_cast<unsigned>((p->n + 7) / 8);  // a warp per row
    const int tm = track_max ? 1 : 0;
    if (digit_bytes == 2)
        k_final_normalize<int16_t><<<blocks, 256, 0, p->stream>>>(reinterpret_cast<const int16_t *>(in), p->n, p->Wo,
                                                                  p->zmag, p->zneg, p->zbits, p->ZW, p->dstat,
                                                                  rhs * p->n, tm);
    else if (digit_bytes == 8)
        k_final_normalize<int64_t><<<blocks, 256, 0, p->stream>>>(reinterpret_cast<const int64_t *>(in), p->n, p->Wo,
                                                                  p->zmag, p->zneg, p->zbits, p->ZW, p->dstat,
                                                                  rhs * p->n, tm);
    else
        k_final_normalize<int32_t><<<blocks, 256, 0, p->stream>>>(in, p->n, p->Wo, p->zmag, p->zneg, p->zbits, p->ZW,
                                                                  p->dstat, rhs * p->n, tm);
    p->launches_total++;
    return cudaGetLastError();
}

cudaError_t launch_colsum_normalize(hmv_plan_s *p, int rhs) {
    k_colsum_normalize<<<blocks_for(p->n, 128), 128, 0, p->stream>>>(p->colsum, p->n, 2 * p->L32, p->zmag, p->zneg,
                                                                     p->zbits, p->ZW, p->dstat, rhs * p->n);
    p->launches_total++;
    return cudaGetLastError();
}

cudaError_t launch_round(hmv_plan_s *p, int rows, int e_in, uint32_t *y_limbs, uint8_t *y_neg) {
    k_round_check<<<blocks_for(rows, 128), 128, 0, p->stream>>>(p->zmag, p->zbits, rows, p->ZW, p->b, p->dstat);
    k_round<<<static_cast<unsigned>((rows + 7) / 8), 256, 0, p->stream>>>(  // a warp per row
        p->zmag, p->zneg, p->n, p->nrhs, p->ZW, p->b, p->L32, e_in, p->kind != HMV_HANKEL ? 1 : 0, p->dstat, y_limbs,
        y_neg);
    p->launches_total += 2;
    return cudaGetLastError();
}

// Normalisation and rounding on caller-given buffers (used by the
// scratch-free entry point); dstat must start zeroed.
// Signed 128-bit column sums with ncols columns per row: normalise to |Z|
// limbs (ZW >= ncols + 3), and optionally round each row to b bits with the
// least shared exponent (value = Z * 2^(e_in - 2b)).
cudaError_t launch_colsum_normalize_cols(const __int128 *colsum, int n, int ncols, uint32_t *zmag, uint8_t *zneg,
                                         int32_t *zbits, int ZW, int32_t *dstat, cudaStream_t stream) {
    k_colsum_normalize<<<blocks_for(n, 128), 128, 0, stream>>>(colsum, n, ncols, zmag, zneg, zbits, ZW, dstat, 0);
    return cudaGetLastError();
}
cudaError_t launch_colsum_round_cols(const __int128 *colsum, int n, int ncols, int L32, uint32_t *zmag, uint8_t *zneg,
                                     int32_t *zbits, int ZW, int32_t *dstat, int b, int e_in, uint32_t *y,
                                     uint8_t *yneg, cudaStream_t stream) {
    k_colsum_normalize<<<blocks_for(n, 128), 128, 0, stream>>>(colsum, n, ncols, zmag, zneg, zbits, ZW, dstat, 0);
    k_round_check<<<blocks_for(n, 128), 128, 0, stream>>>(zmag, zbits, n, ZW, b, dstat);
    k_round<<<static_cast<unsigned>((n + 7) / 8), 256, 0, stream>>>(zmag, zneg, n, 1, ZW, b, L32, e_in, 0, dstat, y,
                                                                    yneg);  // a warp per row
    return cudaGetLastError();
}

cudaError_t launch_colsum_round_raw(const __int128 *colsum, int n, int L32, uint32_t *zmag, uint8_t *zneg,
                                    int32_t *zbits, int ZW, int32_t *dstat, int b, int e_in, int reverse,
                                    uint32_t *y, uint8_t *yneg, cudaStream_t stream) {
    k_colsum_normalize<<<blocks_for(n, 128), 128, 0, stream>>>(colsum, n, 2 * L32, zmag, zneg, zbits, ZW, dstat, 0);
    k_round_check<<<blocks_for(n, 128), 128, 0, stream>>>(zmag, zbits, n, ZW, b, dstat);
    k_round<<<static_cast<unsigned>((n + 7) / 8), 256, 0, stream>>>(zmag, zneg, n, 1, ZW, b, L32, e_in, reverse, dstat,
                                                                    y, yneg);  // a warp per row
    return cudaGetLastError();
}

}  // namespace hmv
