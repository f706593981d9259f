// Karatsuba in the digit dimension, on top of the index recursion.
//
// Algorithm 1 (Beliakov, arXiv:1402.5287, Sec. 3) saves products along the
// matrix index; the same bilinear trick also applies to the numbers
// themselves (Karatsuba's own splitting, which Sec. 3 names as its
// inspiration).  With every mantissa split at s bits, V = V1 2^s + V0
// (|V0| < 2^s, |V1| < 2^(b-s), both with the sign of V), the exact rows are
//     Z = Z11 2^(2s) + (Zm - Z00 - Z11) 2^s + Z00,
//     Z00 = A(h0) x0,  Z11 = A(h1) x1,  Zm = A(h0 + h1)(x0 + x1),
// three Hankel products of about half the width: 3/4 of the digit
// multiply-adds per level.  Each of the three is an ordinary plan (index
// recursion plus tensor-core leaves); a split plan may itself split again.
// All leaf products of all descendants run in ONE persistent tensor-core
// launch; the exact digit vectors of the three children are combined with
// digit shifts (s is a multiple of 32 bits), then normalised and rounded
// once, exactly like an unsplit plan.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hmv_carry.cuh"
#include "hmv_internal.h"

namespace hmv {
namespace {

// Sign-magnitude rows (b bits, L32 limbs) -> the three children's rows
// (bc bits, Lc limbs): lo = M mod 2^s, hi = M >> s, mid = lo + hi, each with
// the sign of the entry (zero magnitudes are +).
__global__ void k_split(const uint32_t *__restrict__ limbs, const uint8_t *__restrict__ neg, int rows, int L32,
                        int sl, int Lc, uint32_t *__restrict__ lo, uint32_t *__restrict__ hi,
                        uint32_t *__restrict__ mid, uint8_t *__restrict__ nlo, uint8_t *__restrict__ nhi,
                        uint8_t *__restrict__ nmid) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const uint32_t *m = limbs + static_cast<size_t>(k) * L32;
    uint32_t *ol = lo + static_cast<size_t>(k) * Lc;
    uint32_t *oh = hi + static_cast<size_t>(k) * Lc;
    uint32_t *om = mid + static_cast<size_t>(k) * Lc;
    uint32_t anyl = 0, anyh = 0;
    unsigned long long c = 0;
    for (int q = 0; q < Lc; ++q) {
        const uint32_t vl = (q < sl && q < L32) ? m[q] : 0u;
        const uint32_t vh = (q + sl < L32) ? m[q + sl] : 0u;
        ol[q] = vl;
        oh[q] = vh;
        c += static_cast<unsigned long long>(vl) + vh;
        om[q] = static_cast<uint32_t>(c);
        c >>= 32;
        anyl |= vl;
        anyh |= vh;
    }
    const uint8_t s = neg[k] ? 1 : 0;
    nlo[k] = anyl ? s : 0;
    nhi[k] = anyh ? s : 0;
    nmid[k] = (anyl | anyh) ? s : 0;
}

// z[u] = Z00[u] + (Zm - Z00 - Z11)[u - ds] + Z11[u - 2 ds], int32 digits,
// radix 2^8, no carries (the digits stay far below 2^31).
// Digit u of z, an int16 (is16) or int32 digit row of width Wc, 0 outside it.
__device__ __forceinline__ int32_t digit_at(const int32_t *z, bool is16, size_t row, int Wc, int v) {
    if (v < 0 || v >= Wc) return 0;
    return is16 ? static_cast<int32_t>(reinterpret_cast<const int16_t *>(z)[row * Wc + v]) : z[row * Wc + v];
}
__global__ void k_combine(const int32_t *__restrict__ z00, const int32_t *__restrict__ zm,
                          const int32_t *__restrict__ z11, int in16_mask, int Wc, int n, int ds,
                          int32_t *__restrict__ out, int Wp) {
    const int i = blockIdx.x;  // grid: (rows, column blocks)
    const bool a16 = in16_mask & 1, m16 = in16_mask & 2, b16 = in16_mask & 4;
    for (int u = blockIdx.y * blockDim.x + threadIdx.x; u < Wp; u += gridDim.y * blockDim.x)
        out[static_cast<size_t>(i) * Wp + u] = digit_at(z00, a16, i, Wc, u) + digit_at(zm, m16, i, Wc, u - ds) -
                                               digit_at(z00, a16, i, Wc, u - ds) - digit_at(z11, b16, i, Wc, u - ds) +
                                               digit_at(z11, b16, i, Wc, u - 2 * ds);
}

// ------------------------------------------------------------------ Toom-Cook
// Each mantissa M = sum_k V_k 2^(ks), k = 0..K-1 (|V_k| < 2^s, all with the
// sign of the entry), read as a polynomial in t = 2^s; so are the exact rows,
// Z(t) = A(h(t)) x(t) = sum_m C_m t^m, m = 0..2K-2.  2K-1 products at chosen
// points fix the C_m; Den C_m = sum_t N[m][t] P_t with the integer matrix N =
// Den times the inverse of the evaluation matrix, and Z = Z(2^s).  A point
// p/q is evaluated homogenised, q^(K-1) V(p/q) = sum_k V_k p^k q^(K-1-k), and
// infinity gives the leading part.  The tables are that evaluation matrix's
// rows and its inverse scaled by Den (exact rational elimination).
//   K = 4: points 0, 1, -1, 2, -2, 1/2, inf; Den = 360; |E| < 15 * 2^s.
//   K = 6: points 0, 1, -1, 2, -2, 1/2, -1/2, 3, -3, 1/3, inf; Den = 1008000;
//          |E| < 364 * 2^s.
//   K = 8: points 0, 1, -1, 2, -2, 1/2, -1/2, 3, -3, 1/3, -1/3, 3/2, -3/2,
//          2/3, inf (the set with the smallest interpolation constants among
//          those tried); Den = 54486432000 = 7776000 * 7007, |N| < 2^44;
//          |E| < 6305 * 2^s.
__constant__ int16_t kToom4Eval[7][4] = {{1, 0, 0, 0}, {1, 1, 1, 1},   {1, -1, 1, -1}, {1, 2, 4, 8},
                                         {1, -2, 4, -8}, {8, 4, 2, 1}, {0, 0, 0, 1}};
__constant__ int32_t kToom4Interp[7][7] = {{360, 0, 0, 0, 0, 0, 0},
                                           {-720, -240, -80, 10, 6, 16, -720},
                                           {-450, 240, 240, -15, -15, 0, 1440},
                                           {900, 540, -140, -20, 0, -20, 900},
                                           {90, -60, -60, 15, 15, 0, -1800},
                                           {-180, -120, 40, 10, -6, 4, -180},
                                           {0, 0, 0, 0, 0, 0, 360}};
__constant__ int16_t kToom6Eval[11][6] = {{1, 0, 0, 0, 0, 0},     {1, 1, 1, 1, 1, 1},         {1, -1, 1, -1, 1, -1},
                                          {1, 2, 4, 8, 16, 32},   {1, -2, 4, -8, 16, -32},    {32, 16, 8, 4, 2, 1},
                                          {32, -16, 8, -4, 2, -1}, {1, 3, 9, 27, 81, 243},    {1, -3, 9, -27, 81, -243},
                                          {243, 81, 27, 9, 3, 1}, {0, 0, 0, 0, 0, 1}};
__constant__ int32_t kToom6Interp[11][11] = {
    {1008000, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {-3024000, 126000, 63000, -2016, -1440, -2880, -576, 60, 48, 108, -3024000},
    {-5404000, -252000, -252000, 5040, 5040, 2880, 2880, -160, -160, 0, 9072000},
    {16212000, -927500, -85750, 13328, 5200, 21200, -2672, -375, -204, -579, 16212000},
    {5880000, 1099000, 1099000, -25760, -25760, -3920, -3920, 840, 840, 0, -48636000},
    {-17640000, 1834000, -731500, -24640, 4480, -24640, 4480, 630, 0, 630, -17640000},
    {-1596000, -371000, -371000, 22960, 22960, 1120, 1120, -840, -840, 0, 52920000},
    {4788000, -570500, 271250, 14672, -9200, 6800, -1328, -375, 204, -171, 4788000},
    {112000, 28000, 28000, -2240, -2240, -80, -80, 160, 160, 0, -14364000},
    {-336000, 42000, -21000, -1344, 960, -480, 96, 60, -48, 12, -336000},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1008000}};
__constant__ int16_t kToom8Eval[15][8] = {{1, 0, 0, 0, 0, 0, 0, 0},
{1, 1, 1, 1, 1, 1, 1, 1},
{1, -1, 1, -1, 1, -1, 1, -1},
{1, 2, 4, 8, 16, 32, 64, 128},
{1, -2, 4, -8, 16, -32, 64, -128},
{128, 64, 32, 16, 8, 4, 2, 1},
{128, -64, 32, -16, 8, -4, 2, -1},
{1, 3, 9, 27, 81, 243, 729, 2187},
{1, -3, 9, -27, 81, -243, 729, -2187},
{2187, 729, 243, 81, 27, 9, 3, 1},
{2187, -729, 243, -81, 27, -9, 3, -1},
{128, 192, 288, 432, 648, 972, 1458, 2187},
{128, -192, 288, -432, 648, -972, 1458, -2187},
{2187, 1458, 972, 648, 432, 288, 192, 128},
{0, 0, 0, 0, 0, 0, 0, 1}};
#define HMV_TOOM8_INTERP {{54486432000LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL},\
{-81729648000LL, -6129723600LL, -1225944720LL, -10007712LL, -5003856LL, -17513496LL, 2501928LL, 30888LL, 19656LL, 75816LL, -25272LL, 14040LL, 5400LL, 19440LL, -81729648000LL},\
{-806701896000LL, 3064861800LL, 3064861800LL, 10007712LL, 10007712LL, -8756748LL, -8756748LL, -36036LL, -36036LL, 113724LL, 113724LL, -11700LL, -11700LL, 0LL, 122594472000LL},\
{1210052844000LL, 93818825100LL, 15085930860LL, 153173592LL, 69081012LL, 241783542LL, -19528938LL, -469326LL, -279006LL, -781326LL, 32994LL, -215670LL, -72150LL, -287820LL, 1210052844000LL},\
{3294579288000LL, -42312119850LL, -42312119850LL, -145667808LL, -145667808LL, 94621527LL, 94621527LL, 529529LL, 529529LL, -660231LL, -660231LL, 168025LL, 168025LL, 0LL, -1815079266000LL},\
{-4941868932000LL, -412952289750LL, -31815914130LL, -677960712LL, -229729500LL, -869728860LL, -37961352LL, 2044185LL, 1012011LL, 2603601LL, 452595LL, 960960LL, 214500LL, 1175460LL, -4941868932000LL},\
{-4256500248000LL, 143007965100LL, 143007965100LL, 568709856LL, 568709856LL, -150999849LL, -150999849LL, -2120118LL, -2120118LL, 934362LL, 934362LL, -632775LL, -632775LL, 0LL, 7412803398000LL},\
{6384750372000LL, 621864243000LL, -47236709520LL, 1066161096LL, 106548156LL, 1066161096LL, 106548156LL, -3119688LL, -828828LL, -3119688LL, -828828LL, -1518660LL, 0LL, -1518660LL, 6384750372000LL},\
{2092178088000LL, -96420173850LL, -96420173850LL, -639628704LL, -639628704LL, 80081001LL, 80081001LL, 2579577LL, 2579577LL, -474903LL, -474903LL, 632775LL, 632775LL, 0LL, -9577125558000LL},\
{-3138267132000LL, -331790208750LL, 49346166870LL, -704091960LL, 127675548LL, -512323812LL, -64092600LL, 2045901LL, -105105LL, 1486485LL, 454311LL, 960960LL, -214500LL, 746460LL, -3138267132000LL},\
{-402257856000LL, 21264843600LL, 21264843600LL, 224370432LL, 224370432LL, -15918903LL, -15918903LL, -1097096LL, -1097096LL, 92664LL, 92664LL, -168025LL, -168025LL, 0LL, 4707400698000LL},\
{603386784000LL, 66518852400LL, -12214041840LL, 186069312LL, -75243168LL, 97459362LL, 13366782LL, -593736LL, 220584LL, -281736LL, -91416LL, -215670LL, 72150LL, -143520LL, 603386784000LL},\
{24216192000LL, -1362160800LL, -1362160800LL, -17791488LL, -17791488LL, 972972LL, 972972LL, 144144LL, 144144LL, -5616LL, -5616LL, 11700LL, 11700LL, 0LL, -905080176000LL},\
{-36324288000LL, -4086482400LL, 817296480LL, -13343616LL, 6671808LL, -5837832LL, -833976LL, 61776LL, -39312LL, 16848LL, 5616LL, 14040LL, -5400LL, 8640LL, -36324288000LL},\
{0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 0LL, 54486432000LL}}
constexpr long long kToom8InterpHost[15][15] = HMV_TOOM8_INTERP;  // for the plan-time overflow bound
#undef HMV_TOOM8_INTERP
// Toom-8's interpolation constants (|N| < 2^44) as N = hi 2^32 + lo with lo
// and hi signed 32-bit integers, so that every product with a child digit is
// one 32 x 32 -> 64-bit multiply-add (and the int64 sum lo + hi 2^32 is formed
// once per digit).
struct InterpSplit {
    int32_t lo[15][15], hi[15][15];
};
constexpr InterpSplit split_interp8() {
    InterpSplit r{};
    for (int m = 0; m < 15; ++m)
        for (int t = 0; t < 15; ++t) {
            const long long c = kToom8InterpHost[m][t];
            long long low = c & 0xFFFFFFFFLL;
            if (low >= (1LL << 31)) low -= (1LL << 32);
            r.lo[m][t] = static_cast<int32_t>(low);
            r.hi[m][t] = static_cast<int32_t>((c - low) / (1LL << 32));
        }
    return r;
}
__constant__ InterpSplit kToom8Split = split_interp8();
template <int K>
struct Toom;
template <>
struct Toom<4> {
    static constexpr int P = 7;
    static constexpr uint64_t Den1 = 360, Den2 = 1;  // Den = Den1 Den2, divided in that order
    static constexpr bool kWide = false;             // constants fit 32 bits: no high halves
    __device__ static int eval(int t, int k) { return kToom4Eval[t][k]; }
    __device__ static int32_t lo(int m, int t) { return kToom4Interp[m][t]; }
    __device__ static int32_t hi(int, int) { return 0; }
};
template <>
struct Toom<6> {
    static constexpr int P = 11;
    static constexpr uint64_t Den1 = 1008000, Den2 = 1;
    static constexpr bool kWide = false;
    __device__ static int eval(int t, int k) { return kToom6Eval[t][k]; }
    __device__ static int32_t lo(int m, int t) { return kToom6Interp[m][t]; }
    __device__ static int32_t hi(int, int) { return 0; }
};
template <>
struct Toom<8> {
    static constexpr int P = 15;
    static constexpr uint64_t Den1 = 7776000, Den2 = 7007;
    static constexpr bool kWide = true;
    __device__ static int eval(int t, int k) { return kToom8Eval[t][k]; }
    __device__ static int32_t lo(int m, int t) { return kToom8Split.lo[m][t]; }
    __device__ static int32_t hi(int m, int t) { return kToom8Split.hi[m][t]; }
};
static_assert(split_interp8().hi[1][0] * (1LL << 32) + split_interp8().lo[1][0] == kToom8InterpHost[1][0],
              "split of the interpolation constants");

// Sign-magnitude rows (L32 limbs) -> the children's rows (Lc limbs): child t
// gets E_t = sum_k eval(t, k) V_k times the entry's sign, as a sign and a
// magnitude (|E_t| < 2^(32 Lc)).  One warp per (row, point): limb q of E_t
// is first the int64 sum sum_k eval(t, k) V_k[q] (|.| < 2^45), then the warp
// carries base 2^32 (4 consecutive limbs per lane, carries passed up one
// lane per round until none is left), a window of 128 limbs at a time; a
// final carry of -1 means E_t < 0 and the limbs, its two's complement, are
// negated in place.
constexpr int kSplitLimbs = 4;  // limbs per lane per window
__device__ __forceinline__ void warp_carry32(long long (&v)[kSplitLimbs], uint32_t (&o)[kSplitLimbs], int lane,
                                             long long &wcarry) {
    long long c = (lane == 0) ? wcarry : 0;
#pragma unroll
    for (int i = 0; i < kSplitLimbs; ++i) {
        const long long t = v[i] + c;
        o[i] = static_cast<uint32_t>(t);
        c = t >> 32;  // arithmetic: floor
    }
    long long pending = c, out = 0;
    for (int round = 0; round <= 32; ++round) {
        out += __shfl_sync(0xffffffffu, pending, 31);
        long long incoming = __shfl_up_sync(0xffffffffu, pending, 1);
        if (lane == 0) incoming = 0;
        if (!__any_sync(0xffffffffu, incoming != 0)) break;
        c = incoming;
#pragma unroll
        for (int i = 0; i < kSplitLimbs; ++i) {
            const long long t = static_cast<long long>(o[i]) + c;
            o[i] = static_cast<uint32_t>(t);
            c = t >> 32;
        }
        pending = c;
    }
    wcarry = out;
}
template <int K>
__global__ void __launch_bounds__(256) k_toom_split(const uint32_t *__restrict__ limbs, const uint8_t *__restrict__ neg,
                                                    int rows, int L32, int sl, int Lc, uint32_t *const *__restrict__ dst,
                                                    uint8_t *const *__restrict__ dneg) {
    constexpr int P = Toom<K>::P;
    const int lane = threadIdx.x & 31;
    const long long w = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w >= static_cast<long long>(rows) * P) return;  // warp-uniform
    const int k = static_cast<int>(w / P), t = static_cast<int>(w % P);
    const uint32_t *m = limbs + static_cast<size_t>(k) * L32;
    uint32_t *o = dst[t] + static_cast<size_t>(k) * Lc;
    int c[K];
#pragma unroll
    for (int p = 0; p < K; ++p) c[p] = Toom<K>::eval(t, p);
    long long wc = 0;
    for (int q0 = 0; q0 < Lc; q0 += 32 * kSplitLimbs) {
        long long v[kSplitLimbs];
        uint32_t r[kSplitLimbs];
#pragma unroll
        for (int i = 0; i < kSplitLimbs; ++i) {
            const int q = q0 + kSplitLimbs * lane + i;  // limb q of every part V_p
            long long e = 0;
#pragma unroll
            for (int p = 0; p < K; ++p) {
                const int li = p * sl + q;
                if (q < sl && li < L32) e += static_cast<long long>(c[p]) * m[li];
            }
            v[i] = e;
        }
        warp_carry32(v, r, lane, wc);
#pragma unroll
        for (int i = 0; i < kSplitLimbs; ++i) {
            const int q = q0 + kSplitLimbs * lane + i;
            if (q < Lc) o[q] = r[i];
        }
    }
    __syncwarp();
    // wc: 0 (E >= 0) or -1 (the limbs are 2^(32 Lc) + E); |E| < 2^(32 Lc) by the children's width
    if (wc < 0) {
        int q0 = Lc;  // lowest non-zero limb
        for (int q = lane; q < Lc; q += 32)
            if (o[q]) { q0 = q; break; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) q0 = min(q0, __shfl_xor_sync(0xffffffffu, q0, off));
        for (int q = lane; q < Lc; q += 32) {
            if (q == q0) o[q] = ~o[q] + 1u;
            else if (q > q0) o[q] = ~o[q];
        }
        __syncwarp();
    }
    bool any = false;
    for (int q = lane; q < Lc; q += 32) any |= o[q] != 0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) {
        const bool eneg = (wc < 0) != (neg[k] != 0);
        dneg[t][k] = (any && eneg) ? 1 : 0;
    }
}

// The children's exact rows are carry-save digit vectors of int16 (bit t of
// in16_mask) or int32 digits; four consecutive digits from digit v (a
// multiple of 4, as are the row widths).
__device__ __forceinline__ int4 child4(const int32_t *z, bool is16, size_t at) {
    if (is16) {
        const uint2 w = *reinterpret_cast<const uint2 *>(reinterpret_cast<const int16_t *>(z) + at);
        return make_int4(static_cast<int16_t>(w.x & 0xFFFFu), static_cast<int>(w.x) >> 16,
                         static_cast<int16_t>(w.y & 0xFFFFu), static_cast<int>(w.y) >> 16);
    }
    return *reinterpret_cast<const int4 *>(z + at);
}
struct ToomChildren {
    const int32_t *z[15];
};

// Exact division of the limbs z[0 .. nl) (little-endian) by Den < 2^24 by one
// warp.  Long division from the top limb carries the remainder
// r -> (r 2^32 + z_w) mod Den, an affine map of r modulo Den: each lane
// composes the maps of its segment of limbs (lane 0 the most significant
// segment), a warp scan composes the segments, and every lane then divides its
// own segment from the remainder that enters it.  Returns (on every lane)
// whether the remainder is zero.
template <uint64_t Den>
__device__ bool warp_div_exact(uint32_t *z, int nl, int lane) {
    static_assert(Den > 1 && Den < (1ull << 24), "r 2^32 + z must fit 64 bits");
    constexpr uint64_t K32 = (uint64_t(1) << 32) % Den;
    const int seg = (nl + 31) / 32;
    const int hi = max(0, nl - lane * seg), lo = max(0, nl - (lane + 1) * seg);
    constexpr int kPre = 8;  // limbs loaded ahead of the serial chains (the row lives in L2)
    uint64_t A = 1, B = 0;   // this segment's map r -> (A r + B) mod Den
    for (int w0 = hi - 1; w0 >= lo; w0 -= kPre) {
        uint32_t zz[kPre];
#pragma unroll
        for (int k = 0; k < kPre; ++k) zz[k] = (w0 - k >= lo) ? z[w0 - k] : 0u;
#pragma unroll
        for (int k = 0; k < kPre; ++k)
            if (w0 - k >= lo) {
                A = (A * K32) % Den;
                B = (B * K32 + zz[k]) % Den;
            }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {  // inclusive scan: maps of lanes 0..l, applied in lane order
        const uint64_t pa = __shfl_up_sync(0xffffffffu, A, off);
        const uint64_t pb = __shfl_up_sync(0xffffffffu, B, off);
        if (lane >= off) {
            B = (A * pb + B) % Den;
            A = (A * pa) % Den;
        }
    }
    uint64_t r = __shfl_up_sync(0xffffffffu, B, 1);  // remainder entering this segment
    if (lane == 0) r = 0;
    for (int w0 = hi - 1; w0 >= lo; w0 -= kPre) {
        uint32_t zz[kPre];
#pragma unroll
        for (int k = 0; k < kPre; ++k) zz[k] = (w0 - k >= lo) ? z[w0 - k] : 0u;
#pragma unroll
        for (int k = 0; k < kPre; ++k)
            if (w0 - k >= lo) {
                const uint64_t cur = (r << 32) | zz[k];  // r < Den < 2^24: no overflow
                const uint64_t q = cur / Den;
                r = cur - q * Den;
                z[w0 - k] = static_cast<uint32_t>(q);
            }
    }
    // lane 31 holds the lowest segment (or none, and the whole remainder)
    return __shfl_sync(0xffffffffu, r, 31) == 0;
}

// Den Z as int64 carry-save digits: z[u] = sum_m sum_t N[m][t] P_t[u - m ds]
// (|z[u]| < 2^62, checked when the plan is made), one block per row, four
// digits per thread; every product of a constant half with a child digit is
// one 32 x 32 -> 64-bit multiply-add.
template <int K>
__global__ void __launch_bounds__(256) k_toom_combine(ToomChildren ch, int in16_mask, int Wc, int ds,
                                                      int64_t *__restrict__ out, int Wp) {
    constexpr int P = Toom<K>::P;
    const int i = blockIdx.x;
    const size_t crow = static_cast<size_t>(i) * Wc;
    for (int g = threadIdx.x; g < Wp / 4; g += blockDim.x) {
        const int u = 4 * g;
        long long l0 = 0, l1 = 0, l2 = 0, l3 = 0, h0 = 0, h1 = 0, h2 = 0, h3 = 0;
        const int m_lo = max(0, (u - Wc) / ds), m_hi = min(P - 1, u / ds);
        for (int mm = m_lo; mm <= m_hi; ++mm) {
            const int v = u - mm * ds;
            if (v < 0 || v >= Wc) continue;
#pragma unroll
            for (int t = 0; t < P; ++t) {
                const int32_t cl = Toom<K>::lo(mm, t), chh = Toom<K>::hi(mm, t);
                if (cl == 0 && chh == 0) continue;
                const int4 d = child4(ch.z[t], (in16_mask >> t) & 1, crow + v);
                l0 += static_cast<long long>(cl) * d.x;
                l1 += static_cast<long long>(cl) * d.y;
                l2 += static_cast<long long>(cl) * d.z;
                l3 += static_cast<long long>(cl) * d.w;
                if (Toom<K>::kWide) {
                    h0 += static_cast<long long>(chh) * d.x;
                    h1 += static_cast<long long>(chh) * d.y;
                    h2 += static_cast<long long>(chh) * d.z;
                    h3 += static_cast<long long>(chh) * d.w;
                }
            }
        }
        constexpr long long k32 = 1LL << 32;
        int64_t *o = out + static_cast<size_t>(i) * Wp + u;
        reinterpret_cast<longlong2 *>(o)[0] = make_longlong2(l0 + h0 * k32, l1 + h1 * k32);
        reinterpret_cast<longlong2 *>(o)[1] = make_longlong2(l2 + h2 * k32, l3 + h3 * k32);
    }
}

// The rest of a Toom plan's rows, one warp per row, in one pass over Den Z's
// int64 digits (k_toom_combine):
//   1. the carry into base-256 digits (warp_carry), a window of 1024 digits
//      at a time (each lane reads 32 consecutive digits), packed into limbs
//      of the row; a final carry of -1 means Den Z < 0 and the limbs hold its
//      two's complement, which is negated in place;
//   2. the exact division by Den, in factors below 2^24;
//   3. the bit length of |Z| and its maximum over rows.
constexpr int kTailWarps = 8;
constexpr int kTailWin = 32 * kDigitsPerLane;  // digits per window
template <int K>
__global__ void __launch_bounds__(32 * kTailWarps) k_toom_finish(const int64_t *__restrict__ in, int Wo, int n,
                                                                 uint32_t *__restrict__ zmag,
                                                                 uint8_t *__restrict__ zneg,
                                                                 int32_t *__restrict__ zbits, int ZW, int32_t *dstat,
                                                                 int row_offset) {
    const int lane = threadIdx.x & 31;
    const int i = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (i >= n) return;  // warp-uniform
    const int64_t *row = in + static_cast<size_t>(i) * Wo;
    uint32_t *z = zmag + static_cast<size_t>(row_offset + i) * ZW;
    const int WL = Wo / 4;  // limbs of Den Z
    long long wc = 0;
    bool bad = false;
    // limbs past the row's WL (windows end at multiples of kTailWin): all zero
    // for Den Z >= 0, all ones (the sign extension) for Den Z < 0
    bool above_nonzero = false, above_not_ones = false;
    for (int u0 = 0; u0 < Wo; u0 += kTailWin) {
        long long d[kDigitsPerLane];
        const int ub0 = u0 + kDigitsPerLane * lane;
#pragma unroll
        for (int g = 0; g < kDigitsPerLane / 2; ++g) {  // Wo is a multiple of 4
            const longlong2 w = (ub0 + 2 * g < Wo) ? *reinterpret_cast<const longlong2 *>(row + ub0 + 2 * g)
                                                   : make_longlong2(0, 0);
            d[2 * g] = w.x;
            d[2 * g + 1] = w.y;
        }
        warp_carry<false, long long>(d, lane, wc);
        const int ub = u0 + kDigitsPerLane * lane;
#pragma unroll
        for (int w = 0; w < kDigitsPerLane / 4; ++w) {
            const uint32_t limb = static_cast<uint32_t>(d[4 * w]) | (static_cast<uint32_t>(d[4 * w + 1]) << 8) |
                                  (static_cast<uint32_t>(d[4 * w + 2]) << 16) |
                                  (static_cast<uint32_t>(d[4 * w + 3]) << 24);
            const int li = ub / 4 + w;
            if (li < WL) {
                z[li] = limb;
            } else {
                above_nonzero |= limb != 0u;
                above_not_ones |= limb != 0xFFFFFFFFu;
            }
        }
    }
    for (int w = WL + lane; w < ZW; w += 32) z[w] = 0u;
    // wc is the same on every lane: 0 (Den Z >= 0) or -1 (the limbs below WL
    // are 2^(32 WL) + Den Z); anything else, or limbs above WL that are not the
    // sign extension, means Den Z does not fit the row
    const bool negative = wc == -1;
    if (wc != 0 && wc != -1) bad = true;
    if (negative ? above_not_ones : above_nonzero) bad = true;
    __syncwarp();
    if (negative) {
        int k0 = WL;  // lowest non-zero limb
        for (int w = lane; w < WL; w += 32)
            if (z[w]) { k0 = w; break; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) k0 = min(k0, __shfl_xor_sync(0xffffffffu, k0, off));
        if (k0 == WL) bad = true;  // -2^(32 WL) does not fit
        for (int w = lane; w < WL; w += 32) {
            if (w == k0) z[w] = ~z[w] + 1u;
            else if (w > k0) z[w] = ~z[w];
        }
        __syncwarp();
    }
    bool exact = warp_div_exact<Toom<K>::Den1>(z, WL, lane);
    __syncwarp();
    if constexpr (Toom<K>::Den2 > 1) {
        exact = warp_div_exact<Toom<K>::Den2>(z, WL, lane) && exact;
        __syncwarp();
    }
    int bits = 0;
    for (int w = lane; w < WL; w += 32)
        if (z[w]) bits = 32 * w + (32 - __clz(z[w]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    if ((__any_sync(0xffffffffu, bad) || !exact) && lane == 0) set_status(dstat, DEV_OVERFLOW);
    if (lane == 0) {
        zbits[row_offset + i] = bits;
        zneg[row_offset + i] = (bits > 0 && negative) ? 1 : 0;
        atomicMax(dstat + 1, bits);
    }
}

// Interpolation (k_toom_combine), then normalisation, exact division and bit
// lengths of a Toom plan's rows (k_toom_finish).
cudaError_t launch_toom_tail(hmv_plan_s *p, int rhs) {
    ToomChildren ch;
    int mask = 0, wc = 0;
    for (size_t t = 0; t < p->children.size(); ++t) {
        hmv_plan_s *c = p->children[t];  // unsplit children
        ch.z[t] = c->post[0];
        mask |= c->post16 ? (1 << t) : 0;
        wc = c->Wo;
    }
    const int ds = p->split_bits / 8;
    const unsigned rows = static_cast<unsigned>(p->n);  // one block per row
    const unsigned blocks = static_cast<unsigned>((p->n + kTailWarps - 1) / kTailWarps);  // a warp per row
    const int ro = rhs * p->n;
    if (p->toom == 4) {
        k_toom_combine<4><<<rows, 256, 0, p->stream>>>(ch, mask, wc, ds, p->combined64, p->Wo);
        k_toom_finish<4><<<blocks, 32 * kTailWarps, 0, p->stream>>>(p->combined64, p->Wo, p->n, p->zmag, p->zneg,
                                                                    p->zbits, p->ZW, p->dstat, ro);
    } else if (p->toom == 6) {
        k_toom_combine<6><<<rows, 256, 0, p->stream>>>(ch, mask, wc, ds, p->combined64, p->Wo);
        k_toom_finish<6><<<blocks, 32 * kTailWarps, 0, p->stream>>>(p->combined64, p->Wo, p->n, p->zmag, p->zneg,
                                                                    p->zbits, p->ZW, p->dstat, ro);
    } else {
        k_toom_combine<8><<<rows, 256, 0, p->stream>>>(ch, mask, wc, ds, p->combined64, p->Wo);
        k_toom_finish<8><<<blocks, 32 * kTailWarps, 0, p->stream>>>(p->combined64, p->Wo, p->n, p->zmag, p->zneg,
                                                                    p->zbits, p->ZW, p->dstat, ro);
    }
    p->launches_total += 2;
    return cudaGetLastError();
}

// Split rows of a vector into the three children's staging buffers,
// recursively down to the unsplit plans.
cudaError_t split_down(hmv_plan_s *p, const uint32_t *limbs, const uint8_t *neg, int rows, bool matrix) {
    if (p->children.empty()) return cudaSuccess;
    if (p->toom) {
        const int P = static_cast<int>(p->children.size());
        uint32_t *const *ddst = p->toom_ptrs + (matrix ? 0 : P);  // the same rows, uploaded at plan creation
        uint8_t *const *dn = p->toom_neg_ptrs + (matrix ? 0 : P);
        const unsigned blocks = static_cast<unsigned>((static_cast<long long>(rows) * P + 7) / 8);  // a warp per (row, point)
        const int sl = p->split_bits / 32, Lc = p->children[0]->L32;
        if (p->toom == 4)
            k_toom_split<4><<<blocks, 256, 0, p->stream>>>(limbs, neg, rows, p->L32, sl, Lc, ddst, dn);
        else if (p->toom == 6)
            k_toom_split<6><<<blocks, 256, 0, p->stream>>>(limbs, neg, rows, p->L32, sl, Lc, ddst, dn);
        else
            k_toom_split<8><<<blocks, 256, 0, p->stream>>>(limbs, neg, rows, p->L32, sl, Lc, ddst, dn);
        p->launches_total++;
        return cudaGetLastError();
    }
    hmv_plan_s *c0 = p->children[0], *c1 = p->children[1], *cm = p->children[2];
    uint32_t *dst[3];
    uint8_t *dneg[3];
    for (int t = 0; t < 3; ++t) {
        dst[t] = matrix ? p->children[t]->h_limbs_d : p->children[t]->x_limbs_d;
        dneg[t] = matrix ? p->children[t]->h_neg_d : p->children[t]->x_neg_d;
    }
    k_split<<<(rows + 127) / 128, 128, 0, p->stream>>>(limbs, neg, rows, p->L32, p->split_bits / 32, c0->L32,
                                                       dst[0], dst[1], dst[2], dneg[0], dneg[1], dneg[2]);
    p->launches_total++;
    cudaError_t e = cudaGetLastError();
    (void)c1;
    (void)cm;
    for (int t = 0; t < 3 && e == cudaSuccess; ++t)
        e = split_down(p->children[t], dst[t], dneg[t], rows, matrix);
    return e;
}

// The exact digit vector of a plan's rows after its post-pass (unsplit) or
// after combining its children (split).
cudaError_t combine_up(hmv_plan_s *p, const int32_t **out, int *width, int *digit_bytes) {
    if (p->children.empty()) {
        *out = p->post[0];
        *width = p->Wo;
        *digit_bytes = p->post16 ? 2 : 4;
        return cudaSuccess;
    }
    if (p->toom) return cudaErrorNotSupported;  // Toom plans finish in launch_toom_tail
    const int32_t *z[3];
    int w[3];
    bool s16[3];
    for (int t = 0; t < 3; ++t) {
        int bytes = 4;
        cudaError_t e = combine_up(p->children[t], &z[t], &w[t], &bytes);
        if (e != cudaSuccess) return e;
        if (bytes == 8) return cudaErrorNotSupported;  // Toom plans are never children
        s16[t] = bytes == 2;
    }
    const int mask = (s16[0] ? 1 : 0) | (s16[2] ? 2 : 0) | (s16[1] ? 4 : 0);
    const dim3 grid(static_cast<unsigned>(p->n), static_cast<unsigned>(std::min(65535, (p->Wo + 255) / 256)));
    k_combine<<<grid, 256, 0, p->stream>>>(z[0], z[2], z[1], mask, w[0], p->n, p->split_bits / 8, p->combined, p->Wo);
    p->launches_total++;
    *out = p->combined;
    *width = p->Wo;
    *digit_bytes = 4;
    return cudaGetLastError();
}

}  // namespace

void collect_leaf_plans(hmv_plan_s *p, std::vector<hmv_plan_s *> &out) {
    if (p->children.empty()) {
        out.push_back(p);
        return;
    }
    for (hmv_plan_s *c : p->children) collect_leaf_plans(c, out);
}

// Children of a split plan (called from plan_create).
hmv_status split_plan_create(hmv_plan_s *p, const hmv_desc &d, int digit_levels) {
    p->split_bits = 32 * ((p->L32 + 1) / 2);
    const int bc = p->split_bits + 1;  // lo, hi < 2^s; lo + hi < 2^(s+1)
    for (int t = 0; t < 3; ++t) {
        hmv_desc cd = d;
        cd.b = bc;
        cd.nrhs = 1;
        cd.kind = HMV_HANKEL;       // the parent maps the kind onto the Hankel sequence
        cd.method = HMV_KARATSUBA;
        cd.flags &= ~(HMV_FLAG_TIMING | HMV_FLAG_DIGIT_SPLIT1 | HMV_FLAG_DIGIT_SPLIT2);
        if (p->tn == 128) cd.flags |= HMV_FLAG_TILE128;
        if (digit_levels > 1) cd.flags |= HMV_FLAG_DIGIT_SPLIT1;
        cd.levels = -1;
        hmv_plan_s *c = nullptr;
        hmv_status st = plan_create(&cd, p->stream, false, &c, p->dry_run);
        if (st != HMV_OK) return st;
        p->children.push_back(c);
        p->device_bytes += c->device_bytes;
    }
    int wc = p->children[0]->Wo;
    for (hmv_plan_s *c : p->children) wc = std::max(wc, c->Wo);
    p->Wo = 2 * (p->split_bits / 8) + wc;
    p->ZW = p->Wo / 4;
    double macs = 0, issued = 0;
    for (hmv_plan_s *c : p->children) {
        macs += c->leaf_macs;
        issued += c->leaf_macs_issued;
    }
    p->leaf_macs = macs;
    p->leaf_macs_issued = issued;
    return HMV_OK;
}

// 2K-1 unsplit children of s + g bits (|E_t| < 15 * 2^s for K = 4, 364 * 2^s
// for K = 6, 6305 * 2^s for K = 8), s = the limb boundary nearest above b/K.
hmv_status toom_plan_create(hmv_plan_s *p, const hmv_desc &d, int K) {
    p->toom = K;
    const int P = 2 * K - 1, grow = (K == 4) ? 4 : ((K == 6) ? 9 : 13);
    p->split_bits = 32 * ((p->L32 + K - 1) / K);
    for (int t = 0; t < P; ++t) {
        hmv_desc cd = d;
        cd.b = p->split_bits + grow;
        cd.nrhs = 1;
        cd.kind = HMV_HANKEL;  // the parent maps the kind onto the Hankel sequence
        cd.method = HMV_KARATSUBA;
        cd.flags &= ~(HMV_FLAG_TIMING | HMV_FLAG_DIGIT_SPLIT1 | HMV_FLAG_DIGIT_SPLIT2 | HMV_FLAG_DIGIT_TOOM4 |
                      HMV_FLAG_DIGIT_TOOM6 | HMV_FLAG_DIGIT_TOOM8 | HMV_FLAG_TILE256);
        if (p->tn == 128) cd.flags |= HMV_FLAG_TILE128;
        cd.levels = -1;
        hmv_plan_s *c = nullptr;
        hmv_status st = plan_create(&cd, p->stream, false, &c, p->dry_run);
        if (st != HMV_OK) return st;
        p->children.push_back(c);
        p->device_bytes += c->device_bytes;
    }
    if (K == 8) {
        // the int64 interpolation sums: at most ceil(Wc / ds) shifted products
        // meet at a digit, each sum_t |N[m][t]| |d| with |d| <= 510 * 2^L
        const hmv_plan_s *c = p->children[0];
        double rowsum = 0;
        for (const auto &row : kToom8InterpHost) {
            double r = 0;
            for (long long v : row) r += std::fabs(static_cast<double>(v));
            rowsum = std::max(rowsum, r);
        }
        const double overlap = std::ceil(static_cast<double>(c->Wo) / (p->split_bits / 8)) + 1;
        if (overlap * rowsum * 510.0 * std::ldexp(1.0, c->L) >= std::ldexp(1.0, 62)) return HMV_EUNSUPPORTED;
    }
    // Den Z spans the 2K-2 shifted products plus one child row and the factor Den
    p->Wo = (2 * K - 2) * (p->split_bits / 8) + p->children[0]->Wo + 4;
    p->ZW = p->Wo / 4;
    double macs = 0, issued = 0;
    for (hmv_plan_s *c : p->children) {
        macs += c->leaf_macs;
        issued += c->leaf_macs_issued;
    }
    p->leaf_macs = macs;
    p->leaf_macs_issued = issued;
    return HMV_OK;
}

// Matrix side: map the kind onto a Hankel sequence of 2n-1 entries, split it
// for every descendant and load the unsplit plans.
hmv_status split_load_matrix(hmv_plan_s *p, const uint32_t *h_limbs, const uint8_t *h_neg) {
    cudaError_t e = split_down(p, h_limbs, h_neg, 2 * p->n - 1, true);
    if (e != cudaSuccess) return HMV_ECUDA;
    std::vector<hmv_plan_s *> leaves;
    collect_leaf_plans(p, leaves);
    for (hmv_plan_s *c : leaves) {
        hmv_vec v;
        memset(&v, 0, sizeof v);
        v.len = 2 * c->n - 1;
        v.nrhs = 1;
        v.b = c->b;
        v.exponent = 0;
        v.limbs = c->h_limbs_d;
        v.neg = c->h_neg_d;
        v.on_device = 1;
        hmv_status st = hmv_load_matrix(c, &v);
        if (st != HMV_OK) return st;
    }
    return HMV_OK;
}

// One right-hand side, in three phases so that the caller can time the leaf
// launch: (1) split x and run the vector side of every unsplit plan; (2) one
// leaf launch for all of them; (3) their post-passes, the combines, and the
// exact rows of right-hand side `rhs` in the top plan.
cudaError_t split_vector_side(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn) {
    cudaError_t e = split_down(p, xl, xn, p->n, false);
    std::vector<hmv_plan_s *> leaves;
    collect_leaf_plans(p, leaves);
    for (hmv_plan_s *c : leaves) c->stream = p->stream;
    if (e == cudaSuccess && same_geometry(leaves.data(), static_cast<int>(leaves.size())))
        return launch_vector_side_group(leaves.data(), static_cast<int>(leaves.size()));
    for (hmv_plan_s *c : leaves) {
        if (e != cudaSuccess) break;
        c->stream = p->stream;
        e = launch_encode(c, c->x_limbs_d, c->x_neg_d, c->n, 0, c->x_lvl[0]);
        for (int l = 0; l < c->L && e == cudaSuccess; ++l)
            e = launch_prepass(c, l, false, c->x_lvl[l % 2], c->x_lvl[(l + 1) % 2]);
        if (e == cudaSuccess) e = launch_pack_vector(c, c->x_lvl[c->L % 2]);
    }
    return e;
}

cudaError_t split_leaf_launch(hmv_plan_s *p) {
    cudaError_t e = cudaSuccess;
    if (!p->split_probs) {
        // the set of unsplit plans is fixed: build and upload the combined lists once
        std::vector<hmv_plan_s *> leaves;
        collect_leaf_plans(p, leaves);
        std::vector<LeafProblem> probs;
        std::vector<Tile> tiles;
        for (hmv_plan_s *c : leaves) {
            const int idx = static_cast<int>(probs.size());
            probs.push_back(c->hprob);
            for (Tile t : c->tiles) {
                t.prob = idx;
                tiles.push_back(t);
            }
        }
        // from the library's pool in the plan's stream order; the host lists
        // live until the stream has copied them
        void *dp = nullptr, *dt = nullptr;
        e = pool_alloc(&dp, probs.size() * sizeof(LeafProblem), p->stream);
        if (e == cudaSuccess) p->allocations.push_back(dp);
        if (e == cudaSuccess) e = pool_alloc(&dt, tiles.size() * sizeof(Tile), p->stream);
        if (e == cudaSuccess) p->allocations.push_back(dt);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp, probs.data(), probs.size() * sizeof(LeafProblem), cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e == cudaSuccess) {
            p->split_probs = static_cast<LeafProblem *>(dp);
            p->split_tiles = static_cast<Tile *>(dt);
        }
        p->ntiles = static_cast<int>(tiles.size());
    }
    if (e == cudaSuccess) {
        const hmv_plan_s *q = p;
        while (!q->children.empty()) q = q->children[0];  // every unsplit descendant has the same width
        e = launch_leaf_tc_multi(p->split_probs, p->split_tiles, p->ntiles, p->dstat, p->d_counter, p->stream,
                                 p->num_sms, q->tn);
        p->launches_leaf++;
        p->launches_total++;
    }
    return e;
}

cudaError_t split_post(hmv_plan_s *p, int rhs) {
    std::vector<hmv_plan_s *> leaves;
    collect_leaf_plans(p, leaves);
    cudaError_t e = cudaSuccess;
    if (same_geometry(leaves.data(), static_cast<int>(leaves.size()))) {
        e = launch_post_group(leaves.data(), static_cast<int>(leaves.size()));
    } else {
        for (hmv_plan_s *c : leaves) {
            if (e != cudaSuccess) break;
            e = launch_post_group(&c, 1);  // leaf normalise and every post-pass level
        }
    }
    if (e == cudaSuccess) {
        if (p->toom) {
            e = launch_toom_tail(p, rhs);
        } else {
            const int32_t *z = nullptr;
            int w = 0, zb = 4;
            e = combine_up(p, &z, &w, &zb);
            if (e == cudaSuccess) e = launch_final_normalize(p, z, rhs, zb);
        }
    }
    for (hmv_plan_s *c : leaves) {
        p->launches_total += c->launches_total;
        c->launches_total = 0;
    }
    return e;
}

namespace {
__global__ void k_wrap(const uint32_t *__restrict__ c, const uint8_t *__restrict__ cn, int n, int L32,
                       uint32_t *__restrict__ h, uint8_t *__restrict__ hn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * n - 1) return;
    const int src = ((n - 1 - k) % n + n) % n;  // circulant -> Toeplitz sequence
    for (int q = 0; q < L32; ++q) h[static_cast<size_t>(k) * L32 + q] = c[static_cast<size_t>(src) * L32 + q];
    hn[k] = cn[src];
}
}  // namespace

cudaError_t launch_wrap_circulant(hmv_plan_s *p, const uint32_t *c_limbs, const uint8_t *c_neg) {
    k_wrap<<<(2 * p->n - 1 + 127) / 128, 128, 0, p->stream>>>(c_limbs, c_neg, p->n, p->L32, p->h_wrap,
                                                                p->h_wrap_neg);
    p->launches_total++;
    return cudaGetLastError();
}

}  // namespace hmv
