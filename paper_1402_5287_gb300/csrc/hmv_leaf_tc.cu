// Leaf products of Algorithm 1 (Beliakov, arXiv:1402.5287, Sec. 3) on the
// sm_103a tensor cores.
//
// A leaf is a small exact Hankel product p_i = sum_{j<m} a_{i+j} x_j whose
// entries are big integers held as balanced radix-2^8 digits.  In digits,
//     Y[i][u] = sum_{j<m} sum_s a_{i+j}[s] * x_j[u-s],
// a GEMM with M = i (leaf rows), N = u (product digits), K = (j, s):
//   * A[i][(j,s)] = a_{i+j}[s] is Hankel in the index: one staged slab of
//     rows of the leaf sequence serves every shift j by moving the
//     descriptor start by j rows (16 bytes), never materialising the matrix;
//   * B[u][(j,s)] = x_j[u-s] is Toeplitz in the digits: with K ordered by
//     descending s, core matrix (n-group g, k-group c) depends only on g + c,
//     so one row of 8x8 blocks (8 shifted copies of x_j, loaded by TMA) with
//     both descriptor strides equal to 128 bytes is the whole operand.
// Digits (|d| <= 128) are exact in bf16; products are <= 2^14; an fp32
// accumulation window of 1024 products keeps every partial sum within 2^24,
// so each window is an exact integer.  The epilogue reads each window from
// TMEM, converts it to int32 and adds it into the tile's exact value kept as
// 256 base-256 digits per row plus a carry word (carry propagation in
// registers), so nothing but the final digits ever leaves the SM.
//
// Warp roles (192 threads): warp 0 issues TMA loads, warp 1 allocates TMEM
// and one lane issues tcgen05.mma, warps 2-5 run the epilogue on the four
// TMEM lane quarters.  128-digit tiles add warp 6 as a second MMA issuer:
// one thread cannot issue 128 x 128 x 16 MMAs (about 65 cycles of tensor
// work each) as fast as the tensor pipe runs them once its loop waits on
// barriers, two threads together can; the two take alternate j-steps of a
// tile into accumulators of their own, and the epilogue adds the pair.
// Tiles are handed out in list order from a global counter (the producer
// takes the next index and passes it to the CTA's consumers through a small
// shared-memory queue), so the grid works on neighbouring tiles of the same
// leaves and their operands stay in L2.  Two fp32 accumulators per issuer
// (all 512 TMEM columns: 2 x 256, or 2 x 2 x 128 on 128-wide tiles) let the
// MMAs of one window overlap the epilogue of the previous one.
// On 128-wide tiles each staged s-block is a frame of KS + 32 digits, so a
// tile's last s-block, when it holds only one or two K = 16 groups below
// s_max, is issued with the block below it (j-steps of 9 or 10 MMAs instead
// of separate steps of 1 or 2, which the issuing threads cannot keep up with).
// Every wait is bounded (wait_ns, 2 s by default) and gives up early once
// another role of the CTA has failed; on a timeout the kernel records
// DEV_TIMEOUT, waits for its own MMAs and for the TMA loads it has issued to
// complete, frees its TMEM and returns.
#include <atomic>
#include <cstring>

#include "hmv_internal.h"
#include "tc_ptx.cuh"

namespace hmv {
namespace {

constexpr int kProducerWarp = 0;
constexpr int kMmaWarp = 1;
constexpr int kNumEpiWarps = 4;
constexpr int kMmaWarp2 = 2 + kNumEpiWarps;  // second issuer of 128-digit tiles
// Tile width in product digits: 256 (one 128x256 MMA per k-step) or 128
// (narrow operands, where the wide tile's triangular edges waste more).
template <int TNv>
struct Geo {
    static constexpr int NI = TNv == 128 ? 2 : 1;           // MMA-issuing threads
    static constexpr int kThreads = (2 + kNumEpiWarps + NI - 1) * 32;
    // Digits of one staged s-block frame: KS, and on 128-wide tiles 32 more
    // above them, so that a last s-block of at most two K = 16 groups joins
    // the block below it (10-group frame) instead of making j-steps of one or
    // two MMAs.  A normal block issues the frame's groups G0 .. G0 + 7.
    static constexpr int KF = TNv == 128 ? KS + 32 : KS;
    static constexpr int G0 = (KF - KS) / 16;
    static constexpr int AB = AR * KF * 2;                  // bf16 bytes of one staged Hankel slab
    static constexpr int NEv = TNv / 8 + KF / 8 - 1;        // core matrices of one shifted-x operand
    static constexpr int BB = NEv * 128;                    // its bytes
    static constexpr int BS = TNv == 256 ? 8 : 16;          // B ring slots (even: see the issuers)
    static constexpr uint32_t kTmemCols = 2 * TNv * NI;     // two accumulators per issuer
    static constexpr uint32_t kIdesc = idesc_bf16_f32(TM, TNv);
    static_assert(BS % 2 == 0 && kTmemCols <= 512, "ring and TMEM layout");
};
constexpr uint32_t kLboA = AR * 16;  // K-direction core-matrix step of the slab
constexpr int kTileQ = 4;            // tile indices handed from the producer to the consumers
constexpr int kTileConsumers = 1 + kNumEpiWarps;  // plus the second issuer where there is one

template <int TNv>
struct __align__(1024) Smem {
    uint8_t a[A_STAGES][Geo<TNv>::AB];
    uint8_t b[Geo<TNv>::BS][Geo<TNv>::BB];
    uint64_t a_full[A_STAGES], a_empty[A_STAGES];
    uint64_t b_full[Geo<TNv>::BS], b_empty[Geo<TNv>::BS];
    uint64_t acc_full[Geo<TNv>::NI][2], acc_empty[Geo<TNv>::NI][2];
    uint64_t tq_full[kTileQ], tq_empty[kTileQ];
    int tile_q[kTileQ];
    uint64_t drain[Geo<TNv>::NI];
    uint32_t tmem_base;
    volatile int abort;
};

struct TileInfo {
    const LeafProblem *pr;
    int leaf, i0, ub, u0, m, s_base, nsb, njc, Q, Dl, Dp;
    int fg;  // first frame group the last s-block issues (those above lie wholly above s_max: zero products)
};

template <int TNv>
__device__ __forceinline__ TileInfo decode(const Tile &t, const LeafProblem *probs) {
    TileInfo ti;
    ti.pr = probs + t.prob;
    const int Dl = ti.pr->Dl;
    ti.Dl = Dl;
    ti.Dp = ti.pr->Dp;
    const int *size = ti.pr->size;
    ti.leaf = t.leaf;
    ti.i0 = t.i0;
    ti.ub = t.ub;
    ti.u0 = t.ub * TNv;
    ti.m = size[t.leaf];
    // s-blocks of KS digits start at the tile's first useful digit (rounded
    // down to 8 for the TMA coordinates), not at multiples of KS
    const int s_min = max(0, ti.u0 - (Dl - 1));
    const int s_max = min(Dl - 1, ti.u0 + TNv - 1);
    ti.s_base = s_min / 8 * 8;
    ti.nsb = (s_max >= s_min) ? (s_max - ti.s_base + KS) / KS : 0;
    const int kk0 = ti.nsb ? (ti.s_base + ti.nsb * KS - 1 - s_max) / 16 : 0;  // groups of digits above s_max
    using G = Geo<TNv>;
    if (G::G0 > 0 && ti.nsb >= 2 && KS / 16 - kk0 <= G::G0) {
        --ti.nsb;  // the last block's groups ride on the block below, in its frame's top G0 groups
        ti.fg = G::G0 - (KS / 16 - kk0);
    } else {
        ti.fg = G::G0 + kk0;
    }
    ti.njc = (ti.m + JC - 1) / JC;
    ti.Q = ti.nsb * ti.m;
    return ti;
}

// Exact accumulation windows of 128-wide tiles: a j-step of s-block sb
// issues step_groups K = 16 groups (16 products per column each); an fp32
// window takes kWinGroups of them (1024 products), so a window spans
// window_span consecutive j-steps of one s-block, half of them (alternate
// steps) each issuer's.  Short steps (the trimmed last block) thus get long
// windows, and both issuers' windows cover the same steps.
constexpr int kWinGroups = FLUSH_J * (KS / 16);
__device__ __forceinline__ int step_groups(const TileInfo &ti, int sb) {
    return (sb + 1 < ti.nsb) ? KS / 16 : Geo<128>::KF / 16 - ti.fg;
}
__device__ __forceinline__ int window_span(const TileInfo &ti, int sb) {
    return 2 * (kWinGroups / step_groups(ti, sb));
}

template <class S>
__device__ __forceinline__ void fail(S &sm, int32_t *dstat) {
    sm.abort = 1;
    set_status(dstat, DEV_TIMEOUT);
}

// Bounded wait for the latest TMA load issued into each slot marked in
// `pending` (bit s; its phase parity is bit s of `phases`): copies still in
// flight after an abort must land before the shared memory is released.
// Earlier loads into a slot have landed: the slot was released before reuse.
__device__ __forceinline__ void wait_issued_loads(uint64_t *full, uint32_t pending, uint32_t phases, uint64_t wait_ns,
                                                  int32_t *dstat) {
    for (int s = 0; pending >> s; ++s)
        if (((pending >> s) & 1u) && !mbar_wait(&full[s], (phases >> s) & 1u, wait_ns)) set_status(dstat, DEV_TIMEOUT);
}

template <int TNv>
__global__ void __launch_bounds__(Geo<TNv>::kThreads, 1)
    k_leaf_tc(const LeafProblem *__restrict__ probs, const Tile *__restrict__ tiles, int ntiles, int *tile_counter,
              int32_t *dstat, uint64_t wait_ns, int stall) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    using G = Geo<TNv>;
    constexpr int NI = G::NI;
    constexpr int B_STAGES = G::BS;
    constexpr int B_BYTES = G::BB;
    constexpr int TN = TNv;
    Smem<TNv> &sm = *reinterpret_cast<Smem<TNv> *>(smem_raw);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int s = 0; s < A_STAGES; ++s) { mbar_init(&sm.a_full[s], 1); mbar_init(&sm.a_empty[s], NI); }
        for (int s = 0; s < B_STAGES; ++s) { mbar_init(&sm.b_full[s], 1); mbar_init(&sm.b_empty[s], 1); }
        for (int w = 0; w < NI; ++w)
            for (int s = 0; s < 2; ++s) {
                mbar_init(&sm.acc_full[w][s], 1);
                mbar_init(&sm.acc_empty[w][s], kNumEpiWarps);
            }
        for (int s = 0; s < kTileQ; ++s) {
            mbar_init(&sm.tq_full[s], 1);
            mbar_init(&sm.tq_empty[s], kTileConsumers + NI - 1);
        }
        for (int w = 0; w < NI; ++w) mbar_init(&sm.drain[w], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(&sm.tmem_base, G::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    if (warp == kProducerWarp) {
        if (lane == 0) {
            int as = 0, aph = 0, bs = 0, bph = 0;
            // slots whose latest load was issued (bit s) and that load's phase parity
            uint32_t a_pend = 0, a_phs = 0, b_pend = 0, b_phs = 0;
            static_assert(A_STAGES <= 32 && B_STAGES <= 32, "one bit per ring slot");
            for (int k = 0; !sm.abort; ++k) {
                // next tile in list order for the whole grid, handed to this CTA's consumers
                const int qs = k % kTileQ, qph = (k / kTileQ) & 1;
                if (!mbar_wait(&sm.tq_empty[qs], qph ^ 1, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                int t = atomicAdd(tile_counter, 1);
                if (t >= ntiles) t = -1;
                sm.tile_q[qs] = t;
                mbar_arrive(&sm.tq_full[qs]);
                if (t < 0) break;
                const TileInfo ti = decode<TNv>(tiles[t], probs);
                const CUtensorMap *mapA = &ti.pr->mapA;
                const CUtensorMap *mapB = &ti.pr->mapB;
                const int Dp = ti.Dp;
                for (int sb = 0; sb < ti.nsb && !sm.abort; ++sb) {
                    const int s_lo = ti.s_base + sb * KS;
                    for (int jc = 0; jc < ti.njc && !sm.abort; ++jc) {
                        const int j0 = jc * JC;
                        const int jn = min(JC, ti.m - j0);
                        if (!mbar_wait(&sm.a_empty[as], aph ^ 1, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                        mbar_arrive_expect_tx(&sm.a_full[as], G::AB);
                        tma_load_4d(sm.a[as], mapA, &sm.a_full[as], 0, (ti.i0 + j0) / 32, (Dp - s_lo - G::KF) / 8,
                                    ti.leaf);
                        a_pend |= 1u << as;
                        a_phs = (a_phs & ~(1u << as)) | (static_cast<uint32_t>(aph) << as);
                        if (++as == A_STAGES) { as = 0; aph ^= 1; }
                        for (int jj = 0; jj < jn; ++jj) {
                            if (!mbar_wait(&sm.b_empty[bs], bph ^ 1, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                            mbar_arrive_expect_tx(&sm.b_full[bs], B_BYTES);
                            tma_load_4d(sm.b[bs], mapB, &sm.b_full[bs], 0, (ti.u0 - s_lo - G::KF) / 8 + 1, j0 + jj,
                                        ti.leaf);
                            b_pend |= 1u << bs;
                            b_phs = (b_phs & ~(1u << bs)) | (static_cast<uint32_t>(bph) << bs);
                            if (++bs == B_STAGES) { bs = 0; bph ^= 1; }
                        }
                    }
                }
            }
            // every load issued has landed before the shared memory is released
            // (without an abort the issuers have waited for all of them already;
            // another role may abort after this thread has left its loop)
            wait_issued_loads(sm.a_full, a_pend, a_phs, wait_ns, dstat);
            wait_issued_loads(sm.b_full, b_pend, b_phs, wait_ns, dstat);
        }
    } else if (warp == kMmaWarp && NI == 1) {
        if (lane == 0) {
            int as = 0, aph = 0, bs = 0, bph = 0, ab = 0;
            int accph[2] = {0, 0};
            const uint32_t a_base0 = smem_u32(sm.a[0]);
            const uint32_t b_base0 = smem_u32(sm.b[0]);
            for (int k = 0; !sm.abort; ++k) {
                const int qs = k % kTileQ, qph = (k / kTileQ) & 1;
                if (!mbar_wait(&sm.tq_full[qs], qph, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                const int t = sm.tile_q[qs];
                mbar_arrive(&sm.tq_empty[qs]);
                if (t < 0) break;
                const TileInfo ti = decode<TNv>(tiles[t], probs);
                int q = 0;
                uint32_t acc_flag = 0;
                for (int sb = 0; sb < ti.nsb && !sm.abort; ++sb) {
                    for (int jc = 0; jc < ti.njc && !sm.abort; ++jc) {
                        const int jn = min(JC, ti.m - jc * JC);
                        if (!mbar_wait(&sm.a_full[as], aph, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                        const uint32_t a_base = a_base0 + as * G::AB;
                        for (int jj = 0; jj < jn; ++jj) {
                            if (q % FLUSH_J == 0) {
                                if (!mbar_wait(&sm.acc_empty[0][ab], accph[ab] ^ 1, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                                acc_flag = 0;
                            }
                            if (!mbar_wait(&sm.b_full[bs], bph, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                            tc_fence_after();
                            const uint32_t b_base = b_base0 + bs * B_BYTES;
                            const uint32_t d_tmem = tmem + ab * TN;
                            // K = 16 steps: A two slab chunks on, B two core matrices on
                            static_assert(KS == 128, "eight K = 16 MMAs per j-step");
                            mma_bf16_ss_k128<2 * kLboA, 256>(d_tmem, smem_desc(a_base + jj * 16, kLboA, 128),
                                                             smem_desc(b_base, 128, 128), G::kIdesc, acc_flag);
                            acc_flag = 1;
                            mma_commit(&sm.b_empty[bs]);
                            if (++bs == B_STAGES) { bs = 0; bph ^= 1; }
                            ++q;
                            if (q % FLUSH_J == 0 || q == ti.Q) {
                                mma_commit(&sm.acc_full[0][ab]);
                                accph[ab] ^= 1;
                                ab ^= 1;
                            }
                        }
                        mma_commit(&sm.a_empty[as]);
                        if (++as == A_STAGES) { as = 0; aph ^= 1; }
                    }
                }
            }
            // all MMAs issued by this thread complete before TMEM is released
            mma_commit(&sm.drain[0]);
            if (!mbar_wait(&sm.drain[0], 0, wait_ns)) fail(sm, dstat);
        }
    } else if (NI == 2 && (warp == kMmaWarp || warp == kMmaWarp2)) {
        // issuer w takes the tile's j-steps q = w, w + 2, ... (q counts the
        // tile's j-steps in the producer's order: s-block, then j); step q
        // is the producer's global step gq + q, whose B slot and phase follow
        // from the ring size, and every A slab is released by both issuers
        const int w = warp == kMmaWarp ? 0 : 1;
        if (lane == 0) {
            int as = 0, aph = 0, ab = 0, gq = 0;
            int accph[2] = {0, 0};
            const uint32_t a_base0 = smem_u32(sm.a[0]);
            const uint32_t b_base0 = smem_u32(sm.b[0]);
            // descriptors of the rings' first slots; the start-address field
            // counts 16-byte units (a shift j of the Hankel slab is + j), and
            // every address stays below 2^18, so offsets add without carry
            const uint64_t adesc0 = smem_desc(a_base0, kLboA, 128);
            const uint64_t bdesc0 = smem_desc(b_base0, 128, 128);
            const uint32_t tmem_w = tmem + static_cast<uint32_t>(w * 2 * TN);
            for (int k = 0; !sm.abort; ++k) {
                const int qs = k % kTileQ, qph = (k / kTileQ) & 1;
                if (!mbar_wait(&sm.tq_full[qs], qph, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                const int t = sm.tile_q[qs];
                mbar_arrive(&sm.tq_empty[qs]);
                if (t < 0) break;
                const TileInfo ti = decode<TNv>(tiles[t], probs);
                bool open = false;  // this issuer has a window open
                uint32_t acc_flag = 0;
                for (int sb = 0; sb < ti.nsb && !sm.abort; ++sb) {
                    const int span = window_span(ti, sb);
                    int wend = 0;  // j at which the open window ends (its s-block's windows start at multiples of span)
                    // frame groups this block issues: G0 .. G0 + 7, or fg .. KF / 16 - 1 in the last block
                    const int g0 = (sb + 1 < ti.nsb) ? G::G0 : ti.fg;
                    const int ng = G::KF / 16 - g0;
                    for (int jc = 0; jc < ti.njc && !sm.abort; ++jc) {
                        const int j0 = jc * JC;
                        const int jn = min(JC, ti.m - j0);
                        const int q0 = sb * ti.m + j0;  // tile step of jj = 0
                        if (!mbar_wait(&sm.a_full[as], aph, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                        const uint64_t adesc_s = adesc0 + static_cast<uint32_t>(as * G::AB + g0 * 2 * kLboA) / 16;
                        for (int jj = (q0 + w) & 1; jj < jn; jj += 2) {
                            if (j0 + jj >= wend) {  // close the open window, open the next (own steps are 2 apart, span >= 12)
                                if (open) {
                                    mma_commit(&sm.acc_full[w][ab]);
                                    accph[ab] ^= 1;
                                    ab ^= 1;
                                }
                                if (!mbar_wait(&sm.acc_empty[w][ab], accph[ab] ^ 1, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                                acc_flag = 0;
                                open = true;
                                wend += span;
                            }
                            const unsigned gs = static_cast<unsigned>(gq + q0 + jj);
                            const unsigned bs = gs % B_STAGES;
                            if (!mbar_wait(&sm.b_full[bs], (gs / B_STAGES) & 1u, wait_ns, &sm.abort)) { fail(sm, dstat); break; }
                            tc_fence_after();
                            const uint64_t ad = adesc_s + jj;
                            const uint64_t bd = bdesc0 + (bs * B_BYTES + g0 * 256) / 16;
                            if (ng == 8)
                                mma_bf16_ss_k128<2 * kLboA, 256>(tmem_w + ab * TN, ad, bd, G::kIdesc, acc_flag);
                            else  // the last s-block: without its groups above s_max, or with the next block's
                                mma_bf16_ss_run<2 * kLboA, 256>(tmem_w + ab * TN, ad, bd, G::kIdesc, acc_flag, ng);
                            acc_flag = 1;
                            mma_commit(&sm.b_empty[bs]);
                        }
                        mma_commit(&sm.a_empty[as]);
                        if (++as == A_STAGES) { as = 0; aph ^= 1; }
                    }
                }
                if (open && !sm.abort) {  // the tile's last window
                    mma_commit(&sm.acc_full[w][ab]);
                    accph[ab] ^= 1;
                    ab ^= 1;
                }
                gq += ti.Q;
            }
            mma_commit(&sm.drain[w]);
            if (!mbar_wait(&sm.drain[w], 0, wait_ns)) fail(sm, dstat);
        }
    } else {
        // epilogue: warp w serves TMEM lanes 32*(w%4) .. +31
        const int lq = warp % 4;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(lq * 32) << 16);
        // issuer w's accumulator pair: TMEM columns (2 w + ab) TN .. + TN - 1
        int ab[NI], eph[NI][2];
#pragma unroll
        for (int w = 0; w < NI; ++w) { ab[w] = 0; eph[w][0] = eph[w][1] = 0; }
        // the warp's 32 lanes wait together and take every decision together
        // (the TMEM loads below are warp-collective): results are voted
        for (int k = 0; !__any_sync(0xffffffffu, sm.abort); ++k) {
            const int qs = k % kTileQ, qph = (k / kTileQ) & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&sm.tq_full[qs], qph, wait_ns, &sm.abort))) { fail(sm, dstat); break; }
            const int t = sm.tile_q[qs];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.tq_empty[qs]);
            if (t < 0) break;
            const TileInfo ti = decode<TNv>(tiles[t], probs);
            // the tile's windows in order: one issuer, FLUSH_J j-steps each; two
            // issuers, window_span j-steps of one s-block each, of which either
            // issuer may have none (the next window starts at j-step wa of s-block wsb)
            const int nw_one = (ti.Q + FLUSH_J - 1) / FLUSH_J;
            int wsb = 0, wa = 0;
            uint32_t st[TN / 4];
#pragma unroll
            for (int w = 0; w < TN / 4; ++w) st[w] = 0;
            int co = 0;
            bool ok = true;
            for (int g = 0;; ++g) {
                bool one = true, two = false;  // issuer 0's / issuer 1's accumulator holds this window
                if (NI == 1) {
                    if (g >= nw_one) break;
                } else {
                    while (wsb < ti.nsb && wa >= ti.m) { ++wsb; wa = 0; }
                    if (wsb >= ti.nsb) break;
                    const int span = window_span(ti, wsb);
                    const int len = min(span, ti.m - wa);
                    const int p0 = (wsb * ti.m + wa) & 1;  // issuer of the window's first j-step
                    one = (len + (p0 == 0 ? 1 : 0)) / 2 > 0;
                    two = (len + (p0 == 1 ? 1 : 0)) / 2 > 0;
                    wa += span;
                }
                if (one) {
                    if (!__all_sync(0xffffffffu, mbar_wait(&sm.acc_full[0][ab[0]], eph[0][ab[0]], wait_ns, &sm.abort))) {
                        fail(sm, dstat);
                        ok = false;
                        break;
                    }
                    eph[0][ab[0]] ^= 1;
                }
                if (two) {
                    if (!__all_sync(0xffffffffu, mbar_wait(&sm.acc_full[NI - 1][ab[NI - 1]], eph[NI - 1][ab[NI - 1]],
                                                           wait_ns, &sm.abort))) {
                        fail(sm, dstat);
                        ok = false;
                        break;
                    }
                    eph[NI - 1][ab[NI - 1]] ^= 1;
                }
                tc_fence_after();
                int c = 0;
#pragma unroll
                for (int ch = 0; ch < TN / 32; ++ch) {
                    uint32_t v[32];
                    int x[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) x[e] = 0;
                    if (one) {
                        tmem_ld_32x32b_x32(lane_addr + ab[0] * TN + ch * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; ++e) x[e] = __float2int_rn(__uint_as_float(v[e]));
                    }
                    if (two) {
                        tmem_ld_32x32b_x32(lane_addr + (2 + ab[NI - 1]) * TN + ch * 32, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; ++e) x[e] += __float2int_rn(__uint_as_float(v[e]));
                    }
#pragma unroll
                    for (int q4 = 0; q4 < 8; ++q4) {
                        const uint32_t word = st[ch * 8 + q4];
                        uint32_t nw = 0;
#pragma unroll
                        for (int by = 0; by < 4; ++by) {
                            const int tt = static_cast<int>((word >> (8 * by)) & 0xFFu) + x[q4 * 4 + by] + c;
                            nw |= static_cast<uint32_t>(tt & 0xFF) << (8 * by);
                            c = tt >> 8;
                        }
                        st[ch * 8 + q4] = nw;
                    }
                }
                co += c;
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    // test hook (stall != 0): the first epilogue warp of the CTA that takes
                    // tile 0 keeps issuer 0's first accumulator, so that issuer's wait for
                    // it runs out and the abort path runs; never set outside tests
                    const bool keep = stall && t == 0 && g == 0 && warp == 2;
                    if (one && !keep) mbar_arrive(&sm.acc_empty[0][ab[0]]);
                    if (two) mbar_arrive(&sm.acc_empty[NI - 1][ab[NI - 1]]);
                }
                if (one) ab[0] ^= 1;
                if (two) ab[NI - 1] ^= 1;
            }
            if (!ok) break;
            const int row = ti.i0 + lq * 32 + lane;
            if (row < ti.m) {
                const LeafProblem &pr = *ti.pr;
                const size_t r = static_cast<size_t>(ti.leaf) * pr.MT * TM + row;
                uint4 *o = reinterpret_cast<uint4 *>(pr.dig + r * pr.Uo + ti.u0);
#pragma unroll
                for (int w = 0; w < TN / 16; ++w)
                    o[w] = make_uint4(st[4 * w], st[4 * w + 1], st[4 * w + 2], st[4 * w + 3]);
                pr.carry[r * pr.NUB + ti.ub] = co;
            }
        }
    }

    // every role has left its loop: the issuers' MMAs have completed (drain
    // barriers) and, after an abort, so have the producer's loads in flight
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, G::kTmemCols);
}

}  // namespace

template <int TNv>
cudaError_t prepare_one() {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf_tc<TNv>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sizeof(Smem<TNv>)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}

cudaError_t leaf_tc_prepare() {
    cudaError_t e = prepare_one<256>();
    if (e == cudaSuccess) e = prepare_one<128>();
    return e;
}

namespace {
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s for any single wait
// Test hook state (hmv_test_leaf_stall): launches still to run with the
// stall, and their wait limit.
std::atomic<int> g_stall_launches{0};
std::atomic<uint64_t> g_stall_wait_ns{kWaitNs};
}  // namespace

cudaError_t launch_leaf_tc_multi(const LeafProblem *probs, const Tile *tiles, int ntiles, int32_t *dstat,
                                 int *tile_counter, cudaStream_t stream, int num_sms, int tn) {
    cudaError_t pe = leaf_tc_prepare();
    if (pe != cudaSuccess) return pe;
    const int grid = std::min(ntiles, num_sms);
    if (grid <= 0) return cudaSuccess;
    cudaError_t me = cudaMemsetAsync(tile_counter, 0, sizeof(int), stream);
    if (me != cudaSuccess) return me;
    int stall = 0;
    uint64_t wait_ns = kWaitNs;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    // a captured launch would keep the hook in every replay of its graph: only direct launches take it
    for (int left = cap == cudaStreamCaptureStatusNone ? g_stall_launches.load() : 0; left > 0;)
        if (g_stall_launches.compare_exchange_weak(left, left - 1)) {
            stall = 1;
            wait_ns = g_stall_wait_ns.load();
            break;
        }
    if (tn == 128)
        k_leaf_tc<128><<<grid, Geo<128>::kThreads, sizeof(Smem<128>), stream>>>(probs, tiles, ntiles, tile_counter, dstat,
                                                                                wait_ns, stall);
    else
        k_leaf_tc<256><<<grid, Geo<256>::kThreads, sizeof(Smem<256>), stream>>>(probs, tiles, ntiles, tile_counter, dstat,
                                                                                wait_ns, stall);
    return cudaGetLastError();
}

cudaError_t launch_leaf_tc(hmv_plan_s *p) {
    p->launches_leaf++;
    p->launches_total++;
    return launch_leaf_tc_multi(p->d_prob, p->d_tiles, p->ntiles, p->dstat, p->d_counter, p->stream, p->num_sms,
                                p->tn);
}

// ------------------------------------------------------------------ tensor maps
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &ptr, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}
}  // namespace

cudaError_t encode_tensor_map_A(hmv_plan_s *p, CUtensorMap *map) {
    const int KF = p->tn == 128 ? Geo<128>::KF : Geo<256>::KF;
    EncodeTiledFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const int nleaves = p->lv[p->L].nodes;
    const cuuint64_t chunks = static_cast<cuuint64_t>(p->Dp / 8);
    // hrev[leaf][chunk][RA][8] bf16 (packed), read as rows of 32 matrix rows
    // (512 B): (256 elements, RA/32 row groups, chunks, leaf).  A box starts
    // at row i0 + j0, a multiple of 32, so it is whole row groups, and it
    // lands in shared memory in the same order as 8-element rows would.
    cuuint64_t dims[4] = {256, static_cast<cuuint64_t>(p->RA / 32), chunks, static_cast<cuuint64_t>(nleaves)};
    cuuint64_t strides[3] = {512, static_cast<cuuint64_t>(p->RA) * 16, chunks * p->RA * 16};
    cuuint32_t box[4] = {256, static_cast<cuuint32_t>(AR / 32), static_cast<cuuint32_t>(KF / 8), 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, p->hrev, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_tensor_map_B(hmv_plan_s *p, uint16_t *xg, CUtensorMap *map) {
    const int KF = p->tn == 128 ? Geo<128>::KF : Geo<256>::KF;
    EncodeTiledFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const int nleaves = p->lv[p->L].nodes;
    // xg[leaf][RX][chunk][8][8] bf16 (packed), one 128-byte core matrix per
    // row: (64 elements, chunks, j, leaf)
    const cuuint64_t xc = static_cast<cuuint64_t>(p->Dp / 8 + 1);
    cuuint64_t dims[4] = {64, xc, static_cast<cuuint64_t>(p->RX), static_cast<cuuint64_t>(nleaves)};
    cuuint64_t strides[3] = {128, xc * 128, static_cast<cuuint64_t>(p->RX) * xc * 128};
    cuuint32_t box[4] = {64, static_cast<cuuint32_t>(p->tn / 8 + KF / 8 - 1), 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, xg, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

void fill_leaf_problem(hmv_plan_s *p, LeafProblem &lp) {
    lp.size = p->lv[p->L].d_size;
    lp.dig = p->leaf_dig;
    lp.carry = p->leaf_carry;
    lp.Dl = p->Dl;
    lp.Dp = p->Dp;
    lp.Uo = p->Uo;
    lp.NUB = p->NUB;
    lp.MT = p->MT;
}

cudaError_t make_tensor_maps(hmv_plan_s *p) {
    LeafProblem lp;
    memset(&lp, 0, sizeof lp);
    cudaError_t e = encode_tensor_map_A(p, &lp.mapA);
    if (e == cudaSuccess) e = encode_tensor_map_B(p, p->xg, &lp.mapB);
    if (e != cudaSuccess) return e;
    p->mapA = lp.mapA;
    p->mapB = lp.mapB;
    fill_leaf_problem(p, lp);
    p->hprob = lp;
    e = cudaMemcpy(p->d_prob, &lp, sizeof lp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) p->maps_ok = true;
    return e;
}

}  // namespace hmv

extern "C" hmv_status hmv_test_leaf_stall(int32_t launches, int64_t wait_ns) {
    if (launches < 0 || wait_ns < 1000000 || wait_ns > 2000000000) return HMV_EINVAL;
    hmv::g_stall_wait_ns.store(static_cast<uint64_t>(wait_ns));
    hmv::g_stall_launches.store(launches);
    return HMV_OK;
}
