// Inline-PTX wrappers for the Blackwell (sm_103a) tensor-core path:
// mbarriers with bounded waits, TMA tiled loads, tcgen05 TMEM allocation,
// MMA issue/commit, TMEM loads and shared-memory matrix descriptors.
#pragma once
#include <cstdint>
#include <cuda.h>

namespace hmv {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete.  Gives up after
// timeout_ns of wall time and returns false; never spins forever.
// The waits count the time spent polling: the global timer's increments
// between consecutive polls, each capped at kPollGapNs.  The timer keeps
// running while a descheduled launch does not poll (a GPU time-sliced with
// another context), and such a stretch counts as one capped gap, so it
// cannot run a wait out by itself; every wait still ends, after at least
// timeout_ns of polling.
constexpr uint64_t kPollGapNs = 1000000;  // 1 ms: far above one poll
__device__ __forceinline__ void poll_clock(uint64_t &last, uint64_t &waited) {
    const uint64_t now = global_ns();
    const uint64_t d = now - last;
    waited += d < kPollGapNs ? d : kPollGapNs;
    last = now;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t last = global_ns(), waited = 0;
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        poll_clock(last, waited);
        if (waited > timeout_ns) return false;
    }
}
// The same wait, which also gives up as soon as *abort is set (another role
// of the CTA has failed, so the phase it waits for may never complete).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns,
                                          const volatile int *abort) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t last = global_ns(), waited = 0;
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        poll_clock(last, waited);
        if (*abort || waited > timeout_ns) return false;
    }
}

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// ------------------------------------------------------------------ tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// N consecutive MMAs along K from one asm block: MMA k reads A at
// adesc + k * A_STEP bytes and B at bdesc + k * B_STEP bytes (the descriptor
// start-address field counts 16-byte units; both start fields must stay
// below 2^14 after the additions).  The first MMA accumulates into D when
// accumulate != 0, the others always do.  One block rather than N separate
// statements measurably shortens the issue path of the thread.
#define HMV_MMA_HEAD                                       \
    "{\n\t.reg .pred p, t;\n\t.reg .b64 a, b;\n\t"         \
    "setp.ne.b32 p, %4, 0;\n\tsetp.eq.u32 t, 0, 0;\n\t"    \
    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
#define HMV_MMA_NEXT(ia, ib)                                                  \
    "add.s64 a, %1, %" #ia ";\n\tadd.s64 b, %2, %" #ib ";\n\t" \
    "tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, t;\n\t"
#define HMV_MMA_ARGS "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
#define HMV_MMA_OFF(k) "n"((k) * A_STEP / 16), "n"((k) * B_STEP / 16)
#define HMV_MMA_N2 HMV_MMA_NEXT(5, 6)
#define HMV_MMA_N3 HMV_MMA_N2 HMV_MMA_NEXT(7, 8)
#define HMV_MMA_N4 HMV_MMA_N3 HMV_MMA_NEXT(9, 10)
#define HMV_MMA_N5 HMV_MMA_N4 HMV_MMA_NEXT(11, 12)
#define HMV_MMA_N6 HMV_MMA_N5 HMV_MMA_NEXT(13, 14)
#define HMV_MMA_N7 HMV_MMA_N6 HMV_MMA_NEXT(15, 16)
#define HMV_MMA_N8 HMV_MMA_N7 HMV_MMA_NEXT(17, 18)
#define HMV_MMA_N9 HMV_MMA_N8 HMV_MMA_NEXT(19, 20)
#define HMV_MMA_N10 HMV_MMA_N9 HMV_MMA_NEXT(21, 22)
#define HMV_MMA_O2 HMV_MMA_OFF(1)
#define HMV_MMA_O3 HMV_MMA_O2, HMV_MMA_OFF(2)
#define HMV_MMA_O4 HMV_MMA_O3, HMV_MMA_OFF(3)
#define HMV_MMA_O5 HMV_MMA_O4, HMV_MMA_OFF(4)
#define HMV_MMA_O6 HMV_MMA_O5, HMV_MMA_OFF(5)
#define HMV_MMA_O7 HMV_MMA_O6, HMV_MMA_OFF(6)
#define HMV_MMA_O8 HMV_MMA_O7, HMV_MMA_OFF(7)
#define HMV_MMA_O9 HMV_MMA_O8, HMV_MMA_OFF(8)
#define HMV_MMA_O10 HMV_MMA_O9, HMV_MMA_OFF(9)
template <uint32_t A_STEP, uint32_t B_STEP, int N>
struct MmaRun;
template <uint32_t A_STEP, uint32_t B_STEP>
struct MmaRun<A_STEP, B_STEP, 1> {
    static __device__ __forceinline__ void run(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
        asm volatile(HMV_MMA_HEAD "}\n" ::HMV_MMA_ARGS : "memory");
    }
};
#define HMV_MMA_RUN(N)                                                                                           \
    template <uint32_t A_STEP, uint32_t B_STEP>                                                                  \
    struct MmaRun<A_STEP, B_STEP, N> {                                                                           \
        static_assert(A_STEP % 16 == 0 && B_STEP % 16 == 0, "descriptor steps are 16-byte units");             \
        static __device__ __forceinline__ void run(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, \
                                                   uint32_t accumulate) {                                        \
            asm volatile(HMV_MMA_HEAD HMV_MMA_N##N "}\n" ::HMV_MMA_ARGS, HMV_MMA_O##N : "memory");              \
        }                                                                                                        \
    };
HMV_MMA_RUN(2)
HMV_MMA_RUN(3)
HMV_MMA_RUN(4)
HMV_MMA_RUN(5)
HMV_MMA_RUN(6)
HMV_MMA_RUN(7)
HMV_MMA_RUN(8)
HMV_MMA_RUN(9)
HMV_MMA_RUN(10)
#undef HMV_MMA_RUN
// Eight MMAs: one j-step of a full K = 128 s-block.
template <uint32_t A_STEP, uint32_t B_STEP>
__device__ __forceinline__ void mma_bf16_ss_k128(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                 uint32_t accumulate) {
    MmaRun<A_STEP, B_STEP, 8>::run(d_tmem, adesc, bdesc, idesc, accumulate);
}
// 1 <= count <= 10 MMAs with the count known at run time: one branch per
// call, then one block.
template <uint32_t A_STEP, uint32_t B_STEP>
__device__ __forceinline__ void mma_bf16_ss_run(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate, int count) {
    switch (count) {
        case 1: MmaRun<A_STEP, B_STEP, 1>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 2: MmaRun<A_STEP, B_STEP, 2>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 3: MmaRun<A_STEP, B_STEP, 3>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 4: MmaRun<A_STEP, B_STEP, 4>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 5: MmaRun<A_STEP, B_STEP, 5>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 6: MmaRun<A_STEP, B_STEP, 6>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 7: MmaRun<A_STEP, B_STEP, 7>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 8: MmaRun<A_STEP, B_STEP, 8>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        case 9: MmaRun<A_STEP, B_STEP, 9>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
        default: MmaRun<A_STEP, B_STEP, 10>::run(d_tmem, adesc, bdesc, idesc, accumulate); break;
    }
}
// Arrive on bar once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 TMEM lanes x 32 consecutive 32-bit columns: thread t of the warp gets
// lane (base lane + t), columns col .. col+31.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes stored contiguously (rows 16 B apart);
// lbo = byte step between core matrices adjacent along K,
// sbo = byte step between core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
    return d;                             // base offset 0, no swizzle
}

// Instruction descriptor: kind::f16 with bf16 A and B, fp32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4)            // D format: f32
           | (1u << 7)          // A format: bf16
           | (1u << 10)         // B format: bf16
           | ((N >> 3) << 17)   // N / 8
           | ((M >> 4) << 24);  // M / 16
}

}  // namespace hmv
