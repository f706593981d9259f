// What the tensor-core leaf kernel depends on: tile geometry, the exactness
// window, device status codes and the per-problem descriptor it reads.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace hmv {

// ---------------------------------------------------------------- geometry
// Leaf contraction tile: TM leaf rows x TN output digits (TN = 256, or 128
// per plan: hmv_plan_s::tn); each s-block holds KS digits of the matrix
// operand; JC shifts j share one staged slab.
constexpr int TM = 128;
constexpr int TN = 256;
constexpr int KS = 128;
constexpr int JC = 64;
constexpr int AR = TM + JC;                   // rows of one staged Hankel slab
static_assert(TM % 32 == 0 && JC % 32 == 0 && AR / 32 <= 256, "A slabs are whole 32-row groups");
constexpr int A_STAGES = 2;
// j-steps per exact fp32 accumulation window of 256-wide tiles: FLUSH_J * KS
// products of magnitude <= 2^14 keep every partial sum within 2^24 (128-wide
// tiles size their windows by the same 1024 products, counted in K groups).
constexpr int FLUSH_J = 1024 / KS;
constexpr int EXTRA_DIGITS = 8;               // room above the leaf product for carries
constexpr int TN_DEFAULT = 256;

// Device error codes written to the plan's status word.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADINPUT = 2, DEV_OVERFLOW = 3 };

// Records a failure in the status word; the first failure of a call stays
// (kernels that run after a failed stage may meet inconsistent data and must
// not replace the code of the failure that caused it).
__device__ __forceinline__ void set_status(int32_t *dstat, int code) { atomicCAS(dstat, DEV_OK, code); }

struct Tile {
    int leaf, i0, ub, cost, prob;  // prob: index into the launch's LeafProblem array
};

// Everything the leaf kernel needs to know about one leaf problem (one
// matrix tree with one right-hand side).  Lives in device memory; the TMA
// descriptors are read from here by the kernel.
struct __align__(128) LeafProblem {  // CUtensorMap is 128-byte aligned
    CUtensorMap mapA;   // bf16 Hankel slabs of the matrix leaves
    CUtensorMap mapB;   // bf16 shifted copies of the vector leaves
    const int *size;    // leaf orders
    uint8_t *dig;       // [leaf][MT*TM][Uo] output digits
    int32_t *carry;     // [leaf][MT*TM][NUB] output block carries
    int Dl, Dp, Uo, NUB, MT, pad_[3];
};

}  // namespace hmv
