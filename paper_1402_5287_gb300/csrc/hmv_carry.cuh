// Warp-parallel carry propagation over base-256 digits, shared by the
// digit kernels (encode, normalise) and the Toom interpolation.
#pragma once
#include <cuda_runtime.h>

namespace hmv {

// Renormalisation of one window of 32 x kDigitsPerLane digits, held
// kDigitsPerLane per lane (lane l: window digits kDigitsPerLane*l ..), to
// balanced digits in [-128, 127] (kBalanced) or digits in [0, 256).  Each lane
// runs a local carry chain, then the carries leaving the lanes are passed up
// by one lane and absorbed until none is left: after round r only lanes
// above r can hold a new carry, so at most 32 rounds.  wcarry: the carry into
// lane 0 on entry, the carry out of lane 31 on return (all lanes).
constexpr int kDigitsPerLane = 32;
template <bool kBalanced, class D>
__device__ __forceinline__ D norm_digit(D t, D &carry) {
    if (kBalanced) {
        carry = (t + 128) >> 8;  // floor((t + 128) / 256)
        return t - (carry << 8);
    }
    carry = t >> 8;  // floor division by 256
    return t & 255;
}
template <bool kBalanced, class D>
__device__ __forceinline__ void warp_carry(D (&d)[kDigitsPerLane], int lane, D &wcarry) {
    D c = (lane == 0) ? wcarry : D(0);
#pragma unroll
    for (int q = 0; q < kDigitsPerLane; ++q) d[q] = norm_digit<kBalanced, D>(d[q] + c, c);
    D pending = c, out = 0;
    for (int round = 0; round <= 32; ++round) {
        out += __shfl_sync(0xffffffffu, pending, 31);
        D incoming = __shfl_up_sync(0xffffffffu, pending, 1);
        if (lane == 0) incoming = 0;
        if (!__any_sync(0xffffffffu, incoming != 0)) break;
        c = incoming;
#pragma unroll
        for (int q = 0; q < kDigitsPerLane; ++q) d[q] = norm_digit<kBalanced, D>(d[q] + c, c);
        pending = c;
    }
    wcarry = out;
}
}  // namespace hmv
