// warp_reduce.cuh -- the warp reduction of per-record gradient sums shared by
// the blend adjoints (hybrid and sorted).
#pragma once

#include "common.cuh"

namespace htgs {

__device__ __forceinline__ float2 shfl_xor2(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Sums 16 per-lane values over the warp; afterwards lane 8q (q = 0..3) holds
// the sums of values 4q .. 4q + 3 in v[0..3]. The first two exchanges halve
// the values each lane carries (each half of the warp keeps one half of them),
// the last three sum the remaining four; the adds run on value pairs.
__device__ __forceinline__ void warp_reduce16_to4(float (&v)[16], int lane) {
    float2 P[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) P[i] = make_float2(v[2 * i], v[2 * i + 1]);
    const bool up16 = lane & 16, up8 = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 send = up16 ? P[i] : P[i + 4];
        const float2 keep = up16 ? P[i + 4] : P[i];
        P[i] = fadd2(keep, shfl_xor2(send, 16));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float2 send = up8 ? P[i] : P[i + 2];
        const float2 keep = up8 ? P[i + 2] : P[i];
        P[i] = fadd2(keep, shfl_xor2(send, 8));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 2; ++i) P[i] = fadd2(P[i], shfl_xor2(P[i], o));
    v[0] = P[0].x; v[1] = P[0].y; v[2] = P[1].x; v[3] = P[1].y;
}

} // namespace htgs
