// common.cuh -- shared device helpers and the internal launch structures of
// the sm_103a renderer (arXiv 2410.08129, Sec. 3.2-3.3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/htgs.h"

namespace htgs {

// ---------------------------------------------------------------------------
// Internal argument blocks (passed by value as kernel parameters).
// ---------------------------------------------------------------------------

struct CamArgs {
    float M[12];          // rows 0..2 of the row-major world-to-camera matrix
    float fx, fy, cx, cy; // pinhole intrinsics in window coordinates
    float z_near;
    float centre[3];      // camera centre in world space
    int width, height;
};

struct ParamArgs {
    int K;
    float tau_alpha, tau_K, alpha_max;
    float bg[3];
    int no_tail;  // 1: the tail is omitted (core over the background)
    int sorted_blend;  // 1: mean-depth-sorted alpha blending with early termination
};

// Sorted blending stops before the fragment that would take T below this.
constexpr float kSortedTmin = 1e-4f;

struct TileArgs {
    int tile_w, tile_h;
    int tiles_x, tiles_y;
    int n_tiles;
    int tile_bits;   // bits of the sort key holding the tile id
    int depth_bits;  // low key bits holding quantised depth
    int batch;       // records per shared-memory batch of the forward blend
};

// Per-Gaussian blend record: 32 floats = 128 bytes = 8 float4.
//   [0] q0, d0, q1, d1        Q and D coefficients, interleaved in pairs
//   [1] q2, d2, q3, d3
//   [2] q4, d4, q5, d5
//   [3] z0, z1, z2, z3        Z = (view depth) * D coefficients
//   [4] z4, z5, xc, yc        ... and the expansion centre (box centre)
//   [5] r, g, b, rho_c        colour and cutoff
//   [6] x0, x1, y0, y1        screen bounding box p -+ h (slightly widened)
//   [7] zlo, -, -, -          lower bound on the view depth of every kept
//                             fragment: the cutoff ellipsoid's nearest z,
//                             lowered by a margin that covers rounding
// Each quadratic is c0 + c1 x' + c2 y' + c3 x'^2 + c4 x'y' + c5 y'^2 in the
// offsets (x', y') = (x - xc, y - yc) of the pixel centre. With
// N = ||m||^2 (m the Pluecker moment) and D = ||d||^2 (d the direction),
// Q = log2(e) (rho_c D - N) / 2, so that rho^2 = N / D <= rho_c <=> Q >= 0
// and alpha = o e^{-rho^2/2} = tau_alpha * 2^{Q / D}. The (Q, D) pairs let
// one packed FP32x2 evaluation produce both.
constexpr int kRecF4 = 8;

// Device status word layout (int32 array at the front of the workspace).
enum StatusSlot {
    kStError = 0,      // htgs_status of the last device-side failure (0 = none)
    kStInstLo = 1,     // total instances of the last render (low 32 bits)
    kStInstHi = 2,
    kStSlots = 16
};

// ---------------------------------------------------------------------------
// Small numeric helpers. The forward and backward must evaluate alpha and
// depth bit-identically, so these use explicit round-to-nearest intrinsics
// that the compiler cannot re-associate or contract differently.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 fused multiply-add (sm_100 and later): two independent
// round-to-nearest fmas, bit-identical to the scalar ones.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// The (Q, D) pair of a record at pixel offset (x, y): the same evaluation
// order as quad_eval, applied to both coefficient sets at once.
__device__ __forceinline__ float2 quad_eval2(const float4 &c01, const float4 &c23, const float4 &c45,
                                             float x, float y) {
    const float2 X = make_float2(x, x), Y = make_float2(y, y);
    const float2 p0 = make_float2(c01.x, c01.y), p1 = make_float2(c01.z, c01.w);
    const float2 p2 = make_float2(c23.x, c23.y), p3 = make_float2(c23.z, c23.w);
    const float2 p4 = make_float2(c45.x, c45.y), p5 = make_float2(c45.z, c45.w);
    const float2 tx = ffma2(p4, Y, ffma2(p3, X, p1));
    const float2 ty = ffma2(p5, Y, p2);
    return ffma2(Y, ty, ffma2(X, tx, p0));
}

// c0 + x (c1 + c3 x + c4 y) + y (c2 + c5 y), fixed evaluation order.
__device__ __forceinline__ float quad_eval(float c0, float c1, float c2, float c3, float c4,
                                           float c5, float x, float y) {
    float tx = __fmaf_rn(c4, y, __fmaf_rn(c3, x, c1));
    float ty = __fmaf_rn(c5, y, c2);
    return __fmaf_rn(y, ty, __fmaf_rn(x, tx, c0));
}

// 16-byte asynchronous global -> shared copy (L2 only); completion is
// awaited with cp_async_wait<N>, which waits for this thread's own copies.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

// Work counters (uint64 array in the workspace, zeroed by every render).
enum StatSlot {
    kStatBoxPairs = 0,   // sum over Gaussians of the pixels inside the tight bounding box
    kStatKept = 1,       // fragments with rho^2 <= rho_c (every pixel)
    kStatAdmitted = 2,   // kept fragments with alpha >= tau_K
    kStatInserted = 3,   // core insertions
    kStatSlots = 8
};

__device__ __forceinline__ void set_error(int *status, int code) {
    atomicCAS(status + kStError, 0, code);
}

} // namespace htgs
