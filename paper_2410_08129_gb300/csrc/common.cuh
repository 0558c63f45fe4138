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
    int cover;       // 0: per tile row the span the cutoff ellipse reaches; 1: the whole rectangle
};

// Per-Gaussian blend record: 32 floats = 128 bytes = 8 float4.
//   [0] q0, d0, q1, d1        Q and D coefficients, interleaved in pairs
//   [1] q2, d2, q3, d3
//   [2] q4, d4, q5, d5
//   [3] z0, z1, z2, z3        Z = (view depth) * D coefficients
//   [4] z4, z5, xc, yc        ... and the expansion centre (box centre)
//   [5] r, g, b, rho_c        colour and cutoff
//   [6] x0, x1, y0, y1        screen bounding box p -+ h (slightly widened)
//   [7] zlo, A11, A12, A22    lower bound on the view depth of every kept
//                             fragment (the cutoff ellipsoid's nearest z,
//                             lowered by a margin that covers rounding), and
//                             an ellipse p^T A p <= 1 about (xc, yc) that
//                             holds every pixel offset p with Q >= 0 (A = 0:
//                             none was found)
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

// First statement of every kernel: waits until the previous kernel of the
// stream has completed and its writes are visible (a no-op unless this
// kernel was launched as a programmatic dependent), then lets the next
// kernel's launch begin.
__device__ __forceinline__ void dependent_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Requests the 128-byte lines of [p, p + bytes) into L2 (no register, no
// completion to wait for), so that a load issued later finds them there.
__device__ __forceinline__ void prefetch_l2(const void *p, int bytes) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)127;
    const uintptr_t a1 = reinterpret_cast<uintptr_t>(p) + (uintptr_t)bytes;
    for (uintptr_t a = a0; a < a1; a += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// 16-byte asynchronous global -> shared copy (L2 only); completion is
// awaited with cp_async_wait<N>, which waits for this thread's own copies.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
// 4-byte asynchronous global -> shared copy (cached in L1 on the way).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem_src) : "memory");
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

// ---------------------------------------------------------------------------
// Tile cover of a record, row by row. Sec. 4.3 bins a Gaussian into the
// tiles it can reach; its bounding rectangle over-covers those of an
// elongated or tilted splat. Every pixel offset with Q >= 0 lies in the
// record's ellipse a x^2 + 2 b x y + c y^2 <= 1 (word 7), which is convex, so
// over the pixel-centre rows of one tile row its x-extent is an interval and
// the tiles it reaches form a contiguous span. Solving the ellipse for x
// gives x = -k y -+ sqrt(p - q y^2) with k = b / a, p = 1 / a and
// q = (a c - b^2) / a^2. The right end of the interval is the + root at the
// y of the rightmost point, y_r = -b / sqrt(c (a c - b^2)), clamped into the
// band (the root is concave in y), and the left end the - root at -y_r
// clamped. The preprocess sums the spans into the record's instance count
// and the binning kernels enumerate them: both run these same steps on the
// same stored inputs, so they get the same spans bit for bit (the
// approximate reciprocals and square roots are deterministic; their error,
// a few 1e-7 relative, is far inside the margins).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct RowCover {
    float xc, yc;   // ellipse centre in pixels
    float k, p, q;  // x-extent at offset y: -k y -+ sqrt(p - q y^2)
    float yr, ym;   // y offset of the rightmost point; half height (0: no ellipse, whole rows)
    float mx, my;   // margins added to both ends in x and y
    uint32_t tx0, tx1, ty0, ty1;  // the bounding rectangle in tiles
};

__device__ __forceinline__ RowCover row_cover(uint2 rect, float xc, float yc, float a, float b, float c,
                                              bool use_ellipse) {
    RowCover r;
    r.tx0 = rect.x & 0xffffu; r.tx1 = rect.x >> 16;
    r.ty0 = rect.y & 0xffffu; r.ty1 = rect.y >> 16;
    r.xc = xc; r.yc = yc;
    r.k = r.p = r.q = r.yr = r.ym = r.mx = r.my = 0.f;
    // A rectangle one tile wide keeps its rows whole: the ellipse spans the
    // box's rows, so it could only drop a row whose pixel centres it misses.
    if (!use_ellipse || r.tx0 == r.tx1 || !(a > 0.f) || !(c > 0.f)) return r;
    const float w = __fmul_rn(b, b);
    const float det = __fadd_rn(__fmaf_rn(a, c, -w), __fmaf_rn(-b, b, w));  // a c - b^2, compensated
    if (!(det > 0.f)) return r;
    const float ra = rcp_approx(a), rdet = rcp_approx(det);
    const float k = __fmul_rn(b, ra), q = __fmul_rn(__fmul_rn(det, ra), ra);
    const float xr = sqrt_approx(__fmul_rn(c, rdet)), ym = sqrt_approx(__fmul_rn(a, rdet));
    const float yr = __fmul_rn(-b, rcp_approx(sqrt_approx(__fmul_rn(c, det))));
    if (!isfinite(k) || !isfinite(q) || !isfinite(ra) || !isfinite(xr) || !isfinite(yr) || !(ym > 0.f) ||
        !isfinite(ym))
        return r;
    r.k = k; r.p = ra; r.q = q; r.yr = yr; r.ym = ym;
    // Relative to the ellipse's size the roots lose at most a few 1e-4 near
    // its top and bottom, where p - q y^2 cancels.
    r.mx = __fmaf_rn(2e-3f, xr, 0.02f);
    r.my = __fmaf_rn(2e-3f, ym, 0.02f);
    return r;
}

// Tiles [s0, s1] of tile row ty reached by the cover; returns the span's
// width (0 when the ellipse misses the row). tile_w is a power of two.
__device__ __forceinline__ uint32_t row_span(const RowCover &r, uint32_t ty, int tile_w, int tile_h,
                                             uint32_t &s0, uint32_t &s1) {
    s0 = r.tx0;
    s1 = r.tx1;
    if (r.ym > 0.f) {
        // Offsets of the row's first and last pixel-centre lines, widened.
        const float yb = __fsub_rn(__fadd_rn((float)(ty * (uint32_t)tile_h), 0.5f), r.yc);
        const float Y0 = __fsub_rn(yb, r.my);
        const float Y1 = __fadd_rn(__fadd_rn(yb, (float)(tile_h - 1)), r.my);
        if (Y0 > r.ym || Y1 < -r.ym) return 0u;
        const float yh = fminf(fmaxf(r.yr, Y0), Y1), yl = fminf(fmaxf(-r.yr, Y0), Y1);
        const float sh = sqrt_approx(fmaxf(__fmaf_rn(-r.q, __fmul_rn(yh, yh), r.p), 0.f));
        const float sl = sqrt_approx(fmaxf(__fmaf_rn(-r.q, __fmul_rn(yl, yl), r.p), 0.f));
        const float xh = __fmaf_rn(-r.k, yh, sh), xl = __fsub_rn(__fmul_rn(-r.k, yl), sl);
        // Pixels i whose centres i + 0.5 lie in [xc + xl - mx, xc + xh + mx],
        // clamped to the rectangle's pixels (a NaN end keeps the rectangle's:
        // fmaxf and fminf return the number), then their tiles.
        const float lo = ceilf(__fsub_rn(__fsub_rn(__fadd_rn(r.xc, xl), r.mx), 0.5f));
        const float hi = floorf(__fsub_rn(__fadd_rn(__fadd_rn(r.xc, xh), r.mx), 0.5f));
        const float f0 = fmaxf(lo, (float)(r.tx0 * (uint32_t)tile_w));
        const float f1 = fminf(hi, (float)(r.tx1 * (uint32_t)tile_w + (uint32_t)tile_w - 1u));
        if (!(f0 <= f1)) return 0u;
        const int shift = __ffs(tile_w) - 1;
        s0 = (uint32_t)f0 >> shift;
        s1 = (uint32_t)f1 >> shift;
    }
    return s1 - s0 + 1u;
}

// What the binning needs of a record, 32 bytes in an array of its own (the
// binning kernels read it instead of the 128-byte blend records):
//   uint4  [0] tx0 | tx1 << 16, ty0 | ty1 << 16, xc bits, yc bits
//   uint4  [1] a, b, c bits (the record's ellipse, word 7), 0
__device__ __forceinline__ void store_cover(uint4 *covers, int64_t rec, uint2 rect, float xc, float yc, float a,
                                            float b, float c) {
    covers[2 * rec] = make_uint4(rect.x, rect.y, __float_as_uint(xc), __float_as_uint(yc));
    covers[2 * rec + 1] = make_uint4(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c), 0u);
}

__device__ __forceinline__ RowCover load_cover(const uint4 *covers, uint32_t rec, bool use_ellipse) {
    const uint4 u = covers[2 * (size_t)rec];
    const uint2 rect = make_uint2(u.x, u.y);
    if (!use_ellipse) return row_cover(rect, 0.f, 0.f, 0.f, 0.f, 0.f, false);
    const uint4 v = covers[2 * (size_t)rec + 1];
    return row_cover(rect, __uint_as_float(u.z), __uint_as_float(u.w), __uint_as_float(v.x), __uint_as_float(v.y),
                     __uint_as_float(v.z), true);
}

// The cover held by lane `src` (all lanes take part).
__device__ __forceinline__ RowCover shfl_cover(const RowCover &r, int src) {
    constexpr unsigned kAll = 0xffffffffu;
    RowCover o;
    o.xc = __shfl_sync(kAll, r.xc, src);
    o.yc = __shfl_sync(kAll, r.yc, src);
    o.k = __shfl_sync(kAll, r.k, src);
    o.p = __shfl_sync(kAll, r.p, src);
    o.q = __shfl_sync(kAll, r.q, src);
    o.yr = __shfl_sync(kAll, r.yr, src);
    o.ym = __shfl_sync(kAll, r.ym, src);
    o.mx = __shfl_sync(kAll, r.mx, src);
    o.my = __shfl_sync(kAll, r.my, src);
    const uint32_t x = __shfl_sync(kAll, r.tx0 | (r.tx1 << 16), src);
    const uint32_t y = __shfl_sync(kAll, r.ty0 | (r.ty1 << 16), src);
    o.tx0 = x & 0xffffu; o.tx1 = x >> 16;
    o.ty0 = y & 0xffffu; o.ty1 = y >> 16;
    return o;
}

// Warp-wide exclusive prefix of v (all lanes take part); *total gets the sum.
__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, int lane, uint32_t *total) {
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    *total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

// The lane whose range [excl, excl + v) holds j < total: the largest lane l
// with excl[l] <= j (lanes with v = 0 share their offset with the next lane
// that has some, so the largest such lane has v > 0).
__device__ __forceinline__ int warp_owner(uint32_t excl, uint32_t j) {
    int L = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, excl, L + step);
        if (v <= j) L += step;
    }
    return L;
}

// The (cover, row) pairs of the warp's covers, 32 at a time, in order: lane
// by lane, each cover's rows [lo, hi] from top to bottom. Each lane computes
// one row's span, so a cover with many rows does not hold up the other
// lanes. g(valid, owner, row, s0, w) is called by all lanes together: owner
// is the lane whose cover the row belongs to, [s0, s0 + w) the row's span.
template <class G>
__device__ __forceinline__ void warp_cover_rows(const RowCover &cov, uint32_t lo, uint32_t hi, int lane, int tile_w,
                                                int tile_h, G &&g) {
    const uint32_t rows = lo <= hi ? hi - lo + 1u : 0u;
    uint32_t rtot;
    const uint32_t rexcl = warp_excl_scan(rows, lane, &rtot);
    for (uint32_t rb = 0; rb < rtot; rb += 32) {
        const uint32_t k = rb + (uint32_t)lane;
        const int L = warp_owner(rexcl, k);
        const RowCover oc = shfl_cover(cov, L);
        const uint32_t row = __shfl_sync(0xffffffffu, lo, L) + (k - __shfl_sync(0xffffffffu, rexcl, L));
        uint32_t s0 = 0, s1 = 0, w = 0;
        if (k < rtot) w = row_span(oc, row, tile_w, tile_h, s0, s1);
        g(k < rtot, (uint32_t)L, row, s0, w);
    }
}

// The instances of the warp's covers, 32 at a time, in the order of
// warp_cover_rows and, within a row, left to right: the (cover, row) pairs
// are dealt out first, then each group's instances, so every span is
// computed once. f(valid, n, row, tx, owner) is called by all lanes
// together: n = instances before this one, (tx, row) its tile, owner the
// lane whose cover it belongs to. Returns the number of instances.
template <class F>
__device__ __forceinline__ uint32_t warp_cover_instances(const RowCover &cov, uint32_t lo, uint32_t hi, int lane,
                                                         int tile_w, int tile_h, F &&f) {
    uint32_t run = 0;
    warp_cover_rows(cov, lo, hi, lane, tile_w, tile_h,
                    [&](bool, uint32_t owner, uint32_t row, uint32_t s0, uint32_t w) {
                        uint32_t wtot;
                        const uint32_t wexcl = warp_excl_scan(w, lane, &wtot);
                        for (uint32_t ib = 0; ib < wtot; ib += 32) {
                            const uint32_t j = ib + (uint32_t)lane;
                            const int M = warp_owner(wexcl, j);
                            const uint32_t e = __shfl_sync(0xffffffffu, wexcl, M);
                            const uint32_t ms0 = __shfl_sync(0xffffffffu, s0, M);
                            const uint32_t mrow = __shfl_sync(0xffffffffu, row, M);
                            const uint32_t mown = __shfl_sync(0xffffffffu, owner, M);
                            f(j < wtot, run + j, mrow, ms0 + (j - e), mown);
                        }
                        run += wtot;
                    });
    return run;
}

} // namespace htgs
