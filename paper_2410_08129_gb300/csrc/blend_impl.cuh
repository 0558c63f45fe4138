// blend_impl.cuh -- per-pixel ray-splat evaluation and hybrid-transparency
// blending (arXiv 2410.08129, Sec. 3.2 Eq. (13), Sec. 3.3 Eq. (14)-(16)) and
// its adjoint.
//
// One CTA per tile of TW x TH pixels; each thread owns PPT vertically
// adjacent pixels. The tile's instance list (gid ascending, no depth order)
// is staged through shared memory in batches of 96-byte records. For every
// (record, pixel) pair the quadratic Q of the record decides rho^2 <= rho_c;
// kept fragments update the per-pixel order-independent sums over all
// fragments (sum alpha, sum alpha c, prod (1 - alpha), count) and, when
// alpha >= tau_K, a depth-sorted K-core of 64-bit (depth, gid) keys held in
// registers. The tail is "all fragments minus the core": its sums are
// recovered in the epilogue, so an evicted core entry needs no colour.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

constexpr int kBatch = 64;

// Alpha and depth of one record at a pixel offset, evaluated identically in
// the main loop, the epilogue and the adjoint.
struct FragEval {
    float D, rD, t, araw, alpha;
};

__device__ __forceinline__ bool frag_alpha(const float4 &c0, const float4 &c1, const float4 &c2,
                                           const float4 &c3, float dx, float dy, float tau_alpha,
                                           float alpha_max, float Qv, FragEval &f) {
    (void)c0;
    (void)c1;
    f.D = quad_eval(c2.x, c2.y, c2.z, c2.w, c3.x, c3.y, dx, dy);
    if (!(f.D > 0.f)) return false; // vanishing denominator: the ray misses
    f.rD = rcp_approx(f.D);
    f.t = __fmul_rn(Qv, f.rD);
    f.araw = __fmul_rn(tau_alpha, ex2_approx(f.t));
    f.alpha = fminf(f.araw, alpha_max);
    return true;
}

__device__ __forceinline__ float frag_depth(const float4 &c3, const float4 &c4, float dx, float dy,
                                            float rD) {
    return __fmul_rn(quad_eval(c3.z, c3.w, c4.x, c4.y, c4.z, c4.w, dx, dy), rD);
}

template <int KMAX>
__device__ __forceinline__ void core_insert(unsigned long long (&core)[KMAX], unsigned long long key) {
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
        const unsigned long long c = core[i];
        const bool sw = key < c;
        core[i] = sw ? key : c;
        key = sw ? c : key;
    }
}

// ---------------------------------------------------------------------------
// Forward (K6).
// ---------------------------------------------------------------------------
template <int KMAX, int TW, int TH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) blend_fwd_kernel(BlendFwdArgs a) {
    constexpr int NT = TW * TH / PPT;
    __shared__ float4 s_rec[kBatch][kRecF4];
    __shared__ uint32_t s_gid[kBatch];
    if (a.status[kStError] != 0) return;

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles.tiles_x, ty = tile / a.tiles.tiles_x;
    const int tid = threadIdx.x;
    const int px_i = tx * TW + tid % TW;
    const int py_i0 = ty * TH + (tid / TW) * PPT;
    const float px = (float)px_i + 0.5f;
    float py[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) py[p] = (float)(py_i0 + p) + 0.5f;

    const int K = a.prm.K;
    const float tau_alpha = a.prm.tau_alpha, tau_K = a.prm.tau_K, alpha_max = a.prm.alpha_max;
    unsigned long long core[PPT][KMAX];
    float sA[PPT], sR[PPT], sG[PPT], sB[PPT], sP[PPT];
    int nall[PPT];
    uint32_t n_adm = 0, n_ins = 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) core[p][k] = (k < KMAX - K) ? 0ull : ~0ull;
        sA[p] = sR[p] = sG[p] = sB[p] = 0.f;
        sP[p] = 1.f;
        nall[p] = 0;
    }

    const uint2 range = a.ranges[tile];
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        const int nb = (int)min((uint32_t)kBatch, range.y - b0);
        __syncthreads();
        for (int k = tid; k < nb; k += NT) s_gid[k] = a.vals[b0 + k];
        __syncthreads();
        for (int k = tid; k < nb * kRecF4; k += NT) {
            const int j = k / kRecF4, f = k - j * kRecF4;
            s_rec[j][f] = a.rec[(size_t)s_gid[j] * kRecF4 + f];
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const float4 c0 = s_rec[j][0], c1 = s_rec[j][1];
            const float dx = __fsub_rn(px, c0.x);
            float Q[PPT];
            bool any = false;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float dy = __fsub_rn(py[p], c0.y);
                Q[p] = quad_eval(c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, dx, dy);
                any |= Q[p] >= 0.f;
            }
            if (!any) continue;
            const float4 c2 = s_rec[j][2], c3 = s_rec[j][3], c4 = s_rec[j][4], c5 = s_rec[j][5];
            const uint32_t gid = s_gid[j];
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                if (!(Q[p] >= 0.f)) continue;
                const float dy = __fsub_rn(py[p], c0.y);
                FragEval f;
                if (!frag_alpha(c0, c1, c2, c3, dx, dy, tau_alpha, alpha_max, Q[p], f)) continue;
                const float al = f.alpha;
                sA[p] += al;
                sR[p] = __fmaf_rn(al, c5.x, sR[p]);
                sG[p] = __fmaf_rn(al, c5.y, sG[p]);
                sB[p] = __fmaf_rn(al, c5.z, sB[p]);
                sP[p] = __fmaf_rn(-sP[p], al, sP[p]);
                nall[p] += 1;
                if (al >= tau_K) {
                    const float z = frag_depth(c3, c4, dx, dy, f.rD);
                    const unsigned long long key = make_key(z, gid);
                    ++n_adm;
                    if (key < core[p][KMAX - 1]) {
                        core_insert<KMAX>(core[p], key);
                        ++n_ins;
                    }
                }
            }
        }
    }

    // Work counters: one atomic per warp.
    {
        unsigned long long kept = 0;
#pragma unroll
        for (int p = 0; p < PPT; ++p)
            if (px_i < a.width && py_i0 + p < a.height) kept += (unsigned)nall[p];
        unsigned long long adm = n_adm, ins = n_ins;
        for (int o = 16; o > 0; o >>= 1) {
            kept += __shfl_xor_sync(0xffffffffu, kept, o);
            adm += __shfl_xor_sync(0xffffffffu, adm, o);
            ins += __shfl_xor_sync(0xffffffffu, ins, o);
        }
        if ((tid & 31) == 0 && a.stats) {
            atomicAdd(a.stats + kStatKept, kept);
            atomicAdd(a.stats + kStatAdmitted, adm);
            atomicAdd(a.stats + kStatInserted, ins);
        }
    }

    // Epilogue: composite the core front to back (Eq. (15)), recover the
    // tail sums and composite the tail behind it.
    const size_t npix = (size_t)a.width * a.height;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int x = px_i, y = py_i0 + p;
        if (x >= a.width || y >= a.height) continue;
        const size_t pix = (size_t)y * a.width + x;
        float C[3] = {0.f, 0.f, 0.f};
        float T = 1.f, Ac = 0.f, Sc[3] = {0.f, 0.f, 0.f};
        int n_core = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const unsigned long long key = core[p][k];
            if (k < KMAX - K || key == ~0ull) continue;
            const uint32_t gid = (uint32_t)(key & 0xffffffffull);
            const float4 *r = a.rec + (size_t)gid * kRecF4;
            const float4 c0 = r[0], c1 = r[1], c2 = r[2], c3 = r[3], c5 = r[5];
            const float ex = __fsub_rn(px, c0.x), ey = __fsub_rn(py[p], c0.y);
            const float Qv = quad_eval(c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, ex, ey);
            FragEval f;
            frag_alpha(c0, c1, c2, c3, ex, ey, tau_alpha, alpha_max, Qv, f);
            const float al = f.alpha;
            const float w = al * T;
            C[0] += w * c5.x; C[1] += w * c5.y; C[2] += w * c5.z;
            Ac += al;
            Sc[0] += al * c5.x; Sc[1] += al * c5.y; Sc[2] += al * c5.z;
            T = __fmaf_rn(-T, al, T);
            if (a.saved) a.saved[(size_t)(7 + n_core) * npix + pix] = __uint_as_float(gid);
            ++n_core;
        }
        const int n_tail = nall[p] - n_core;
        float At = 0.f, ct[3] = {0.f, 0.f, 0.f}, Pc = T;
        if (n_tail > 0) {
            At = fmaxf(sA[p] - Ac, 0.f);
            const float inv = At > 0.f ? 1.f / At : 0.f;
            ct[0] = fmaxf((sR[p] - Sc[0]) * inv, 0.f);
            ct[1] = fmaxf((sG[p] - Sc[1]) * inv, 0.f);
            ct[2] = fmaxf((sB[p] - Sc[2]) * inv, 0.f);
            Pc = fminf(sP[p], T);
        }
        const float wt = T - Pc;
        float *img = a.image + pix * 3;
        img[0] = C[0] + wt * ct[0] + Pc * a.prm.bg[0];
        img[1] = C[1] + wt * ct[1] + Pc * a.prm.bg[1];
        img[2] = C[2] + wt * ct[2] + Pc * a.prm.bg[2];
        if (a.saved) {
            a.saved[0 * npix + pix] = __int_as_float(n_core);
            a.saved[1 * npix + pix] = T;
            a.saved[2 * npix + pix] = Pc;
            a.saved[3 * npix + pix] = At;
            a.saved[4 * npix + pix] = ct[0];
            a.saved[5 * npix + pix] = ct[1];
            a.saved[6 * npix + pix] = ct[2];
            for (int k = n_core; k < K; ++k) a.saved[(size_t)(7 + k) * npix + pix] = __uint_as_float(0xffffffffu);
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint (K7). The derivative of the colour with respect to every tail
// fragment uses only per-pixel constants (Sec. 3.3): with u = g (T_c - P)/A,
// k0 = -u.c_tail and k1 = P g.(c_tail - bg), dL/dalpha_j = u.c_j + k0 +
// k1/(1 - alpha_j) and dL/dc_j = u alpha_j. Core fragment r (depth order)
// has dL/dalpha_r = T_r g.(c_r - G_r) and dL/dc_r = g alpha_r T_r, with G_r
// the colour seen behind r.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_transpose_reduce16(float (&v)[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    // Even lane l now holds the warp sum of value index l >> 1.
}

template <int KMAX, int TW, int TH, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) blend_bwd_kernel(BlendBwdArgs a) {
    constexpr int NT = TW * TH / PPT;
    __shared__ float4 s_rec[kBatch][kRecF4];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ float s_acc[kBatch][16];
    if (a.status[kStError] != 0) return;

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles.tiles_x, ty = tile / a.tiles.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int px_i = tx * TW + tid % TW;
    const int py_i0 = ty * TH + (tid / TW) * PPT;
    const float px = (float)px_i + 0.5f;
    float py[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) py[p] = (float)(py_i0 + p) + 0.5f;

    const int K = a.prm.K;
    const float tau_alpha = a.prm.tau_alpha, tau_K = a.prm.tau_K, alpha_max = a.prm.alpha_max;
    const size_t npix = (size_t)a.width * a.height;
    constexpr float kTwoLn2 = 1.3862943611198906f;

    // Per-pixel constants.
    float g[PPT][3], u[PPT][3], k0[PPT], k1[PPT];
    uint32_t cgid[PPT][KMAX];
    float cw[PPT][KMAX], cv[PPT][KMAX];
    unsigned long long last_key[PPT];
    bool core_possible[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int x = px_i, y = py_i0 + p;
        const bool inside = x < a.width && y < a.height;
        const size_t pix = inside ? (size_t)y * a.width + x : 0;
        int n_core = 0;
        float Tc = 1.f, Pc = 1.f, At = 0.f, ct[3] = {0.f, 0.f, 0.f};
        if (inside) {
            g[p][0] = a.dl_dimg[pix * 3 + 0];
            g[p][1] = a.dl_dimg[pix * 3 + 1];
            g[p][2] = a.dl_dimg[pix * 3 + 2];
            n_core = min(max(__float_as_int(a.saved[0 * npix + pix]), 0), K);
            Tc = a.saved[1 * npix + pix];
            Pc = a.saved[2 * npix + pix];
            At = a.saved[3 * npix + pix];
            ct[0] = a.saved[4 * npix + pix];
            ct[1] = a.saved[5 * npix + pix];
            ct[2] = a.saved[6 * npix + pix];
        } else {
            g[p][0] = g[p][1] = g[p][2] = 0.f;
        }
        const float bg0 = a.prm.bg[0], bg1 = a.prm.bg[1], bg2 = a.prm.bg[2];
        if (At > 0.f) {
            const float s = (Tc - Pc) / At;
            u[p][0] = g[p][0] * s; u[p][1] = g[p][1] * s; u[p][2] = g[p][2] * s;
            k0[p] = -(u[p][0] * ct[0] + u[p][1] * ct[1] + u[p][2] * ct[2]);
            k1[p] = Pc * (g[p][0] * (ct[0] - bg0) + g[p][1] * (ct[1] - bg1) + g[p][2] * (ct[2] - bg2));
        } else {
            u[p][0] = u[p][1] = u[p][2] = 0.f;
            k0[p] = k1[p] = 0.f;
        }
        // Colour seen behind the core: (1 - T_tail) c_tail + T_tail bg with
        // T_tail = P / T_c.
        const float Tt = (At > 0.f && Tc > 0.f) ? fminf(Pc / Tc, 1.f) : 1.f;
        float G[3] = {(1.f - Tt) * ct[0] + Tt * bg0, (1.f - Tt) * ct[1] + Tt * bg1,
                      (1.f - Tt) * ct[2] + Tt * bg2};
        last_key[p] = ~0ull;
        // Back to front: u_r = g.(c_r - G_r), alpha_r kept in cv.
#pragma unroll
        for (int r = KMAX - 1; r >= 0; --r) {
            cgid[p][r] = 0xffffffffu;
            cw[p][r] = 0.f;
            cv[p][r] = 0.f;
            const uint32_t gid = r < n_core ? __float_as_uint(a.saved[(size_t)(7 + r) * npix + pix]) : 0xffffffffu;
            if (r < n_core && (int64_t)gid < a.n) {
                const float4 *rr = a.rec + (size_t)gid * kRecF4;
                const float4 c0 = rr[0], c1 = rr[1], c2 = rr[2], c3 = rr[3], c5 = rr[5];
                const float ex = __fsub_rn(px, c0.x), ey = __fsub_rn(py[p], c0.y);
                const float Qv = quad_eval(c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, ex, ey);
                FragEval f;
                frag_alpha(c0, c1, c2, c3, ex, ey, tau_alpha, alpha_max, Qv, f);
                const float al = f.alpha;
                cgid[p][r] = gid;
                cw[p][r] = g[p][0] * (c5.x - G[0]) + g[p][1] * (c5.y - G[1]) + g[p][2] * (c5.z - G[2]);
                cv[p][r] = al;
                G[0] = al * c5.x + (1.f - al) * G[0];
                G[1] = al * c5.y + (1.f - al) * G[1];
                G[2] = al * c5.z + (1.f - al) * G[2];
                if (r == K - 1) {
                    const float4 c4 = rr[4];
                    last_key[p] = make_key(frag_depth(c3, c4, ex, ey, f.rD), gid);
                }
            }
        }
        // Front to back: T_r; dL/dalpha_r = T_r u_r, dL/dc_r = g alpha_r T_r.
        float T = 1.f;
#pragma unroll
        for (int r = 0; r < KMAX; ++r) {
            const float al = cv[p][r];
            cw[p][r] = T * cw[p][r];
            cv[p][r] = al * T;
            T = __fmaf_rn(-T, al, T);
        }
        core_possible[p] = K > 0;
        if (n_core < K) last_key[p] = ~0ull;
    }

    for (int k = tid; k < kBatch * 16; k += NT) (&s_acc[0][0])[k] = 0.f;
    const uint2 range = a.ranges[tile];
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        const int nb = (int)min((uint32_t)kBatch, range.y - b0);
        __syncthreads();
        for (int k = tid; k < nb; k += NT) s_gid[k] = a.vals[b0 + k];
        __syncthreads();
        for (int k = tid; k < nb * kRecF4; k += NT) {
            const int j = k / kRecF4, f = k - j * kRecF4;
            s_rec[j][f] = a.rec[(size_t)s_gid[j] * kRecF4 + f];
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const float4 c0 = s_rec[j][0], c1 = s_rec[j][1];
            const float dx = __fsub_rn(px, c0.x);
            float Q[PPT];
            bool any = false;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const float dy = __fsub_rn(py[p], c0.y);
                Q[p] = quad_eval(c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, dx, dy);
                any |= Q[p] >= 0.f;
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float4 c2 = s_rec[j][2], c3 = s_rec[j][3], c4 = s_rec[j][4], c5 = s_rec[j][5];
            const uint32_t gid = s_gid[j];
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0.f;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                if (!(Q[p] >= 0.f)) continue;
                const float dy = __fsub_rn(py[p], c0.y);
                FragEval f;
                if (!frag_alpha(c0, c1, c2, c3, dx, dy, tau_alpha, alpha_max, Q[p], f)) continue;
                const float al = f.alpha;
                bool in_core = false;
                if (core_possible[p] && al >= tau_K) {
                    const unsigned long long key = make_key(frag_depth(c3, c4, dx, dy, f.rD), gid);
                    in_core = key <= last_key[p];
                }
                float dA, dc0, dc1, dc2;
                if (in_core) {
                    float w = 0.f, s = 0.f;
#pragma unroll
                    for (int r = 0; r < KMAX; ++r)
                        if (cgid[p][r] == gid) { w = cw[p][r]; s = cv[p][r]; }
                    dA = w;
                    dc0 = g[p][0] * s; dc1 = g[p][1] * s; dc2 = g[p][2] * s;
                } else {
                    const float inv = rcp_approx(1.f - al);
                    dA = u[p][0] * c5.x + u[p][1] * c5.y + u[p][2] * c5.z + k0[p] + k1[p] * inv;
                    dc0 = u[p][0] * al; dc1 = u[p][1] * al; dc2 = u[p][2] * al;
                }
                v[13] += dc0; v[14] += dc1; v[15] += dc2;
                if (f.araw < alpha_max) {
                    v[12] += dA * al;
                    const float drho2 = -0.5f * al * dA;
                    const float rho2 = c5.w - kTwoLn2 * f.t;
                    const float dN = drho2 * f.rD;
                    const float dD = -dN * rho2;
                    const float mx = dx, my = dy;
                    const float mxx = mx * mx, mxy = mx * my, myy = my * my;
                    v[0] += dN; v[1] += dN * mx; v[2] += dN * my;
                    v[3] += dN * mxx; v[4] += dN * mxy; v[5] += dN * myy;
                    v[6] += dD; v[7] += dD * mx; v[8] += dD * my;
                    v[9] += dD * mxx; v[10] += dD * mxy; v[11] += dD * myy;
                }
            }
            warp_transpose_reduce16(v, lane);
            if ((lane & 1) == 0) atomicAdd(&s_acc[j][lane >> 1], v[0]);
        }
        __syncthreads();
        // Flush the batch's accumulators: one vector reduction per 4 values.
        for (int k = tid; k < nb * 4; k += NT) {
            const int j = k >> 2, q = k & 3;
            const float4 s = reinterpret_cast<const float4 *>(&s_acc[j][0])[q];
            if (s.x != 0.f || s.y != 0.f || s.z != 0.f || s.w != 0.f)
                red_add_v4(a.acc + (size_t)s_gid[j] * 16 + q * 4, s.x, s.y, s.z, s.w);
            reinterpret_cast<float4 *>(&s_acc[j][0])[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// ---------------------------------------------------------------------------
// Dispatch over tile shape and pixels per thread for one KMAX.
// ---------------------------------------------------------------------------
template <int KMAX, int TW, int TH, int PPT>
void run_fwd(const BlendFwdArgs &a, cudaStream_t s) {
    blend_fwd_kernel<KMAX, TW, TH, PPT><<<a.tiles.n_tiles, TW * TH / PPT, 0, s>>>(a);
}
template <int KMAX, int TW, int TH, int PPT>
void run_bwd(const BlendBwdArgs &a, cudaStream_t s) {
    blend_bwd_kernel<KMAX, TW, TH, PPT><<<a.tiles.n_tiles, TW * TH / PPT, 0, s>>>(a);
}

template <int KMAX, int PPT>
bool dispatch_shape_fwd(const BlendFwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) { run_fwd<KMAX, 16, 16, PPT>(a, s); return true; }
    if (tw == 16 && th == 8) { run_fwd<KMAX, 16, 8, PPT>(a, s); return true; }
    if (tw == 8 && th == 8 && PPT <= 2) { run_fwd<KMAX, 8, 8, (PPT <= 2 ? PPT : 2)>(a, s); return true; }
    return false;
}
template <int KMAX, int PPT>
bool dispatch_shape_bwd(const BlendBwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) { run_bwd<KMAX, 16, 16, PPT>(a, s); return true; }
    if (tw == 16 && th == 8) { run_bwd<KMAX, 16, 8, PPT>(a, s); return true; }
    if (tw == 8 && th == 8 && PPT <= 2) { run_bwd<KMAX, 8, 8, (PPT <= 2 ? PPT : 2)>(a, s); return true; }
    return false;
}

} // namespace htgs
