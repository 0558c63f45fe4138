// blend_bwd.cu -- the blend adjoint (Sec. 3.3): one persistent kernel per
// tile shape, core size at run time, per-pixel state in dynamic shared memory.
//
// One CTA per tile. The per-pixel adjoint state (the shared tail partials of
// Sec. 3.3 and the core's dL/dalpha, dL/dc) is built once in shared memory;
// then every warp independently pulls whole records from a shared counter
// (prefetching the next with cp.async into a private slot) and its lanes walk
// the pixels of the record's bounding box inside the tile, so the 16 gradient
// accumulators of a record are reduced once per (record, tile) and no
// block-wide barrier is needed.
#include "blend_impl.cuh"
#include "warp_reduce.cuh"

namespace htgs {

// ---------------------------------------------------------------------------
// Adjoint (K7). The derivative of the colour with respect to every tail
// fragment uses only per-pixel constants (Sec. 3.3): with u = g (T_c - P)/A,
// k0 = -u.c_tail and k1 = P g.(c_tail - bg), dL/dalpha_j = u.c_j + k0 +
// k1/(1 - alpha_j) and dL/dc_j = u alpha_j. Core fragment r (depth order)
// has dL/dalpha_r = T_r g.(c_r - G_r) and dL/dc_r = g alpha_r T_r, with G_r
// the colour seen behind r.
// ---------------------------------------------------------------------------

constexpr int kBwdThreads = 256;

// A compile-time flag passed to the record walk (one instance per case).
template <bool V>
struct Flag {
    static constexpr bool value = V;
};

// frag_alpha without the early exit: every field is computed, and the result
// says whether the fragment is kept (for a kept one the fields equal those of
// frag_alpha bit for bit; for the others they are unused). CLAMP = false is
// for records whose alpha cannot reach alpha_max (there the clamp is the
// identity).
template <bool CLAMP = true>
__device__ __forceinline__ bool frag_alpha_all(float2 qd, float tau_alpha, float alpha_max, FragEval &f) {
    f.D = qd.y;
    f.rD = rcp_approx(f.D);
    f.t = __fmul_rn(qd.x, f.rD);
    f.araw = __fmul_rn(tau_alpha, ex2_approx(f.t));
    f.alpha = CLAMP ? fminf(f.araw, alpha_max) : f.araw;
    return qd.x >= 0.f && qd.y > 0.f;
}

// Dynamic shared memory of the adjoint for a TP-pixel tile and core size K.
__host__ __device__ inline size_t bwd_smem_bytes(int TP, int K) {
    return (size_t)TP * (2 * sizeof(float4) + sizeof(float2) + (size_t)K * 3 * sizeof(float) + sizeof(float));
}

template <int TW, int TH, bool NOTAIL, bool VIS>
__global__ void __launch_bounds__(kBwdThreads, 3) blend_bwd_kernel(const __grid_constant__ Batch bt, BlendBwdArgs a) {
    dependent_entry();
    constexpr int TP = TW * TH;
    constexpr int NW = kBwdThreads / 32;
    extern __shared__ float4 smem[];
    __shared__ float4 s_wrec[NW][2][kRecF4];  // per-warp double-buffered record
    __shared__ uint32_t s_wgid[NW][2];
    __shared__ uint32_t s_next;
    __shared__ int s_item;
    __shared__ float s_wzmax[NW];
    __shared__ int s_wopen[NW];
    const int K = a.prm.K;
    const int n_items = min((int)*a.n_items, a.max_items);
    float4 *s_pa = smem;                 // g.xyz, k0
    float4 *s_pb = s_pa + TP;            // u.xyz, k1
    // Last core entry (depth, gid) of a full core; depth +inf where the core
    // is not full (every candidate there belongs to it).
    float2 *s_pc = reinterpret_cast<float2 *>(s_pb + TP);
    uint32_t *s_cg = reinterpret_cast<uint32_t *>(s_pc + TP);        // [K][TP] core gids
    float *s_cw = reinterpret_cast<float *>(s_cg + (size_t)K * TP);  // [K][TP] dL/dalpha_r
    float *s_cv = s_cw + (size_t)K * TP;                             // [K][TP] alpha_r T_r
    float *s_wt = s_cv + (size_t)K * TP;                             // [TP] T_core (1 - T_tail) / A
    if (a.status[kStError] != 0) return;

    // Persistent CTA: take (view, tile, chunk) items from the shared queue.
    // The adjoint of a chunk needs only the saved per-pixel state, so the
    // chunks of a split tile are independent.
    for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    const int4 work = a.items[item];
    const int tile = work.x;
    if (!item_ok(work, bt.total_tiles, a.max_items)) continue;  // (the adjoint uses no slots)
    const ViewDesc &view = bt.v[view_of_tile(bt, tile)];
    const int local = tile - view.tile_off;
    const int tx = local % view.tiles_x, ty = local / view.tiles_x;
    const int width = view.cam.width, height = view.cam.height;
    const float *const saved = view.saved;
    const float *const dl_dimg = view.dl_dimg;
    const long long n_rec = bt.n_rec;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = tx * TW, y0 = ty * TH;
    const int x1 = min(x0 + TW, width) - 1, y1 = min(y0 + TH, height) - 1;
    const float tau_alpha = a.prm.tau_alpha, tau_K = a.prm.tau_K, alpha_max = a.prm.alpha_max;
    const float bg0 = a.prm.bg[0], bg1 = a.prm.bg[1], bg2 = a.prm.bg[2];
    const size_t npix = (size_t)width * height;
    const uint2 range = chunk_range(a.ranges[tile], work.y, work.z);

    // Phase A: per-pixel adjoint state. Also, over the tile's pixels: the
    // deepest last core entry of full cores and whether a core is not full
    // (there every candidate belongs to it).
    float zmax_l = -INFINITY;
    bool open_l = false;
    for (int p = tid; p < TP; p += kBwdThreads) {
        const int x = x0 + p % TW, y = y0 + p / TW;
        const bool inside = x < width && y < height;
        const size_t pix = inside ? (size_t)y * width + x : 0;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        int n_core = 0;
        float Tc = 1.f, Pc = 1.f, At = 0.f, ct0 = 0.f, ct1 = 0.f, ct2 = 0.f;
        if (inside) {
            g0 = dl_dimg[pix * 3 + 0];
            g1 = dl_dimg[pix * 3 + 1];
            g2 = dl_dimg[pix * 3 + 2];
            n_core = min(max(__float_as_int(saved[0 * npix + pix]), 0), K);
            Tc = saved[1 * npix + pix];
            Pc = saved[2 * npix + pix];
            At = saved[3 * npix + pix];
            ct0 = saved[4 * npix + pix];
            ct1 = saved[5 * npix + pix];
            ct2 = saved[6 * npix + pix];
        }
        float u0 = 0.f, u1 = 0.f, u2 = 0.f, k0 = 0.f, k1 = 0.f;
        // A tail fragment's blending weight is alpha_j T_core (1 - T_tail) / A.
        s_wt[p] = At > 0.f ? __fdividef(Tc - Pc, At) : 0.f;
        if (At > 0.f) {
            const float s = __fdividef(Tc - Pc, At);
            u0 = g0 * s; u1 = g1 * s; u2 = g2 * s;
            k0 = -(u0 * ct0 + u1 * ct1 + u2 * ct2);
            k1 = Pc * (g0 * (ct0 - bg0) + g1 * (ct1 - bg1) + g2 * (ct2 - bg2));
        }
        s_pa[p] = make_float4(g0, g1, g2, k0);
        s_pb[p] = make_float4(u0, u1, u2, k1);
        // Colour seen behind the core: (1 - T_tail) c_tail + T_tail bg, T_tail = P / T_c.
        const float Tt = (At > 0.f && Tc > 0.f) ? fminf(__fdividef(Pc, Tc), 1.f) : 1.f;
        float G0 = (1.f - Tt) * ct0 + Tt * bg0, G1 = (1.f - Tt) * ct1 + Tt * bg1, G2 = (1.f - Tt) * ct2 + Tt * bg2;
        float lastz = INFINITY;
        uint32_t lastg = 0xffffffffu;
        // Back to front: u_r = g.(c_r - G_r) into s_cw, alpha_r into s_cv.
        for (int r = n_core - 1; r >= 0; --r) {
            const uint32_t gid = __float_as_uint(saved[(size_t)(7 + r) * npix + pix]);
            float ur = 0.f, al = 0.f;
            if ((long long)gid < n_rec) {
                const float4 *rr = a.rec + (size_t)gid * kRecF4;
                const float4 c0 = rr[0], c1 = rr[1], c2 = rr[2], c4 = rr[4], c5 = rr[5];
                const float ex = __fsub_rn((float)x + 0.5f, c4.z), ey = __fsub_rn((float)y + 0.5f, c4.w);
                FragEval f;
                frag_alpha(quad_eval2(c0, c1, c2, ex, ey), tau_alpha, alpha_max, f);
                al = f.alpha;
                ur = g0 * (c5.x - G0) + g1 * (c5.y - G1) + g2 * (c5.z - G2);
                G0 = al * c5.x + (1.f - al) * G0;
                G1 = al * c5.y + (1.f - al) * G1;
                G2 = al * c5.z + (1.f - al) * G2;
                if (r == K - 1) {
                    lastz = frag_depth(rr[3], c4, ex, ey, f.rD);
                    lastg = gid;
                }
            }
            s_cg[(size_t)r * TP + p] = gid;
            s_cw[(size_t)r * TP + p] = ur;
            s_cv[(size_t)r * TP + p] = al;
        }
        // Front to back: T_r; dL/dalpha_r = T_r u_r, dL/dc_r = g alpha_r T_r.
        float T = 1.f;
        for (int r = 0; r < n_core; ++r) {
            const float al = s_cv[(size_t)r * TP + p];
            s_cw[(size_t)r * TP + p] *= T;
            s_cv[(size_t)r * TP + p] = al * T;
            T = __fmaf_rn(-T, al, T);
        }
        // A core that is not full takes every candidate (K = 0 has no core:
        // the record loop then skips the test altogether).
        const bool open = n_core < K;
        s_pc[p] = make_float2(open ? INFINITY : lastz, __uint_as_float(lastg));
        if (inside && K > 0) {
            if (open) open_l = true;
            else zmax_l = fmaxf(zmax_l, lastz);
        }
    }
    for (int o = 16; o > 0; o >>= 1) zmax_l = fmaxf(zmax_l, __shfl_xor_sync(0xffffffffu, zmax_l, o));
    open_l = __any_sync(0xffffffffu, open_l);
    if (lane == 0) {
        s_wzmax[warp] = zmax_l;
        s_wopen[warp] = open_l ? 1 : 0;
    }
    if (tid == 0) s_next = range.x;
    __syncthreads();
    // A record whose depths all exceed the deepest last core entry belongs
    // to no pixel's core in this tile (unless some core is not full).
    float tile_zmax = -INFINITY;
    int tile_open = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        tile_zmax = fmaxf(tile_zmax, s_wzmax[w]);
        tile_open |= s_wopen[w];
    }

    // Phase B: warps pull records; lanes walk the record's box in the tile.
    auto grab = [&]() -> uint32_t {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(&s_next, 1u);
        return __shfl_sync(0xffffffffu, j, 0);
    };
    auto issue = [&](uint32_t j, int slot) {
        if (lane < kRecF4) {
            const uint32_t gid = a.vals[j];
            cp_async16(&s_wrec[warp][slot][lane], a.rec + (size_t)gid * kRecF4 + lane);
            if (lane == 0) s_wgid[warp][slot] = gid;
        }
        cp_async_commit();
    };
    constexpr float kLn2 = 0.69314718055994531f;
    const float rc_clamp = 2.f * logf(alpha_max / tau_alpha) - 1e-3f;
    uint32_t j = grab();
    int slot = 0;
    if (j < range.y) issue(j, 0);
    while (j < range.y) {
        const uint32_t jn = grab();
        if (jn < range.y) {
            issue(jn, slot ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        const float4 *rec = s_wrec[warp][slot];
        const uint32_t gid = s_wgid[warp][slot];
        const float4 c6 = rec[6];
        const int ix0 = (int)fmaxf(ceilf(c6.x - 0.5f), (float)x0);
        const int ix1 = (int)fminf(floorf(c6.y - 0.5f), (float)x1);
        const int iy0 = (int)fmaxf(ceilf(c6.z - 0.5f), (float)y0);
        const int iy1 = (int)fminf(floorf(c6.w - 0.5f), (float)y1);
        if (ix0 <= ix1 && iy0 <= iy1) {
            const float4 c0 = rec[0], c1 = rec[1], c2 = rec[2], c4 = rec[4], c5 = rec[5];
            const float zlo = rec[7].x;
            const bool may_core = K > 0 && (tile_open || !(zlo > tile_zmax));
            // alpha reaches its clamp only where o >= alpha_max, i.e. rho_c >=
            // 2 ln(alpha_max / tau_alpha) (less a margin for rounding).
            const bool may_clamp = c5.w >= rc_clamp;
            float2 acc[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] = make_float2(0.f, 0.f);
            float gaa = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
            float wmax = 0.f;  // largest blending weight of the record in this tile
            bool touched = false;
            const int lx = lane & 7, ly = lane >> 3;
            // The walk over the record's box, compiled for each case of three
            // record-wide conditions: whether a fragment can belong to a core
            // of this tile (most records of a deep tile cannot), whether its
            // alpha can reach the clamp, and (for the common case of neither)
            // whether its box covers the whole tile, whose rows are then an
            // unrolled loop without column bounds.
            auto walk = [&](auto core_flag, auto clamp_flag, auto full_flag) {
                constexpr bool CORE = decltype(core_flag)::value;
                constexpr bool CLAMP = decltype(clamp_flag)::value;
                constexpr bool FULL = decltype(full_flag)::value;  // the box spans the whole tile
                // The adjoint of one kept fragment at pixel p (offset dx, dy).
                auto fragment = [&](float dx, float dy, int p, const FragEval &f) {
                    const float al = f.alpha;
                    bool in_core = false;
                    if (CORE && al >= tau_K) {
                        const float2 PC = s_pc[p];
                        if (PC.x == INFINITY) {
                            in_core = true;
                        } else if (!(zlo > PC.x)) {
                            // (depths of this splat are >= zlo, so zlo > last
                            // core depth means the fragment is not in the core)
                            const float z = frag_depth(rec[3], c4, dx, dy, f.rD);
                            in_core = z < PC.x || (z == PC.x && gid <= __float_as_uint(PC.y));
                        }
                    }
                    if (NOTAIL && !in_core) return;  // an omitted tail has no gradient
                    float dA;
                    if (in_core) {
                        const float4 PA = s_pa[p];
                        float w = 0.f, s = 0.f;
                        for (int r = 0; r < K; ++r)
                            if (s_cg[(size_t)r * TP + p] == gid) {
                                w = s_cw[(size_t)r * TP + p];
                                s = s_cv[(size_t)r * TP + p];
                                break;
                            }
                        dA = w;
                        gc0 = __fmaf_rn(PA.x, s, gc0);
                        gc1 = __fmaf_rn(PA.y, s, gc1);
                        gc2 = __fmaf_rn(PA.z, s, gc2);
                        if (VIS) wmax = fmaxf(wmax, s);
                    } else {
                        const float4 PB = s_pb[p];
                        const float k0 = s_pa[p].w;
                        const float inv = rcp_approx(1.f - al);
                        dA = PB.x * c5.x + PB.y * c5.y + PB.z * c5.z + k0 + PB.w * inv;
                        gc0 = __fmaf_rn(PB.x, al, gc0);
                        gc1 = __fmaf_rn(PB.y, al, gc1);
                        gc2 = __fmaf_rn(PB.z, al, gc2);
                        if (VIS) wmax = fmaxf(wmax, al * s_wt[p]);
                    }
                    touched = true;
                    // With g = alpha dL/dalpha: dL/drho^2 = -g/2, and as
                    // rho^2 = N / D = rho_c - 2 ln2 t, dL/dN = -e/2 and
                    // dL/dD = e rho^2 / 2 = (rho_c e - 2 ln2 e t) / 2 for
                    // e = g / D. The pixel adds the moments of (e, e t); the
                    // (record, tile) sums become dL/dN and dL/dD once, after
                    // the warp reduction. A clamped alpha (araw >= alpha_max)
                    // passes no gradient to the geometry: g = 0 adds nothing.
                    const float g = (!CLAMP || f.araw < alpha_max) ? dA * al : 0.f;
                    gaa += g;
                    const float e = g * f.rD;
                    const float2 et = make_float2(e, e * f.t);
                    const float2 X = make_float2(dx, dx), Y = make_float2(dy, dy);
                    const float2 ex = fmul2(et, X), ey = fmul2(et, Y);
                    acc[0] = fadd2(acc[0], et);
                    acc[1] = fadd2(acc[1], ex);
                    acc[2] = fadd2(acc[2], ey);
                    acc[3] = ffma2(ex, X, acc[3]);
                    acc[4] = ffma2(ex, Y, acc[4]);
                    acc[5] = ffma2(ey, Y, acc[5]);
                };
                // Pixel centres are integers plus 1/2, exact in FP32, so
                // stepping them by whole pixels gives (float)x + 0.5 bit for
                // bit. Two pixels of a row are evaluated together (the cutoff
                // test and alpha for both before either's adjoint), which
                // gives the scheduler two independent chains; each lane still
                // visits its pixels in row order.
                const float pxl = (float)(ix0 + lx) + 0.5f;
                auto row = [&](int y) {
                    const float dy = __fsub_rn((float)y + 0.5f, c4.w);
                    const int prow = (y - y0) * TW - x0 + ix0 + lx;
#pragma unroll
                    for (int q = 0; q < TW / 8; q += 2) {
                        const bool in0 = FULL || ix0 + lx + 8 * q <= ix1;
                        const bool in1 = q + 1 < TW / 8 && (FULL || ix0 + lx + 8 * (q + 1) <= ix1);
                        const float dx0 = __fsub_rn(pxl + 8.f * q, c4.z);
                        const float dx1 = __fsub_rn(pxl + 8.f * (q + 1), c4.z);
                        FragEval f0, f1;
                        const bool k0 =
                            frag_alpha_all<CLAMP>(quad_eval2(c0, c1, c2, dx0, dy), tau_alpha, alpha_max, f0) && in0;
                        const bool k1 =
                            frag_alpha_all<CLAMP>(quad_eval2(c0, c1, c2, dx1, dy), tau_alpha, alpha_max, f1) && in1;
                        if (k0) fragment(dx0, dy, prow + 8 * q, f0);
                        if (k1) fragment(dx1, dy, prow + 8 * (q + 1), f1);
                        if (!in1) break;
                    }
                };
                if constexpr (FULL) {
                    // The whole tile: TH / 4 rows per lane.
#pragma unroll
                    for (int r = 0; r < TH / 4; ++r) row(y0 + ly + 4 * r);
                } else {
                    for (int y = iy0 + ly; y <= iy1; y += 4) row(y);
                }
            };
            const bool full = ix0 == x0 && ix1 == x0 + TW - 1 && iy0 == y0 && iy1 == y0 + TH - 1;
            if (may_core) {
                if (may_clamp) walk(Flag<true>{}, Flag<true>{}, Flag<false>{});
                else walk(Flag<true>{}, Flag<false>{}, Flag<false>{});
            } else if (may_clamp) {
                walk(Flag<false>{}, Flag<true>{}, Flag<false>{});
            } else if (full) {
                walk(Flag<false>{}, Flag<false>{}, Flag<true>{});
            } else {
                walk(Flag<false>{}, Flag<false>{}, Flag<false>{});
            }
            if (VIS) {
                for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
                // Non-negative floats order like their bit patterns.
                if (lane == 0 && wmax > 0.f) atomicMax(reinterpret_cast<int *>(a.vis) + gid, __float_as_int(wmax));
            }
            if (__any_sync(0xffffffffu, touched)) {
                float v[16] = {acc[0].x, acc[0].y, acc[1].x, acc[1].y, acc[2].x, acc[2].y, acc[3].x, acc[3].y,
                               acc[4].x, acc[4].y, acc[5].x, acc[5].y, gaa, gc0, gc1, gc2};
                warp_reduce16_to4(v, lane);
                if ((lane & 7) == 0) {
                    if (lane < 24) {  // two (sum e m, sum e t m) pairs -> (dL/dN_m, dL/dD_m)
                        const float rc = c5.w;
                        const float n0 = -0.5f * v[0], d0 = 0.5f * rc * v[0] - kLn2 * v[1];
                        const float n1 = -0.5f * v[2], d1 = 0.5f * rc * v[2] - kLn2 * v[3];
                        v[0] = n0; v[1] = d0; v[2] = n1; v[3] = d1;
                    }
                    red_add_v4(a.acc + (size_t)gid * 16 + (lane >> 3) * 4, v[0], v[1], v[2], v[3]);
                }
            }
        }
        __syncwarp();
        slot ^= 1;
        j = jn;
    }
    __syncthreads();  // the next item rebuilds the per-pixel state
    } // next item
}

namespace {

template <int TW, int TH, bool NOTAIL, bool VIS>
bool run_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    const size_t smem = bwd_smem_bytes(TW * TH, a.prm.K);
    const void *fn = (const void *)blend_bwd_kernel<TW, TH, NOTAIL, VIS>;
    if (!allow_dynamic_smem(fn, bwd_smem_bytes(TW * TH, HTGS_MAX_K))) return false;
    const int grid = persistent_grid(fn, kBwdThreads, smem, a.max_items);
    launch_k(blend_bwd_kernel<TW, TH, NOTAIL, VIS>, grid, kBwdThreads, smem, s, b, a);
    return true;
}

// The tail-less variant and the visibility statistic are compiled into
// separate instances so that the default adjoint keeps its code.
template <int TW, int TH>
bool run_bwd_mode(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    if (a.vis) return a.prm.no_tail ? run_bwd<TW, TH, true, true>(b, a, s) : run_bwd<TW, TH, false, true>(b, a, s);
    return a.prm.no_tail ? run_bwd<TW, TH, true, false>(b, a, s) : run_bwd<TW, TH, false, false>(b, a, s);
}

} // namespace

bool launch_blend_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    if (a.prm.K < 0 || a.prm.K > HTGS_MAX_K) return false;
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_bwd_mode<16, 16>(b, a, s);
    if (tw == 32 && th == 16) return run_bwd_mode<32, 16>(b, a, s);
    if (tw == 16 && th == 8) return run_bwd_mode<16, 8>(b, a, s);
    if (tw == 8 && th == 8) return run_bwd_mode<8, 8>(b, a, s);
    return false;
}

} // namespace htgs
