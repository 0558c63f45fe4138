// blend_impl.cuh -- per-pixel ray-splat evaluation and hybrid-transparency
// blending (arXiv 2410.08129, Sec. 3.2 Eq. (13), Sec. 3.3 Eq. (14)-(16)) and
// its adjoint.
//
// Forward: one CTA per tile of TW x TH pixels; each warp owns an 8 x (4 PPT)
// pixel footprint and each lane PPT vertically adjacent pixels. The tile's
// instance list (gid ascending, no depth order) is staged through shared
// memory in batches of records, double-buffered with cp.async so that the
// gather of the next batch overlaps the evaluation of the current one. A
// warp first culls a batch against its footprint (one bounding-box test per
// lane and record, one ballot per 32 records) and evaluates only the records
// that touch it. For each pixel one packed FP32x2 evaluation gives the pair
// (Q, D) of a record: Q >= 0 decides rho^2 <= rho_c and D gives alpha. Kept
// fragments update the per-pixel order-independent sums over all fragments
// (sum alpha, sum alpha c, prod (1 - alpha), count) and, when
// alpha >= tau_K, a K-core of (depth, gid) pairs held in registers in
// ascending order. The tail is "all fragments minus the core": its sums are
// recovered in the epilogue, so an evicted core entry needs no colour.
//
// Adjoint: one CTA per tile. The per-pixel adjoint state (the shared tail
// partials of Sec. 3.3 and the core's dL/dalpha, dL/dc) is built once in
// shared memory; then every warp independently pulls whole records from a
// shared counter (prefetching the next with cp.async into a private slot)
// and its lanes walk the pixels of the record's bounding box inside the
// tile, so the 16 gradient accumulators of a record are reduced once per
// (record, tile) and no block-wide barrier is needed.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

// Dynamic shared memory of the forward: three staging buffers of B records
// and their ids (B = htgs_launch.smem_batch: 32, 64 or 128).
__host__ __device__ inline size_t fwd_smem_bytes(int B) {
    return (size_t)3 * B * (kRecF4 * sizeof(float4) + sizeof(uint32_t));
}

constexpr int kBwdThreads = 256;

// Alpha of one record at a pixel from its (Q, D) pair, evaluated identically
// in the main loop, the epilogue and the adjoint.
struct FragEval {
    float D, rD, t, araw, alpha;
};

__device__ __forceinline__ bool frag_alpha(float2 qd, float tau_alpha, float alpha_max, FragEval &f) {
    if (!(qd.x >= 0.f) || !(qd.y > 0.f)) return false; // outside the cutoff, or the ray misses
    f.D = qd.y;
    f.rD = rcp_approx(f.D);
    f.t = __fmul_rn(qd.x, f.rD);
    f.araw = __fmul_rn(tau_alpha, ex2_approx(f.t));
    f.alpha = fminf(f.araw, alpha_max);
    return true;
}

// View depth of the point of maximum contribution (Sec. 3.3, Eq. (14)).
__device__ __forceinline__ float frag_depth(const float4 &c3, const float4 &c4, float dx, float dy,
                                            float rD) {
    return __fmul_rn(quad_eval(c3.x, c3.y, c3.z, c3.w, c4.x, c4.y, dx, dy), rD);
}

// Insertion into a list sorted by (depth, gid). The new entry's gid exceeds
// that of every listed entry of equal depth (records are visited in
// ascending gid, and partial lists are merged in chunk order), so it goes
// before the first strictly deeper entry, the entries from there on shift
// down by one (equal depths included) and the last one drops out. The
// predicates "new entry is nearer than slot i" are monotone along the list
// and independent of each other, so all slots update in parallel.
template <int KMAX>
__device__ __forceinline__ void core_insert(float (&cz)[KMAX], uint32_t (&cg)[KMAX], float z, uint32_t g) {
    bool nearer[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) nearer[i] = z < cz[i];
#pragma unroll
    for (int i = KMAX - 1; i > 0; --i) {
        cz[i] = nearer[i] ? (nearer[i - 1] ? cz[i - 1] : z) : cz[i];
        cg[i] = nearer[i] ? (nearer[i - 1] ? cg[i - 1] : g) : cg[i];
    }
    cz[0] = nearer[0] ? z : cz[0];
    cg[0] = nearer[0] ? g : cg[0];
}

// ---------------------------------------------------------------------------
// Forward (K6).
// ---------------------------------------------------------------------------
template <int KMAX, int TW, int TH, int PPT, bool NOTAIL>
__global__ void __launch_bounds__(TW *TH / PPT, (PPT == 1 && KMAX <= 8) ? 1024 / (TW * TH / PPT) : 1)
blend_fwd_kernel(const __grid_constant__ Batch bt, BlendFwdArgs a) {
    constexpr int NT = TW * TH / PPT;
    constexpr int WY = 4 * PPT;  // warp footprint: 8 x WY pixels
    constexpr int WPR = TW / 8;  // footprints per tile row
    static_assert(TW % 8 == 0 && TH % WY == 0 && NT % 32 == 0, "unsupported blend shape");
    constexpr int TP = TW * TH;
    extern __shared__ float4 s_dyn[];
    const int B = a.tiles.batch;
    float4 *const s_rec = s_dyn;                                                   // [3][B][kRecF4]
    uint32_t *const s_gid = reinterpret_cast<uint32_t *>(s_dyn + 3 * B * kRecF4);  // [3][B]
    __shared__ int s_item;
    __shared__ int s_last;
    if (a.status[kStError] != 0) return;
    const int n_items = min((int)*a.n_items, a.max_items);

    // Persistent CTA: take (view, tile, chunk) items from the shared queue.
    for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    const int4 work = a.items[item];
    const int tile = work.x, chunk_k = work.y, chunk_m = work.z, slot0 = work.w;
    if (!item_ok(work, bt.total_tiles, a.slots)) continue;
    const ViewDesc &view = bt.v[view_of_tile(bt, tile)];
    const int local = tile - view.tile_off;
    const int tx = local % view.tiles_x, ty = local / view.tiles_x;
    const int width = view.cam.width, height = view.cam.height;
    float *const image = view.image;
    float *const saved = view.saved;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wx0 = tx * TW + (warp % WPR) * 8;
    const int wy0 = ty * TH + (warp / WPR) * WY;
    const int px_i = wx0 + (lane & 7);
    const int py_i0 = wy0 + (lane >> 3) * PPT;
    const float px = (float)px_i + 0.5f;
    float py[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) py[p] = (float)(py_i0 + p) + 0.5f;
    // The warp's footprint in pixel-centre coordinates.
    const float fx0 = (float)wx0 + 0.5f, fx1 = (float)wx0 + 7.5f;
    const float fy0 = (float)wy0 + 0.5f, fy1 = (float)(wy0 + WY) - 0.5f;

    const int K = a.prm.K;
    const float tau_alpha = a.prm.tau_alpha, tau_K = a.prm.tau_K, alpha_max = a.prm.alpha_max;
    constexpr bool no_tail = NOTAIL;  // inference without the tail (compiled separately)
    float cz[PPT][KMAX];
    uint32_t cg[PPT][KMAX];
    float sA[PPT], sR[PPT], sG[PPT], sB[PPT], sP[PPT];
    int nall[PPT];
    uint32_t n_adm = 0, n_ins = 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            // Slots below KMAX - K hold -inf and are never displaced.
            cz[p][k] = (k < KMAX - K) ? -INFINITY : INFINITY;
            cg[p][k] = 0xffffffffu;
        }
        sA[p] = sR[p] = sG[p] = sB[p] = 0.f;
        sP[p] = 1.f;
        nall[p] = 0;
    }

    const uint2 range = chunk_range(a.ranges[tile], chunk_k, chunk_m);
    const int nbatches = (int)((range.y - range.x + B - 1) / B);
    auto batch_size = [&](int b) { return (int)min((uint32_t)B, range.y - range.x - (uint32_t)b * B); };
    // Stage batch b into buffer b % 3: each thread fetches the ids of the
    // records it copies (8 threads per record read the same id), so no
    // barrier separates the id loads from the copies.
    auto issue = [&](int b) {
        const int nb = batch_size(b);
        const uint32_t base = range.x + (uint32_t)b * B;
        const int buf = b % 3;
        float4 *dst = s_rec + (size_t)buf * B * kRecF4;
        uint32_t *ids = s_gid + buf * B;
        for (int k = tid; k < nb * kRecF4; k += NT) {
            const int j = k / kRecF4, f = k - j * kRecF4;
            const uint32_t gid = a.vals[base + j];
            if (f == 0) ids[j] = gid;
            cp_async16(dst + k, a.rec + (size_t)gid * kRecF4 + f);
        }
        cp_async_commit();
    };
    // Two batches in flight, one barrier per batch: after it, batch b is
    // visible to every thread and every thread has finished batch b - 1,
    // whose buffer the copies of batch b + 2 then overwrite.
    if (nbatches > 0) issue(0);
    if (nbatches > 1) issue(1);
    for (int b = 0; b < nbatches; ++b) {
        if (b + 1 < nbatches) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        if (b + 2 < nbatches) issue(b + 2);
        const int nb = batch_size(b);
        const float4(*rec)[kRecF4] = reinterpret_cast<const float4(*)[kRecF4]>(s_rec + (size_t)(b % 3) * B * kRecF4);
        const uint32_t *gids = s_gid + (b % 3) * B;
        for (int c = 0; c < nb; c += 32) {
            bool hit = false;
            if (c + lane < nb) {
                const float4 bb = rec[c + lane][6];
                hit = bb.x <= fx1 && bb.y >= fx0 && bb.z <= fy1 && bb.w >= fy0;
            }
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            while (mask) {
                const int j = c + __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 c0 = rec[j][0], c1 = rec[j][1], c2 = rec[j][2], c4 = rec[j][4];
                const float dx = __fsub_rn(px, c4.z);
                float2 qd[PPT];
                bool any = false;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    qd[p] = quad_eval2(c0, c1, c2, dx, __fsub_rn(py[p], c4.w));
                    any |= qd[p].x >= 0.f;
                }
                if (!any) continue;
                const float4 c3 = rec[j][3], c5 = rec[j][5];
                const float zlo = rec[j][7].x;
                const uint32_t gid = gids[j];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    FragEval f;
                    if (!frag_alpha(qd[p], tau_alpha, alpha_max, f)) continue;
                    const float al = f.alpha;
                    if (!no_tail) {  // without the tail the sums stay empty
                        sA[p] += al;
                        sR[p] = __fmaf_rn(al, c5.x, sR[p]);
                        sG[p] = __fmaf_rn(al, c5.y, sG[p]);
                        sB[p] = __fmaf_rn(al, c5.z, sB[p]);
                        sP[p] = __fmaf_rn(-sP[p], al, sP[p]);
                    }
                    nall[p] += 1;
                    if (al >= tau_K) {
                        ++n_adm;
                        // Every depth of this splat is >= zlo: skip the depth
                        // when it cannot beat the current K-th entry.
                        if (zlo < cz[p][KMAX - 1]) {
                            const float z = frag_depth(c3, c4, dx, __fsub_rn(py[p], c4.w), f.rD);
                            if (z < cz[p][KMAX - 1]) {
                                core_insert<KMAX>(cz[p], cg[p], z, gid);
                                ++n_ins;
                            }
                        }
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
            if (px_i < width && py_i0 + p < height) kept += (unsigned)nall[p];
        unsigned long long adm = n_adm, ins = n_ins;
        for (int o = 16; o > 0; o >>= 1) {
            kept += __shfl_xor_sync(0xffffffffu, kept, o);
            adm += __shfl_xor_sync(0xffffffffu, adm, o);
            ins += __shfl_xor_sync(0xffffffffu, ins, o);
        }
        if (lane == 0 && a.stats) {
            atomicAdd(a.stats + kStatKept, kept);
            atomicAdd(a.stats + kStatAdmitted, adm);
            atomicAdd(a.stats + kStatInserted, ins);
        }
    }

    // A chunk of a split tile leaves its partial state (the sums over its
    // fragments and its K nearest candidates); the tile's last chunk to
    // finish merges all of them in chunk order. Chunks are ascending gid
    // ranges, so inserting their core lists in chunk order keeps the
    // (depth, gid) order of a single pass, and the merged core is the K
    // nearest candidates of the whole list.
    if (chunk_m > 1) {
        const int W = 6 + 2 * K;
        const int lx = px_i - tx * TW, ly0 = py_i0 - ty * TH;
        float *part = a.partials + (size_t)(slot0 + chunk_k) * W * TP;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int lp = (ly0 + p) * TW + lx;
            part[0 * TP + lp] = sA[p];
            part[1 * TP + lp] = sR[p];
            part[2 * TP + lp] = sG[p];
            part[3 * TP + lp] = sB[p];
            part[4 * TP + lp] = sP[p];
            part[5 * TP + lp] = __int_as_float(nall[p]);
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k < KMAX - K) continue;
                const int i = k - (KMAX - K);
                part[(size_t)(6 + 2 * i) * TP + lp] = cz[p][k];
                part[(size_t)(7 + 2 * i) * TP + lp] = __uint_as_float(cg[p][k]);
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) s_last = atomicAdd(a.done + slot0, 1u) == (unsigned)(chunk_m - 1);
        __syncthreads();
        if (!s_last) continue;
        __threadfence();
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                cz[p][k] = (k < KMAX - K) ? -INFINITY : INFINITY;
                cg[p][k] = 0xffffffffu;
            }
            sA[p] = sR[p] = sG[p] = sB[p] = 0.f;
            sP[p] = 1.f;
            nall[p] = 0;
        }
        for (int c = 0; c < chunk_m; ++c) {
            const float *pc = a.partials + (size_t)(slot0 + c) * W * TP;
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                const int lp = (ly0 + p) * TW + lx;
                sA[p] += __ldcg(pc + 0 * TP + lp);
                sR[p] += __ldcg(pc + 1 * TP + lp);
                sG[p] += __ldcg(pc + 2 * TP + lp);
                sB[p] += __ldcg(pc + 3 * TP + lp);
                sP[p] *= __ldcg(pc + 4 * TP + lp);
                nall[p] += __float_as_int(__ldcg(pc + 5 * TP + lp));
                for (int i = 0; i < K; ++i) {
                    const float z = __ldcg(pc + (size_t)(6 + 2 * i) * TP + lp);
                    if (!(z < cz[p][KMAX - 1])) break;  // each list is ascending
                    core_insert<KMAX>(cz[p], cg[p], z, __float_as_uint(__ldcg(pc + (size_t)(7 + 2 * i) * TP + lp)));
                }
            }
        }
    }

    // Epilogue: composite the core front to back (Eq. (15)), recover the
    // tail sums and composite the tail behind it.
    const size_t npix = (size_t)width * height;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int x = px_i, y = py_i0 + p;
        if (x >= width || y >= height) continue;
        const size_t pix = (size_t)y * width + x;
        float C[3] = {0.f, 0.f, 0.f};
        float T = 1.f, Ac = 0.f, Sc[3] = {0.f, 0.f, 0.f};
        int n_core = 0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < KMAX - K || !(cz[p][k] < INFINITY)) continue;
            const uint32_t gid = cg[p][k];
            const float4 *r = a.rec + (size_t)gid * kRecF4;
            const float4 c0 = r[0], c1 = r[1], c2 = r[2], c4 = r[4], c5 = r[5];
            FragEval f;
            frag_alpha(quad_eval2(c0, c1, c2, __fsub_rn(px, c4.z), __fsub_rn(py[p], c4.w)), tau_alpha,
                       alpha_max, f);
            const float al = f.alpha;
            const float w = al * T;
            C[0] += w * c5.x; C[1] += w * c5.y; C[2] += w * c5.z;
            Ac += al;
            Sc[0] += al * c5.x; Sc[1] += al * c5.y; Sc[2] += al * c5.z;
            T = __fmaf_rn(-T, al, T);
            if (saved) saved[(size_t)(7 + n_core) * npix + pix] = __uint_as_float(gid);
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
        float *img = image + pix * 3;
        img[0] = C[0] + wt * ct[0] + Pc * a.prm.bg[0];
        img[1] = C[1] + wt * ct[1] + Pc * a.prm.bg[1];
        img[2] = C[2] + wt * ct[2] + Pc * a.prm.bg[2];
        if (saved) {
            saved[0 * npix + pix] = __int_as_float(n_core);
            saved[1 * npix + pix] = T;
            saved[2 * npix + pix] = Pc;
            saved[3 * npix + pix] = At;
            saved[4 * npix + pix] = ct[0];
            saved[5 * npix + pix] = ct[1];
            saved[6 * npix + pix] = ct[2];
            for (int k = n_core; k < K; ++k) saved[(size_t)(7 + k) * npix + pix] = __uint_as_float(0xffffffffu);
        }
    }
    } // next item
}

// ---------------------------------------------------------------------------
// Adjoint (K7). The derivative of the colour with respect to every tail
// fragment uses only per-pixel constants (Sec. 3.3): with u = g (T_c - P)/A,
// k0 = -u.c_tail and k1 = P g.(c_tail - bg), dL/dalpha_j = u.c_j + k0 +
// k1/(1 - alpha_j) and dL/dc_j = u alpha_j. Core fragment r (depth order)
// has dL/dalpha_r = T_r g.(c_r - G_r) and dL/dc_r = g alpha_r T_r, with G_r
// the colour seen behind r.
// ---------------------------------------------------------------------------

// Sums 16 per-lane values over the warp; afterwards lane 8q (q = 0..3) holds
// the sums of values 4q .. 4q + 3 in v[0..3].
__device__ __forceinline__ void warp_reduce16_to4(float (&v)[16], int lane) {
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
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// Dynamic shared memory of the adjoint for a TP-pixel tile and core size K.
__host__ __device__ inline size_t bwd_smem_bytes(int TP, int K) {
    return (size_t)TP * (3 * sizeof(float4) + (size_t)K * 3 * sizeof(float) + sizeof(float));
}

template <int TW, int TH, bool NOTAIL, bool VIS>
__global__ void __launch_bounds__(kBwdThreads, 3) blend_bwd_kernel(const __grid_constant__ Batch bt, BlendBwdArgs a) {
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
    float4 *s_pc = s_pb + TP;            // last core depth, last core gid, mode, -
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
        // mode 0: no core (K = 0); 1: every candidate is in the core; 2: compare with the last entry.
        const int mode = K == 0 ? 0 : (n_core < K ? 1 : 2);
        s_pc[p] = make_float4(lastz, __uint_as_float(lastg), __int_as_float(mode), 0.f);
        if (inside && mode == 1) open_l = true;
        if (inside && mode == 2) zmax_l = fmaxf(zmax_l, lastz);
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
            const float4 c0 = rec[0], c1 = rec[1], c2 = rec[2], c3 = rec[3], c4 = rec[4], c5 = rec[5];
            const float zlo = rec[7].x;
            const bool may_core = tile_open || !(zlo > tile_zmax);
            float2 acc[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] = make_float2(0.f, 0.f);
            float gaa = 0.f, gc0 = 0.f, gc1 = 0.f, gc2 = 0.f;
            float wmax = 0.f;  // largest blending weight of the record in this tile
            bool touched = false;
            const int lx = lane & 7, ly = lane >> 3;
            for (int by = iy0; by <= iy1; by += 4) {
                const int y = by + ly;
                const float dy = __fsub_rn((float)y + 0.5f, c4.w);
                const int prow = (y - y0) * TW - x0;
                for (int bx = ix0; bx <= ix1; bx += 8) {
                    const int x = bx + lx;
                    if (x > ix1 || y > iy1) continue;
                    const float dx = __fsub_rn((float)x + 0.5f, c4.z);
                    FragEval f;
                    if (!frag_alpha(quad_eval2(c0, c1, c2, dx, dy), tau_alpha, alpha_max, f)) continue;
                    const int p = prow + x;
                    const float al = f.alpha;
                    bool in_core = false;
                    if (may_core && al >= tau_K) {
                        const float4 PC = s_pc[p];
                        const int mode = __float_as_int(PC.z);
                        if (mode == 1) {
                            in_core = true;
                        } else if (mode == 2 && !(zlo > PC.x)) {
                            // (depths of this splat are >= zlo, so zlo > last
                            // core depth means the fragment is not in the core)
                            const float z = frag_depth(c3, c4, dx, dy, f.rD);
                            in_core = z < PC.x || (z == PC.x && gid <= __float_as_uint(PC.y));
                        }
                    }
                    if (NOTAIL && !in_core) continue;  // an omitted tail has no gradient
                    float dA, dc0, dc1, dc2;
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
                        dc0 = PA.x * s; dc1 = PA.y * s; dc2 = PA.z * s;
                        if (VIS) wmax = fmaxf(wmax, s);
                    } else {
                        const float4 PB = s_pb[p];
                        const float k0 = s_pa[p].w;
                        const float inv = rcp_approx(1.f - al);
                        dA = PB.x * c5.x + PB.y * c5.y + PB.z * c5.z + k0 + PB.w * inv;
                        dc0 = PB.x * al; dc1 = PB.y * al; dc2 = PB.z * al;
                        if (VIS) wmax = fmaxf(wmax, al * s_wt[p]);
                    }
                    touched = true;
                    gc0 += dc0; gc1 += dc1; gc2 += dc2;
                    if (f.araw < alpha_max) {
                        // With g = alpha dL/dalpha: dL/drho^2 = -g/2, and as
                        // rho^2 = N / D = rho_c - 2 ln2 t, dL/dN = -e/2 and
                        // dL/dD = e rho^2 / 2 = (rho_c e - 2 ln2 e t) / 2 for
                        // e = g / D. The pixel adds the moments of (e, e t);
                        // the (record, tile) sums become dL/dN and dL/dD once,
                        // after the warp reduction.
                        const float g = dA * al;
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
                    }
                }
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

// ---------------------------------------------------------------------------
// Dispatch over tile shape and pixels per thread for one KMAX.
// ---------------------------------------------------------------------------
template <int KMAX, int TW, int TH, int PPT, bool NOTAIL>
bool run_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    constexpr int NT = TW * TH / PPT;
    const void *fn = (const void *)blend_fwd_kernel<KMAX, TW, TH, PPT, NOTAIL>;
    const size_t smem = fwd_smem_bytes(a.tiles.batch);
    if (!allow_dynamic_smem(fn, fwd_smem_bytes(128))) return false;
    const int grid = persistent_grid(fn, NT, smem, a.max_items);
    blend_fwd_kernel<KMAX, TW, TH, PPT, NOTAIL><<<grid, NT, smem, s>>>(b, a);
    return true;
}

template <int KMAX, int PPT, bool NOTAIL = false>
bool dispatch_shape_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_fwd<KMAX, 16, 16, PPT, NOTAIL>(b, a, s);
    if (tw == 16 && th == 8 && PPT <= 2) return run_fwd<KMAX, 16, 8, (PPT <= 2 ? PPT : 2), NOTAIL>(b, a, s);
    if (tw == 8 && th == 8 && PPT <= 2) return run_fwd<KMAX, 8, 8, (PPT <= 2 ? PPT : 2), NOTAIL>(b, a, s);
    return false;
}

} // namespace htgs
