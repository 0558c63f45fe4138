// blend_impl.cuh -- per-pixel ray-splat evaluation and hybrid-transparency
// blending (arXiv 2410.08129, Sec. 3.2 Eq. (13), Sec. 3.3 Eq. (14)-(16)):
// the forward kernel and the evaluation helpers its adjoints share.
//
// Forward: one CTA per tile of TW x TH pixels; each warp owns an 8 x (4 PPT)
// pixel footprint and each lane PPT vertically adjacent pixels. The tile's
// instance list (gid ascending, no depth order) is staged through shared
// memory in batches of records with cp.async: three buffers deep, so that the
// gathers of the next two batches overlap the evaluation of the current one,
// or, for 192-record batches, two buffers deep (one batch in flight).
// A warp first culls a batch against its footprint (per lane and record a
// bounding-box test and one separating axis against the record's cutoff
// ellipse; one ballot per 32 records) and evaluates only the records that
// touch it. For each pixel one packed FP32x2 evaluation gives the pair
// (Q, D) of a record: Q >= 0 decides rho^2 <= rho_c and D gives alpha. Kept
// fragments update the per-pixel order-independent sums over all fragments
// (sum alpha, sum alpha c, prod (1 - alpha), count) and, when
// alpha >= tau_K, a K-core of (depth, gid) pairs held in registers in
// ascending order. The tail is "all fragments minus the core": its sums are
// recovered in the epilogue, so an evicted core entry needs no colour.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

// A staged record takes kStageF4 = 9 float4 slots: the 8 of the record and
// one holding its id. The 144-byte stride spreads the per-lane cull loads
// (slot 6 and 7 of 32 consecutive records) over every bank: at a 128-byte
// stride all of them fall in the same four banks and each quarter-warp load
// serialises eight ways.
constexpr int kStageF4 = kRecF4 + 1;

// Staging buffers of the forward for B records per batch
// (B = htgs_launch.smem_batch: 32, 64, 128 or 192): three, so that two
// batches are in flight while one is evaluated, or two for 192-record
// batches (the same shared memory as three of 128; one batch in flight).
__host__ __device__ inline int fwd_buffers(int B) { return B > 128 ? 2 : 3; }

// Dynamic shared memory of the forward: the staging buffers of B records
// and as many buffers of B record ids.
__host__ __device__ inline size_t fwd_smem_bytes(int B) {
    return (size_t)fwd_buffers(B) * B * (kStageF4 * sizeof(float4) + sizeof(uint32_t));
}

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
// Resident CTAs per SM the register budget is sized for: at one pixel per
// thread 4 (K <= 8), 3 (K = 16) or 2 (K = 32) CTAs of 256 threads, where the
// core's 2K registers still fit without spilling; 2 x 128 threads at two
// pixels per thread (K <= 8).
template <int KMAX, int PPT, int NT>
constexpr int fwd_min_blocks() {
    constexpr int threads = PPT == 1 ? (KMAX <= 8 ? 1024 : KMAX <= 16 ? 768 : 512)
                                     : (PPT == 2 && KMAX <= 8 ? 512 : NT);
    return threads / NT > 0 ? threads / NT : 1;
}

template <int KMAX, int TW, int TH, int PPT, bool NOTAIL>
__global__ void __launch_bounds__(TW *TH / PPT, fwd_min_blocks<KMAX, PPT, TW * TH / PPT>())
blend_fwd_kernel(const __grid_constant__ Batch bt, BlendFwdArgs a) {
    dependent_entry();
    constexpr int NT = TW * TH / PPT;
    constexpr int WY = 4 * PPT;  // warp footprint: 8 x WY pixels
    constexpr int WPR = TW / 8;  // footprints per tile row
    static_assert(TW % 8 == 0 && TH % WY == 0 && NT % 32 == 0, "unsupported blend shape");
    constexpr int TP = TW * TH;
    extern __shared__ float4 s_dyn[];
    const int B = a.tiles.batch;
    // Whole records in rows of kStageF4 float4s, the id in the last one.
    // (Moving the cull words 6 and 7 to arrays of their own also removes the
    // bank conflicts of the per-lane cull loads but costs registers, and
    // measured 10-15% slower.)
    const int NBUF = fwd_buffers(B);
    float4 *const s_rec = s_dyn;  // [NBUF][B][kStageF4]
    uint32_t *const s_ids = reinterpret_cast<uint32_t *>(s_rec + NBUF * B * kStageF4);  // [NBUF][B]
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
    const float fxc = (float)wx0 + 4.f, fyc = (float)wy0 + 0.5f * WY;  // its centre
    const float fhw = 3.5f, fhh = 0.5f * WY - 0.5f;                     // and half extents

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
    // Staging of batch b's records into buffer b % NBUF; their ids come
    // from the id buffer b % NBUF (staged by cp.async earlier) or, for the
    // first batches, from global memory.
    auto issue = [&](int b, bool ids_staged) {
        if (b >= nbatches) return;
        const int nb = batch_size(b);
        const uint32_t base = range.x + (uint32_t)b * B;
        float4 *dst = s_rec + (size_t)(b % NBUF) * B * kStageF4;
        const uint32_t *ids = s_ids + (b % NBUF) * B;
        for (int k = tid; k < nb * kRecF4; k += NT) {
            const int j = k / kRecF4, f = k - j * kRecF4;
            const uint32_t gid = ids_staged ? ids[j] : a.vals[base + j];
            if (f == 0) reinterpret_cast<uint32_t *>(dst + j * kStageF4 + kRecF4)[0] = gid;
            cp_async16(dst + j * kStageF4 + f, a.rec + (size_t)gid * kRecF4 + f);
        }
    };
    // Staging of batch b's record ids into id buffer b % NBUF.
    auto issue_ids = [&](int b) {
        if (b >= nbatches) return;
        const int nb = batch_size(b);
        const uint32_t base = range.x + (uint32_t)b * B;
        for (int j = tid; j < nb; j += NT) cp_async4(s_ids + (b % NBUF) * B + j, a.vals + base + j);
    };
    // Two batches of records in flight, their ids two batches further
    // ahead, so that no record copy waits on a global load of its id. Every
    // iteration commits two groups (records of b + 2, ids of b + 4; either
    // may be empty), so waiting until two groups remain pending completes
    // the records of b and the ids of b + 2. One barrier per batch: after it,
    // those are visible to every thread and every thread has finished batch
    // b - 1, whose record buffer the copies of batch b + 2 then overwrite
    // (and the ids of b + 1, whose buffer the ids of b + 4 take).
    // With two buffers (192-record batches) one batch of records is in
    // flight and its ids one batch further ahead: every iteration waits for
    // all copies, then issues the records of b + 1 and the ids of b + 2.
    if (NBUF == 3) {
        issue(0, false);
        cp_async_commit();
        issue_ids(2);
        cp_async_commit();
        issue(1, false);
        cp_async_commit();
        issue_ids(3);
        cp_async_commit();
    } else {
        issue(0, false);
        issue_ids(1);
        cp_async_commit();
    }
    for (int b = 0; b < nbatches; ++b) {
        if (NBUF == 3) {
            cp_async_wait<2>();
            __syncthreads();
            issue(b + 2, true);
            cp_async_commit();
            issue_ids(b + 4);
            cp_async_commit();
        } else {
            cp_async_wait<0>();
            __syncthreads();
            issue(b + 1, true);
            issue_ids(b + 2);
            cp_async_commit();
        }
        const int nb = batch_size(b);
        const float4(*rec)[kStageF4] =
            reinterpret_cast<const float4(*)[kStageF4]>(s_rec + (size_t)(b % NBUF) * B * kStageF4);
        for (int c = 0; c < nb; c += 32) {
            // Lane c + l tests record c + l against the warp's footprint:
            // its box, then the axis n = A v through the cutoff ellipse
            // p^T A p <= 1 (centred on the box), v from the ellipse's centre
            // to the footprint's. Over the footprint n.(p - centre) >= near,
            // over the ellipse it is <= sqrt(v^T A v): near beyond that
            // separates them. A = 0 (no ellipse) never separates.
            bool hit = false;
            if (c + lane < nb) {
                const float4 bb = rec[c + lane][6];
                hit = bb.x <= fx1 && bb.y >= fx0 && bb.z <= fy1 && bb.w >= fy0;
                if (hit) {
                    const float4 cu = rec[c + lane][7];
                    const float vx = fxc - 0.5f * (bb.x + bb.y), vy = fyc - 0.5f * (bb.z + bb.w);
                    const float nx = cu.y * vx + cu.z * vy, ny = cu.z * vx + cu.w * vy;
                    const float sv = vx * nx + vy * ny;
                    const float near = sv - fabsf(nx) * fhw - fabsf(ny) * fhh;
                    hit = !(near > 0.f && near * near > sv);
                }
            }
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            // The kept-fragment work of record j at this lane's pixels, from
            // its (Q, D) pairs.
            auto blend_record = [&](int j, const float2 (&qd)[PPT]) {
                const float4 c3 = rec[j][3], c4 = rec[j][4], c5 = rec[j][5];
                const float zlo = rec[j][7].x;
                const uint32_t gid = reinterpret_cast<const uint32_t *>(&rec[j][kRecF4])[0];
                const float dx = __fsub_rn(px, c4.z);
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
            };
            // With a small core (K <= 4) two records per step: both (Q, D)
            // evaluations are independent chains, and the fragments are then
            // blended in record order (1080p frame at K = 4: 0.686 -> 0.653 ms).
            // A larger core leaves no registers for the second record's pairs
            // under the 4-CTA budget (K = 8: no gain and a spill at the cap),
            // so it takes one record per step.
            constexpr bool kPair = KMAX <= 4;
            while (mask) {
                const int ja = c + __ffs(mask) - 1;
                mask &= mask - 1;
                const int jb = (kPair && mask) ? c + __ffs(mask) - 1 : -1;
                if (kPair && mask) mask &= mask - 1;
                float2 qa[PPT], qb[PPT];
                bool anya = false, anyb = false;
                {
                    const float4 c0 = rec[ja][0], c1 = rec[ja][1], c2 = rec[ja][2], c4 = rec[ja][4];
                    const float dx = __fsub_rn(px, c4.z);
#pragma unroll
                    for (int p = 0; p < PPT; ++p) {
                        qa[p] = quad_eval2(c0, c1, c2, dx, __fsub_rn(py[p], c4.w));
                        anya |= qa[p].x >= 0.f;
                    }
                }
                if (kPair && jb >= 0) {
                    const float4 c0 = rec[jb][0], c1 = rec[jb][1], c2 = rec[jb][2], c4 = rec[jb][4];
                    const float dx = __fsub_rn(px, c4.z);
#pragma unroll
                    for (int p = 0; p < PPT; ++p) {
                        qb[p] = quad_eval2(c0, c1, c2, dx, __fsub_rn(py[p], c4.w));
                        anyb |= qb[p].x >= 0.f;
                    }
                }
                if (anya) blend_record(ja, qa);
                if (kPair && anyb) blend_record(jb, qb);
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
// Dispatch over tile shape and pixels per thread for one KMAX.
// ---------------------------------------------------------------------------
template <int KMAX, int TW, int TH, int PPT, bool NOTAIL>
bool run_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    constexpr int NT = TW * TH / PPT;
    const void *fn = (const void *)blend_fwd_kernel<KMAX, TW, TH, PPT, NOTAIL>;
    const size_t smem = fwd_smem_bytes(a.tiles.batch);
    if (!allow_dynamic_smem(fn, fwd_smem_bytes(128) > fwd_smem_bytes(192) ? fwd_smem_bytes(128)
                                                                          : fwd_smem_bytes(192)))
        return false;
    const int grid = persistent_grid(fn, NT, smem, a.max_items);
    launch_k(blend_fwd_kernel<KMAX, TW, TH, PPT, NOTAIL>, grid, NT, smem, s, b, a);
    return true;
}

template <int KMAX, int PPT, bool NOTAIL = false>
bool dispatch_shape_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_fwd<KMAX, 16, 16, PPT, NOTAIL>(b, a, s);
    if (tw == 32 && th == 16) return run_fwd<KMAX, 32, 16, (PPT <= 2 ? PPT : 2), NOTAIL>(b, a, s);
    if (tw == 16 && th == 8 && PPT <= 2) return run_fwd<KMAX, 16, 8, (PPT <= 2 ? PPT : 2), NOTAIL>(b, a, s);
    if (tw == 8 && th == 8 && PPT <= 2) return run_fwd<KMAX, 8, 8, (PPT <= 2 ? PPT : 2), NOTAIL>(b, a, s);
    return false;
}

} // namespace htgs
