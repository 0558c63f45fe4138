// blend_sorted.cu -- the variant without per-pixel hybrid transparency
// (arXiv 2410.08129, Tab. 3): the perspective-correct fragments of a pixel
// (Sec. 3.2) blended front to back, Eq. (2) plus background, in the order of
// their Gaussians' view-space mean depth (the tile lists come out of the
// binning in that order), stopping before the fragment that would take the
// transmittance below kSortedTmin. Forward and adjoint, one pixel per thread.
//
// The adjoint needs each fragment's transmittance T_i and the colour blended
// in front of it, so every thread walks its pixel's list in order: with
// S_i = (C + T_end c_bg) - sum_{j <= i} T_j alpha_j c_j, the colour behind
// fragment i, dC/dalpha_i = T_i c_i - S_i / (1 - alpha_i) and
// dC/dc_i = T_i alpha_i. A record's 16 gradient sums are reduced per warp,
// added over the tile's warps in shared memory and reduced into global
// memory once per (record, tile).
#include "blend_impl.cuh"
#include "warp_reduce.cuh"

namespace htgs {

namespace {

constexpr int kSortedBwdBatch = 64;  // records per batch of the adjoint

// Shared memory of the sorted forward: three buffers of B staged records
// (kStageF4 float4 slots each: the record and its id).
inline size_t sorted_fwd_smem_bytes(int B) {
    return (size_t)3 * B * kStageF4 * sizeof(float4);
}

// Staging shared by both kernels: batch c of the list into buffer c % 3,
// each record in kStageF4 slots with its id in the last (the 144-byte stride
// keeps the per-lane box loads of the cull free of bank conflicts).
template <int NT>
struct Stager {
    float4 *s_rec;
    const float4 *rec;
    const uint32_t *vals;
    uint2 range;
    int B;
    __device__ int size(int c) const { return (int)min((uint32_t)B, range.y - range.x - (uint32_t)c * B); }
    __device__ void issue(int c, int tid) const {
        const int nb = size(c);
        const uint32_t base = range.x + (uint32_t)c * B;
        float4 *dst = s_rec + (size_t)(c % 3) * B * kStageF4;
        for (int k = tid; k < nb * kRecF4; k += NT) {
            const int j = k / kRecF4, f = k - j * kRecF4;
            const uint32_t gid = vals[base + j];
            if (f == 0) reinterpret_cast<uint32_t *>(dst + j * kStageF4 + kRecF4)[0] = gid;
            cp_async16(dst + j * kStageF4 + f, rec + (size_t)gid * kRecF4 + f);
        }
        cp_async_commit();
    }
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH, 1024 / (TW * TH))
blend_sorted_fwd_kernel(const __grid_constant__ Batch bt, BlendFwdArgs a) {
    dependent_entry();
    constexpr int NT = TW * TH;
    constexpr int WPR = TW / 8;
    extern __shared__ float4 s_dyn[];
    const int B = a.tiles.batch;
    __shared__ int s_item;
    if (a.status[kStError] != 0) return;
    const int n_items = min((int)*a.n_items, a.max_items);
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int4 work = a.items[item];
        if (!item_ok(work, bt.total_tiles, a.slots)) continue;
        const int tile = work.x;
        const ViewDesc &view = bt.v[view_of_tile(bt, tile)];
        const int local = tile - view.tile_off;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const int width = view.cam.width, height = view.cam.height;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int wx0 = tx * TW + (warp % WPR) * 8, wy0 = ty * TH + (warp / WPR) * 4;
        const int px_i = wx0 + (lane & 7), py_i = wy0 + (lane >> 3);
        const float px = (float)px_i + 0.5f, py = (float)py_i + 0.5f;
        const float fx0 = (float)wx0 + 0.5f, fx1 = (float)wx0 + 7.5f;
        const float fy0 = (float)wy0 + 0.5f, fy1 = (float)wy0 + 3.5f;
        const bool inside = px_i < width && py_i < height;
        const float tau_alpha = a.prm.tau_alpha, alpha_max = a.prm.alpha_max;
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        uint32_t last = 0;  // list position after the last blended fragment
        bool done = !inside;

        Stager<NT> st{s_dyn, a.rec, a.vals,
                      a.ranges[tile], B};
        const int nbatches = (int)((st.range.y - st.range.x + B - 1) / B);
        if (nbatches > 0) st.issue(0, tid);
        if (nbatches > 1) st.issue(1, tid);
        for (int b = 0; b < nbatches; ++b) {
            if (b + 1 < nbatches) cp_async_wait<1>();
            else cp_async_wait<0>();
            // Batch b is visible and batch b - 1 is finished; the whole tile may stop here.
            if (__syncthreads_and(done)) break;
            if (b + 2 < nbatches) st.issue(b + 2, tid);
            const int nb = st.size(b);
            const float4(*rec)[kStageF4] =
                reinterpret_cast<const float4(*)[kStageF4]>(st.s_rec + (size_t)(b % 3) * B * kStageF4);
            const uint32_t pos0 = st.range.x + (uint32_t)b * B;
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
                    if (done) continue;
                    const float4 c0 = rec[j][0], c1 = rec[j][1], c2 = rec[j][2], c4 = rec[j][4];
                    FragEval f;
                    if (!frag_alpha(quad_eval2(c0, c1, c2, __fsub_rn(px, c4.z), __fsub_rn(py, c4.w)), tau_alpha,
                                    alpha_max, f))
                        continue;
                    const float Tn = __fmaf_rn(-T, f.alpha, T);
                    if (Tn < kSortedTmin) {
                        done = true;
                        continue;
                    }
                    const float4 c5 = rec[j][5];
                    const float w = f.alpha * T;
                    C0 = __fmaf_rn(w, c5.x, C0);
                    C1 = __fmaf_rn(w, c5.y, C1);
                    C2 = __fmaf_rn(w, c5.z, C2);
                    T = Tn;
                    last = pos0 + (uint32_t)j + 1u;
                }
            }
        }
        cp_async_wait<0>();  // copies of batches not reached after an early stop
        if (inside) {
            const size_t npix = (size_t)width * height, pix = (size_t)py_i * width + px_i;
            float *img = view.image + pix * 3;
            img[0] = C0 + T * a.prm.bg[0];
            img[1] = C1 + T * a.prm.bg[1];
            img[2] = C2 + T * a.prm.bg[2];
            if (float *saved = view.saved) {
                saved[0 * npix + pix] = T;
                saved[1 * npix + pix] = __uint_as_float(last);
                saved[2 * npix + pix] = C0;
                saved[3 * npix + pix] = C1;
                saved[4 * npix + pix] = C2;
            }
        }
        __syncthreads();  // the next item restages the buffers
    }
}

// Shared memory of the adjoint: the staging buffers and, for two batches in
// turn, the records' 16 sums, largest weight, rho_c and id.
__host__ __device__ inline size_t sorted_bwd_smem_bytes() {
    constexpr int B = kSortedBwdBatch;
    return (size_t)3 * B * kStageF4 * sizeof(float4) + (size_t)2 * B * 19 * sizeof(float);
}

template <int TW, int TH, bool VIS>
__global__ void __launch_bounds__(TW *TH, 768 / (TW * TH) > 0 ? 768 / (TW * TH) : 1)
blend_sorted_bwd_kernel(const __grid_constant__ Batch bt, BlendBwdArgs a) {
    dependent_entry();
    constexpr int NT = TW * TH;
    constexpr int WPR = TW / 8;
    constexpr int B = kSortedBwdBatch;
    constexpr float kLn2 = 0.69314718055994531f;
    extern __shared__ float4 s_dyn[];
    float *s_acc = reinterpret_cast<float *>(s_dyn + 3 * B * kStageF4);  // [2][B][19]
    __shared__ int s_item;
    if (a.status[kStError] != 0) return;
    const int n_items = min((int)*a.n_items, a.max_items);
    const long long n_rec = bt.n_rec;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int4 work = a.items[item];
        if (!item_ok(work, bt.total_tiles, a.max_items)) continue;
        const int tile = work.x;
        const ViewDesc &view = bt.v[view_of_tile(bt, tile)];
        const int local = tile - view.tile_off;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const int width = view.cam.width, height = view.cam.height;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int wx0 = tx * TW + (warp % WPR) * 8, wy0 = ty * TH + (warp / WPR) * 4;
        const int px_i = wx0 + (lane & 7), py_i = wy0 + (lane >> 3);
        const float px = (float)px_i + 0.5f, py = (float)py_i + 0.5f;
        const float fx0 = (float)wx0 + 0.5f, fx1 = (float)wx0 + 7.5f;
        const float fy0 = (float)wy0 + 0.5f, fy1 = (float)wy0 + 3.5f;
        const bool inside = px_i < width && py_i < height;
        const float tau_alpha = a.prm.tau_alpha, alpha_max = a.prm.alpha_max;
        const size_t npix = (size_t)width * height, pix = inside ? (size_t)py_i * width + px_i : 0;
        // Per-pixel state: dL/dC, the colour with background, T and the
        // colour blended so far.
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, S0 = 0.f, S1 = 0.f, S2 = 0.f;
        uint32_t last = 0;
        if (inside) {
            const float Tend = view.saved[0 * npix + pix];
            last = __float_as_uint(view.saved[1 * npix + pix]);
            S0 = view.saved[2 * npix + pix] + Tend * a.prm.bg[0];
            S1 = view.saved[3 * npix + pix] + Tend * a.prm.bg[1];
            S2 = view.saved[4 * npix + pix] + Tend * a.prm.bg[2];
            g0 = view.dl_dimg[pix * 3 + 0];
            g1 = view.dl_dimg[pix * 3 + 1];
            g2 = view.dl_dimg[pix * 3 + 2];
        }
        float T = 1.f;  // S tracks the colour behind the current fragment (S_i after it)

        Stager<NT> st{s_dyn, a.rec, a.vals,
                      a.ranges[tile], B};
        const int nbatches = (int)((st.range.y - st.range.x + B - 1) / B);
        // Accumulators of batch c live in slot c & 1; they are cleared before
        // use and flushed after the barrier that follows the batch.
        auto clear = [&](int slot) {
            for (int k = tid; k < B * 19; k += NT) s_acc[slot * B * 19 + k] = 0.f;
        };
        auto flush = [&](int c) {
            const int nb = st.size(c);
            const float *acc = s_acc + (c & 1) * B * 19;
            for (int k = tid; k < nb * 4; k += NT) {
                const int j = k >> 2, q = k & 3;
                const float *v = acc + j * 19;
                const uint32_t gid = __float_as_uint(v[18]);
                if ((long long)gid >= n_rec) continue;
                float o0 = v[4 * q], o1 = v[4 * q + 1], o2 = v[4 * q + 2], o3 = v[4 * q + 3];
                if (q < 3) {  // (sum e m, sum e t m) pairs -> (dL/dN_m, dL/dD_m)
                    const float rc = v[17];
                    const float n0 = -0.5f * o0, d0 = 0.5f * rc * o0 - kLn2 * o1;
                    const float n1 = -0.5f * o2, d1 = 0.5f * rc * o2 - kLn2 * o3;
                    o0 = n0; o1 = d0; o2 = n1; o3 = d1;
                }
                if (o0 != 0.f || o1 != 0.f || o2 != 0.f || o3 != 0.f)
                    red_add_v4(a.acc + (size_t)gid * 16 + q * 4, o0, o1, o2, o3);
                if (VIS && q == 0 && v[16] > 0.f)
                    atomicMax(reinterpret_cast<int *>(a.vis) + gid, __float_as_int(v[16]));
            }
        };
        clear(0);
        clear(1);
        if (nbatches > 0) st.issue(0, tid);
        if (nbatches > 1) st.issue(1, tid);
        for (int b = 0; b < nbatches; ++b) {
            if (b + 1 < nbatches) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
            if (b > 0) {
                flush(b - 1);
                __syncthreads();
                clear((b - 1) & 1);  // slot of batch b + 1
            }
            if (b + 2 < nbatches) st.issue(b + 2, tid);
            const int nb = st.size(b);
            const float4(*rec)[kStageF4] =
                reinterpret_cast<const float4(*)[kStageF4]>(st.s_rec + (size_t)(b % 3) * B * kStageF4);
            float *acc_b = s_acc + (b & 1) * B * 19;
            const uint32_t pos0 = st.range.x + (uint32_t)b * B;
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
                    const float4 c0 = rec[j][0], c1 = rec[j][1], c2 = rec[j][2], c4 = rec[j][4], c5 = rec[j][5];
                    const float dx = __fsub_rn(px, c4.z), dy = __fsub_rn(py, c4.w);
                    float v[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = 0.f;
                    float wmax = 0.f;
                    bool touched = false;
                    FragEval f;
                    if (pos0 + (uint32_t)j < last &&
                        frag_alpha(quad_eval2(c0, c1, c2, dx, dy), tau_alpha, alpha_max, f)) {
                        const float al = f.alpha;
                        const float w = al * T;
                        // Colour behind this fragment, then dL/dalpha and dL/dc.
                        S0 = __fmaf_rn(-w, c5.x, S0);
                        S1 = __fmaf_rn(-w, c5.y, S1);
                        S2 = __fmaf_rn(-w, c5.z, S2);
                        const float inv = rcp_approx(1.f - al);
                        const float dA = g0 * (T * c5.x - S0 * inv) + g1 * (T * c5.y - S1 * inv) +
                                         g2 * (T * c5.z - S2 * inv);
                        v[13] = g0 * w; v[14] = g1 * w; v[15] = g2 * w;
                        if (f.araw < alpha_max) {
                            const float gg = dA * al;
                            v[12] = gg;
                            const float e = gg * f.rD, et = e * f.t;
                            v[0] = e; v[1] = et;
                            v[2] = e * dx; v[3] = et * dx;
                            v[4] = e * dy; v[5] = et * dy;
                            v[6] = e * dx * dx; v[7] = et * dx * dx;
                            v[8] = e * dx * dy; v[9] = et * dx * dy;
                            v[10] = e * dy * dy; v[11] = et * dy * dy;
                        }
                        wmax = w;
                        T = __fmaf_rn(-T, al, T);
                        touched = true;
                    }
                    if (__any_sync(0xffffffffu, touched)) {
                        if (VIS)
                            for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
                        warp_reduce16_to4(v, lane);
                        float *dst = acc_b + j * 19;
                        if ((lane & 7) == 0) {
                            const int q = lane >> 3;
                            atomicAdd(dst + 4 * q + 0, v[0]);
                            atomicAdd(dst + 4 * q + 1, v[1]);
                            atomicAdd(dst + 4 * q + 2, v[2]);
                            atomicAdd(dst + 4 * q + 3, v[3]);
                        }
                        if (lane == 0) {
                            if (VIS) atomicMax(reinterpret_cast<int *>(dst + 16), __float_as_int(wmax));
                            dst[17] = c5.w;
                            dst[18] = rec[j][kRecF4].x;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (nbatches > 0) flush(nbatches - 1);
        __syncthreads();  // the next item restages the buffers
    }
}

template <int TW, int TH>
bool run_sorted_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    const void *fn = (const void *)blend_sorted_fwd_kernel<TW, TH>;
    // (At most 128 records per batch: three buffers of 192 would not fit.)
    BlendFwdArgs args = a;
    if (args.tiles.batch > 128) args.tiles.batch = 128;
    const size_t smem = sorted_fwd_smem_bytes(args.tiles.batch);
    if (!allow_dynamic_smem(fn, sorted_fwd_smem_bytes(128))) return false;
    const int grid = persistent_grid(fn, TW * TH, smem, args.max_items);
    launch_k(blend_sorted_fwd_kernel<TW, TH>, grid, TW * TH, smem, s, b, args);
    return true;
}

template <int TW, int TH, bool VIS>
bool run_sorted_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    const void *fn = (const void *)blend_sorted_bwd_kernel<TW, TH, VIS>;
    const size_t smem = sorted_bwd_smem_bytes();
    if (!allow_dynamic_smem(fn, smem)) return false;
    const int grid = persistent_grid(fn, TW * TH, smem, a.max_items);
    launch_k(blend_sorted_bwd_kernel<TW, TH, VIS>, grid, TW * TH, smem, s, b, a);
    return true;
}

} // namespace

bool launch_blend_sorted_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return run_sorted_fwd<16, 16>(b, a, s);
    if (tw == 32 && th == 16) return run_sorted_fwd<32, 16>(b, a, s);
    if (tw == 16 && th == 8) return run_sorted_fwd<16, 8>(b, a, s);
    if (tw == 8 && th == 8) return run_sorted_fwd<8, 8>(b, a, s);
    return false;
}

bool launch_blend_sorted_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s) {
    const int tw = a.tiles.tile_w, th = a.tiles.tile_h;
    if (tw == 16 && th == 16) return a.vis ? run_sorted_bwd<16, 16, true>(b, a, s) : run_sorted_bwd<16, 16, false>(b, a, s);
    if (tw == 32 && th == 16) return a.vis ? run_sorted_bwd<32, 16, true>(b, a, s) : run_sorted_bwd<32, 16, false>(b, a, s);
    if (tw == 16 && th == 8) return a.vis ? run_sorted_bwd<16, 8, true>(b, a, s) : run_sorted_bwd<16, 8, false>(b, a, s);
    if (tw == 8 && th == 8) return a.vis ? run_sorted_bwd<8, 8, true>(b, a, s) : run_sorted_bwd<8, 8, false>(b, a, s);
    return false;
}

} // namespace htgs
