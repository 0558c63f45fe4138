// api.cu -- the C ABI declared in include/htgs.h: argument checks, the
// workspace layout and the launch sequence of the render path
// (arXiv 2410.08129, Sec. 3.2-3.3; tiling as in Sec. 4.3).
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kMaxCapacity = (1ll << 30) - 1; // look-back count field
constexpr int64_t kMaxGaussians = 0xfffffffell;   // gids are 32-bit

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    // byte offsets inside the workspace
    size_t status, stats, total, ghist, tickets, ranges, lookback, zero_end;
    size_t rec, rect, count, block_sums, keys0, vals0, keys1, vals1, acc, end;
    int n_blocks, n_sort_blocks, passes;
    TileArgs tiles;
    size_t saved_floats;
};

bool make_tiles(const htgs_camera *cam, const htgs_launch *launch, TileArgs &t) {
    t.tile_w = (launch && launch->tile_w) ? launch->tile_w : 16;
    t.tile_h = (launch && launch->tile_h) ? launch->tile_h : 16;
    t.depth_bits = launch ? launch->depth_bits : 0;
    const bool shape_ok = (t.tile_w == 16 && t.tile_h == 16) || (t.tile_w == 16 && t.tile_h == 8) ||
                          (t.tile_w == 8 && t.tile_h == 8);
    if (!shape_ok || t.depth_bits != 0) return false;
    t.tiles_x = (cam->width + t.tile_w - 1) / t.tile_w;
    t.tiles_y = (cam->height + t.tile_h - 1) / t.tile_h;
    if (t.tiles_x > 65535 || t.tiles_y > 65535) return false;
    t.n_tiles = t.tiles_x * t.tiles_y;
    int bits = 1;
    while ((1ll << bits) < t.n_tiles) ++bits;
    t.tile_bits = bits;
    return t.tile_bits + t.depth_bits <= 32;
}

htgs_status make_layout(int64_t n, const htgs_camera *cam, const htgs_params *prm,
                        const htgs_launch *launch, int64_t capacity, Layout &L) {
    if (!cam || !prm || n < 0 || n > kMaxGaussians || capacity < 0 || capacity > kMaxCapacity)
        return HTGS_ERR_INVALID_ARG;
    if (cam->width <= 0 || cam->height <= 0 || cam->width > (1 << 20) || cam->height > (1 << 20))
        return HTGS_ERR_INVALID_ARG;
    if (prm->K < 0) return HTGS_ERR_INVALID_ARG;
    if (prm->K > HTGS_MAX_K) return HTGS_ERR_NOT_SUPPORTED;
    if (!(prm->tau_alpha > 0.f) || !(prm->alpha_max < 1.f) || !(prm->alpha_max > 0.f))
        return HTGS_ERR_INVALID_ARG;
    if (launch && (launch->px_per_thread < 0 || launch->px_per_thread > 4)) return HTGS_ERR_INVALID_ARG;
    if (!make_tiles(cam, launch, L.tiles)) return HTGS_ERR_NOT_SUPPORTED;
    L.n_blocks = (int)((n + kPreThreads - 1) / kPreThreads);
    L.n_sort_blocks = (int)((capacity + kSortTile - 1) / kSortTile);
    if (L.n_sort_blocks < 1) L.n_sort_blocks = 1;
    L.passes = (L.tiles.tile_bits + L.tiles.depth_bits + kRadixBits - 1) / kRadixBits;
    size_t o = 0;
    // Zero-initialised region (one memset per render).
    L.status = o; o = align_up(o + kStSlots * sizeof(int));
    L.stats = o; o = align_up(o + kStatSlots * sizeof(unsigned long long));
    L.total = o; o = align_up(o + 4 * sizeof(uint32_t));
    L.ghist = o; o = align_up(o + kMaxPasses * kRadix * sizeof(uint32_t));
    L.tickets = o; o = align_up(o + kMaxPasses * sizeof(uint32_t));
    L.ranges = o; o = align_up(o + (size_t)L.tiles.n_tiles * sizeof(uint2));
    L.lookback = o; o = align_up(o + (size_t)L.passes * L.n_sort_blocks * kRadix * sizeof(uint32_t));
    L.zero_end = o;
    L.rec = o; o = align_up(o + (size_t)n * kRecF4 * sizeof(float4));
    L.rect = o; o = align_up(o + (size_t)n * sizeof(uint2));
    L.count = o; o = align_up(o + (size_t)n * sizeof(uint32_t));
    L.block_sums = o; o = align_up(o + (size_t)(L.n_blocks + 1) * sizeof(uint32_t));
    L.keys0 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.vals0 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.keys1 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.vals1 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.acc = o; o = align_up(o + (size_t)n * 16 * sizeof(float));
    L.end = o;
    L.saved_floats = (size_t)(7 + prm->K) * cam->width * cam->height;
    return HTGS_OK;
}

void make_cam(const htgs_camera *c, CamArgs &a) {
    for (int i = 0; i < 12; ++i) a.M[i] = c->world_to_cam[i];
    a.fx = c->fx; a.fy = c->fy; a.cx = c->cx; a.cy = c->cy;
    a.z_near = c->z_near;
    a.width = c->width; a.height = c->height;
    // Camera centre -R^T t, in double.
    const float *M = c->world_to_cam;
    for (int i = 0; i < 3; ++i)
        a.centre[i] = (float)(-((double)M[0 * 4 + i] * M[3] + (double)M[1 * 4 + i] * M[7] +
                                (double)M[2 * 4 + i] * M[11]));
}

void make_prm(const htgs_params *p, ParamArgs &a) {
    a.K = p->K;
    a.tau_alpha = p->tau_alpha;
    a.tau_K = p->tau_K;
    a.alpha_max = p->alpha_max;
    for (int i = 0; i < 3; ++i) a.bg[i] = p->bg[i];
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

htgs_status check_gaussians(const htgs_gaussians *g) {
    if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return HTGS_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return HTGS_ERR_INVALID_ARG;
    if (g->n > 0 && !aligned16(g->quats)) return HTGS_ERR_INVALID_ARG;
    return HTGS_OK;
}

template <typename T>
T *at(void *ws, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

int sorted_buffer(const Layout &L) { return L.passes & 1; }

// Records the caller's timing event `idx` of htgs_launch::events, if any.
void mark(const htgs_launch *launch, int idx, cudaStream_t s) {
    if (launch && launch->events[idx]) cudaEventRecord(static_cast<cudaEvent_t>(launch->events[idx]), s);
}

} // namespace

} // namespace htgs

using namespace htgs;

extern "C" {

const char *htgs_status_string(htgs_status s) {
    switch (s) {
    case HTGS_OK: return "ok";
    case HTGS_ERR_INVALID_ARG: return "invalid argument";
    case HTGS_ERR_WORKSPACE: return "workspace or saved buffer too small";
    case HTGS_ERR_OVERFLOW: return "tile instances exceed instance_capacity";
    case HTGS_ERR_CUDA: return "CUDA error";
    case HTGS_ERR_TIMEOUT: return "bounded device wait gave up";
    case HTGS_ERR_NOT_SUPPORTED: return "configuration not supported";
    default: return "unknown status";
    }
}

htgs_status htgs_workspace_size(int64_t n_gaussians, const htgs_camera *cam, const htgs_params *params,
                                const htgs_launch *launch, int64_t instance_capacity, size_t *fwd_bytes,
                                size_t *saved_bytes) {
    Layout L;
    htgs_status st = make_layout(n_gaussians, cam, params, launch, instance_capacity, L);
    if (st) return st;
    if (fwd_bytes) *fwd_bytes = L.end;
    if (saved_bytes) *saved_bytes = L.saved_floats * sizeof(float);
    return HTGS_OK;
}

htgs_status htgs_workspace_layout(int64_t n_gaussians, const htgs_camera *cam, const htgs_params *params,
                                  const htgs_launch *launch, int64_t instance_capacity, htgs_layout *out) {
    if (!out) return HTGS_ERR_INVALID_ARG;
    Layout L;
    htgs_status st = make_layout(n_gaussians, cam, params, launch, instance_capacity, L);
    if (st) return st;
    const int sb = sorted_buffer(L);
    out->rec = L.rec;
    out->rect = L.rect;
    out->count = L.count;
    out->sorted_keys = sb ? L.keys1 : L.keys0;
    out->sorted_vals = sb ? L.vals1 : L.vals0;
    out->ranges = L.ranges;
    out->acc = L.acc;
    out->n_tiles = L.tiles.n_tiles;
    out->tiles_x = L.tiles.tiles_x;
    out->tiles_y = L.tiles.tiles_y;
    out->tile_bits = L.tiles.tile_bits;
    return HTGS_OK;
}

htgs_status htgs_render(const htgs_gaussians *g, const htgs_camera *cam, const htgs_params *params,
                        const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                        int64_t instance_capacity, float *saved, float *image, void *stream) {
    htgs_status st = check_gaussians(g);
    if (st) return st;
    if (!image || !workspace || ((uintptr_t)workspace % kAlign)) return HTGS_ERR_INVALID_ARG;
    Layout L;
    st = make_layout(g->n, cam, params, launch, instance_capacity, L);
    if (st) return st;
    if (workspace_bytes < L.end) return HTGS_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (cudaMemsetAsync(workspace, 0, L.zero_end, s) != cudaSuccess) return HTGS_ERR_CUDA;

    CamArgs ca;
    make_cam(cam, ca);
    ParamArgs pa;
    make_prm(params, pa);
    int *status = at<int>(workspace, L.status);
    uint32_t *total = at<uint32_t>(workspace, L.total);

    mark(launch, 0, s);
    if (L.n_blocks > 0) {
        PreArgs pre{};
        pre.means = g->means; pre.log_scales = g->log_scales; pre.quats = g->quats;
        pre.logits = g->opacity_logits; pre.sh = g->sh;
        pre.n = g->n; pre.sh_degree = g->sh_degree;
        pre.cam = ca; pre.prm = pa; pre.tiles = L.tiles;
        pre.rec = at<float4>(workspace, L.rec);
        pre.rect = at<uint2>(workspace, L.rect);
        pre.count = at<uint32_t>(workspace, L.count);
        pre.block_sums = at<uint32_t>(workspace, L.block_sums);
        pre.stats = at<unsigned long long>(workspace, L.stats);
        preprocess_kernel<<<L.n_blocks, kPreThreads, 0, s>>>(pre);
    }
    mark(launch, 1, s);
    mark(launch, 2, s);
    BinArgs bin{};
    bin.n = g->n; bin.n_blocks = L.n_blocks;
    bin.rect = at<uint2>(workspace, L.rect);
    bin.count = at<uint32_t>(workspace, L.count);
    bin.block_sums = at<uint32_t>(workspace, L.block_sums);
    bin.status = status; bin.capacity = instance_capacity; bin.tiles = L.tiles;
    bin.keys = at<uint32_t>(workspace, L.keys0);
    bin.vals = at<uint32_t>(workspace, L.vals0);
    bin.total = total;
    launch_scan_blocks(bin, s);
    launch_emit(bin, s);

    SortArgs so{};
    so.capacity = instance_capacity; so.total = total; so.passes = L.passes;
    so.keys[0] = at<uint32_t>(workspace, L.keys0); so.vals[0] = at<uint32_t>(workspace, L.vals0);
    so.keys[1] = at<uint32_t>(workspace, L.keys1); so.vals[1] = at<uint32_t>(workspace, L.vals1);
    so.ghist = at<uint32_t>(workspace, L.ghist);
    so.lookback = at<uint32_t>(workspace, L.lookback);
    so.tickets = at<uint32_t>(workspace, L.tickets);
    so.n_sort_blocks = L.n_sort_blocks; so.status = status;
    const int sb = launch_sort(so, s);

    RangeArgs ra{};
    ra.total = total; ra.keys = so.keys[sb]; ra.shift = L.tiles.depth_bits;
    ra.ranges = at<uint2>(workspace, L.ranges); ra.capacity = instance_capacity;
    launch_ranges(ra, L.tiles.n_tiles, s);

    BlendFwdArgs ba{};
    ba.rec = at<float4>(workspace, L.rec);
    ba.vals = so.vals[sb];
    ba.ranges = at<uint2>(workspace, L.ranges);
    ba.status = status; ba.tiles = L.tiles; ba.prm = pa;
    ba.width = cam->width; ba.height = cam->height;
    ba.image = image; ba.saved = saved;
    ba.stats = at<unsigned long long>(workspace, L.stats);
    const int ppt = (launch && launch->px_per_thread) ? launch->px_per_thread : 1;
    mark(launch, 3, s);
    mark(launch, 4, s);
    if (!launch_blend_fwd(ba, ppt, s)) return HTGS_ERR_NOT_SUPPORTED;
    mark(launch, 5, s);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}

htgs_status htgs_render_backward(const htgs_gaussians *g, const htgs_camera *cam,
                                 const htgs_params *params, const htgs_launch *launch, void *workspace,
                                 size_t workspace_bytes, int64_t instance_capacity, const float *saved,
                                 const float *dl_dimage, const htgs_gaussians_grad *grads, void *stream) {
    htgs_status st = check_gaussians(g);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace % kAlign) || !saved || !dl_dimage || !grads)
        return HTGS_ERR_INVALID_ARG;
    if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits ||
                     !grads->sh))
        return HTGS_ERR_INVALID_ARG;
    Layout L;
    st = make_layout(g->n, cam, params, launch, instance_capacity, L);
    if (st) return st;
    if (workspace_bytes < L.end) return HTGS_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    float *acc = at<float>(workspace, L.acc);
    if (g->n > 0 && cudaMemsetAsync(acc, 0, (size_t)g->n * 16 * sizeof(float), s) != cudaSuccess)
        return HTGS_ERR_CUDA;
    ParamArgs pa;
    make_prm(params, pa);
    CamArgs ca;
    make_cam(cam, ca);
    const int sb = sorted_buffer(L);

    BlendBwdArgs bb{};
    bb.rec = at<float4>(workspace, L.rec);
    bb.vals = at<uint32_t>(workspace, sb ? L.vals1 : L.vals0);
    bb.ranges = at<uint2>(workspace, L.ranges);
    bb.status = at<int>(workspace, L.status);
    bb.tiles = L.tiles; bb.prm = pa;
    bb.width = cam->width; bb.height = cam->height;
    bb.saved = saved; bb.dl_dimg = dl_dimage; bb.acc = acc; bb.n = g->n;
    const int ppt = (launch && launch->px_per_thread) ? launch->px_per_thread : 2;
    mark(launch, 0, s);
    if (!launch_blend_bwd(bb, ppt, s)) return HTGS_ERR_NOT_SUPPORTED;
    mark(launch, 1, s);
    mark(launch, 2, s);

    if (L.n_blocks > 0) {
        PreBwdArgs pb{};
        pb.means = g->means; pb.log_scales = g->log_scales; pb.quats = g->quats;
        pb.logits = g->opacity_logits; pb.sh = g->sh;
        pb.n = g->n; pb.sh_degree = g->sh_degree;
        pb.cam = ca; pb.prm = pa;
        pb.rec = at<float4>(workspace, L.rec);
        pb.rect = at<uint2>(workspace, L.rect);
        pb.acc = acc;
        pb.g_means = grads->means; pb.g_log_scales = grads->log_scales; pb.g_quats = grads->quats;
        pb.g_logits = grads->opacity_logits; pb.g_sh = grads->sh;
        preprocess_backward_kernel<<<L.n_blocks, kPreThreads, 0, s>>>(pb);
    }
    mark(launch, 3, s);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}

htgs_status htgs_get_error(void *workspace, size_t workspace_bytes, void *stream, htgs_status *status,
                           int64_t *instances) {
    if (!workspace || !status || workspace_bytes < kStSlots * sizeof(int)) return HTGS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int host[kStSlots];
    if (cudaMemcpyAsync(host, workspace, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HTGS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HTGS_ERR_CUDA;
    *status = host[kStError];
    if (instances)
        *instances = (int64_t)(((uint64_t)(uint32_t)host[kStInstHi] << 32) | (uint32_t)host[kStInstLo]);
    return HTGS_OK;
}

htgs_status htgs_get_counters(void *workspace, size_t workspace_bytes, void *stream, uint64_t *counters) {
    if (!workspace || !counters || workspace_bytes < 2 * kAlign) return HTGS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The counters sit right after the status slots (see make_layout).
    const size_t off = align_up(kStSlots * sizeof(int));
    if (cudaMemcpyAsync(counters, static_cast<char *>(workspace) + off, 4 * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HTGS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}

} // extern "C"
