// api.cu -- the C ABI declared in include/htgs.h: argument checks, the
// workspace layout and the launch sequence of the render path
// (arXiv 2410.08129, Sec. 3.2-3.3; tiling as in Sec. 4.3).
//
// Every render is a batch of views; the single-view entry points build a
// batch of one. The launch sequence per batch is fixed: memset of the zeroed
// workspace region, preprocess, scan, emit, histogram + onesweep passes,
// ranges, persistent blend. Nothing synchronises the stream, so the whole
// sequence can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

namespace {

constexpr size_t kAlign = 256;
constexpr int64_t kMaxCapacity = HTGS_MAX_CAPACITY;  // 32-bit indices, headroom for grid strides
constexpr int64_t kMaxRecords = 0xfffffffell;     // record ids are 32-bit

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    // byte offsets inside the workspace
    size_t status, stats, total, work, ghist, tickets, ranges, lookback, n_items, done;
    size_t d_ghist, d_tickets, d_lookback, zero_end;  // depth sort (sorted blending)
    size_t dkeys0, dvals0, dkeys1, dvals1, count_p, block_sums_p;
    int sorted, n_dsort_blocks;
    size_t rec, rect, cover, count, block_sums, keys0, vals0, keys1, vals1, items, partials, bwd_work, acc, vis, end;
    int n_blocks, n_sort_blocks, passes, digit_bits, slots_cap, max_items;
    // Counting-sort binning (used when `cs`): per-block tile counts and
    // offsets, per-tile totals.
    int cs;
    CsPlan csp;
    size_t cs_hist, cs_off, cs_tot;
    TileArgs tiles;
    int64_t n_rec;
};

bool tile_shape(const htgs_launch *launch, TileArgs &t) {
    t.tile_w = (launch && launch->tile_w) ? launch->tile_w : 16;
    t.tile_h = (launch && launch->tile_h) ? launch->tile_h : 16;
    t.depth_bits = launch ? launch->depth_bits : 0;
    t.batch = (launch && launch->smem_batch) ? launch->smem_batch : 128;
    t.cover = launch ? launch->tile_cover : 0;
    const bool shape_ok = (t.tile_w == 16 && t.tile_h == 16) || (t.tile_w == 16 && t.tile_h == 8) ||
                          (t.tile_w == 8 && t.tile_h == 8) || (t.tile_w == 32 && t.tile_h == 16);
    const bool batch_ok = t.batch == 32 || t.batch == 64 || t.batch == 128 || t.batch == 192;
    return shape_ok && batch_ok && t.depth_bits == 0;
}

bool camera_ok(const htgs_camera *cam) {
    return cam && cam->width > 0 && cam->height > 0 && cam->width <= (1 << 20) && cam->height <= (1 << 20);
}

htgs_status params_ok(const htgs_params *prm, const htgs_launch *launch) {
    if (!prm || prm->K < 0) return HTGS_ERR_INVALID_ARG;
    if (prm->K > HTGS_MAX_K) return HTGS_ERR_NOT_SUPPORTED;
    if (!(prm->tau_alpha > 0.f) || !(prm->alpha_max < 1.f) || !(prm->alpha_max > 0.f))
        return HTGS_ERR_INVALID_ARG;
    if (launch && (launch->px_per_thread < 0 || launch->px_per_thread > 4)) return HTGS_ERR_INVALID_ARG;
    if (launch && (launch->tile_cover < 0 || launch->tile_cover > 1)) return HTGS_ERR_INVALID_ARG;
    return HTGS_OK;
}

// The host-side description of a batch: per view its Gaussian count and camera.
struct HostView {
    int64_t n;
    const htgs_camera *cam;
};

htgs_status make_layout(int n_views, const HostView *views, const htgs_params *prm, const htgs_launch *launch,
                        int64_t capacity, Layout &L) {
    if (n_views < 1 || n_views > kMaxViews || capacity < 0 || capacity > kMaxCapacity)
        return HTGS_ERR_INVALID_ARG;
    htgs_status st = params_ok(prm, launch);
    if (st) return st;
    if (!tile_shape(launch, L.tiles)) return HTGS_ERR_NOT_SUPPORTED;
    int64_t n_rec = 0, n_tiles = 0, tiles_x0 = 0, tiles_y0 = 0;
    for (int v = 0; v < n_views; ++v) {
        if (!camera_ok(views[v].cam) || views[v].n < 0) return HTGS_ERR_INVALID_ARG;
        const int64_t tx = (views[v].cam->width + L.tiles.tile_w - 1) / L.tiles.tile_w;
        const int64_t ty = (views[v].cam->height + L.tiles.tile_h - 1) / L.tiles.tile_h;
        if (tx > 65535 || ty > 65535) return HTGS_ERR_NOT_SUPPORTED;
        n_rec += views[v].n;
        n_tiles += tx * ty;
        if (v == 0) { tiles_x0 = tx; tiles_y0 = ty; }
    }
    if (n_rec > kMaxRecords || n_tiles > (1ll << 30)) return HTGS_ERR_INVALID_ARG;
    L.n_rec = n_rec;
    L.tiles.n_tiles = (int)n_tiles;
    L.tiles.tiles_x = 0;
    L.tiles.tiles_y = 0;
    int bits = 1;
    while ((1ll << bits) < n_tiles) ++bits;
    L.tiles.tile_bits = bits;
    L.n_blocks = (int)((n_rec + kPreThreads - 1) / kPreThreads);
    L.n_sort_blocks = (int)((capacity + kSortTile - 1) / kSortTile);
    if (L.n_sort_blocks < 1) L.n_sort_blocks = 1;
    // Fewest passes of at most kMaxRadixBits bits, the bits split evenly.
    L.passes = (bits + kMaxRadixBits - 1) / kMaxRadixBits;
    L.digit_bits = (bits + L.passes - 1) / L.passes;
    size_t o = 0;
    // Zero-initialised region (one memset per render).
    L.status = o; o = align_up(o + kStSlots * sizeof(int));
    L.stats = o; o = align_up(o + kStatSlots * sizeof(unsigned long long));
    L.total = o; o = align_up(o + 4 * sizeof(uint32_t));
    L.work = o; o = align_up(o + 4 * sizeof(uint32_t));
    L.ghist = o; o = align_up(o + kMaxPasses * kMaxRadix * sizeof(uint32_t));
    L.tickets = o; o = align_up(o + kMaxPasses * sizeof(uint32_t));
    L.ranges = o; o = align_up(o + (size_t)n_tiles * sizeof(uint2));
    L.lookback = o;  // (plus one word nothing writes: the target of htgs_launch.test_lookback_stall)
    o = align_up(o + ((size_t)L.passes * L.n_sort_blocks * ((size_t)1 << L.digit_bits) + 1) *
                         sizeof(unsigned long long));
    // Split-tile slots: enough for chunks of kMinChunk over the whole capacity, at most kMaxSlots.
    L.slots_cap = (int)std::min<int64_t>(kMaxSlots, 2 * ((capacity + kMinChunk - 1) / kMinChunk) + 2);
    L.max_items = (int)(n_tiles + L.slots_cap);
    L.n_items = o; o = align_up(o + 4 * sizeof(uint32_t));
    // Sorted blending: a 4-pass 32-bit radix sort of the records by mean depth.
    L.sorted = prm->sorted_blend ? 1 : 0;
    const bool dsort = L.sorted;
    L.n_dsort_blocks = dsort ? (int)std::max<int64_t>(1, (n_rec + kSortTile - 1) / kSortTile) : 0;
    L.d_ghist = o; o = align_up(o + (dsort ? kMaxPasses * kMaxRadix * sizeof(uint32_t) : 0));
    L.d_tickets = o; o = align_up(o + (dsort ? kMaxPasses * sizeof(uint32_t) : 0));
    L.d_lookback = o; o = align_up(o + (size_t)(dsort ? 4 : 0) * L.n_dsort_blocks * 256 * sizeof(unsigned long long));
    L.done = o; o = align_up(o + (size_t)L.slots_cap * sizeof(uint32_t));
    L.zero_end = o;
    L.rec = o; o = align_up(o + (size_t)n_rec * kRecF4 * sizeof(float4));
    L.rect = o; o = align_up(o + (size_t)n_rec * sizeof(uint2));
    L.cover = o; o = align_up(o + (size_t)n_rec * 2 * sizeof(uint4));
    L.count = o; o = align_up(o + (size_t)n_rec * sizeof(uint32_t));
    L.block_sums = o; o = align_up(o + (size_t)(L.n_blocks + 1) * sizeof(uint32_t));
    const size_t dn = dsort ? (size_t)n_rec : 0;
    L.dkeys0 = o; o = align_up(o + dn * sizeof(uint32_t));
    L.dvals0 = o; o = align_up(o + dn * sizeof(uint32_t));
    L.dkeys1 = o; o = align_up(o + dn * sizeof(uint32_t));
    L.dvals1 = o; o = align_up(o + dn * sizeof(uint32_t));
    L.count_p = o; o = align_up(o + dn * sizeof(uint32_t));
    L.block_sums_p = o; o = align_up(o + (dsort ? (size_t)(L.n_blocks + 1) : 0) * sizeof(uint32_t));
    L.keys0 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.vals0 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.keys1 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    L.vals1 = o; o = align_up(o + (size_t)capacity * sizeof(uint32_t));
    // Counting-sort binning when every tile's counters fit shared memory and
    // the per-(block, tile) matrix is not much larger than the instances.
    const int binning = launch ? launch->binning : 0;
    if (binning < 0 || binning > 2) return HTGS_ERR_INVALID_ARG;
    const bool cs_ok = cs_plan(n_views, (int)tiles_x0, (int)tiles_y0, n_rec, L.csp);
    if (binning == 2 && !cs_ok) return HTGS_ERR_NOT_SUPPORTED;
    // The counting sort builds the same lists; measured on the 1080p frame it
    // is no faster than the radix sort (0.167 vs 0.168 ms at 16x16, slower
    // at 16x8 and 8x8), so it runs only when asked for.
    L.cs = binning == 2 ? 1 : 0;
    const size_t cs_cells = L.cs ? (size_t)L.csp.nb * (size_t)n_tiles : 0;
    L.cs_hist = o; o = align_up(o + cs_cells * sizeof(uint16_t));
    L.cs_off = o; o = align_up(o + cs_cells * sizeof(uint32_t));
    L.cs_tot = o; o = align_up(o + (L.cs ? (size_t)n_tiles : 0) * sizeof(uint32_t));
    L.items = o; o = align_up(o + (size_t)L.max_items * sizeof(int4));
    L.partials = o;
    o = align_up(o + (size_t)L.slots_cap * (6 + 2 * prm->K) * L.tiles.tile_w * L.tiles.tile_h * sizeof(float));
    L.bwd_work = o; o = align_up(o + 4 * sizeof(uint32_t));
    L.acc = o; o = align_up(o + (size_t)n_rec * 16 * sizeof(float));
    L.vis = o; o = align_up(o + (size_t)n_rec * sizeof(float));
    L.end = o;
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
    a.no_tail = p->no_tail ? 1 : 0;
    a.sorted_blend = p->sorted_blend ? 1 : 0;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// A baked scene (forward only) needs its aligned records; a raw one its five
// parameter arrays.
htgs_status check_gaussians(const htgs_gaussians *g, bool backward = false) {
    if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3) return HTGS_ERR_INVALID_ARG;
    if (g->baked) {
        if (backward || !aligned16(g->baked)) return HTGS_ERR_INVALID_ARG;
        return HTGS_OK;
    }
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

htgs_status collect(int n_views, const htgs_view *views, HostView *hv, bool backward = false) {
    if (!views || n_views < 1 || n_views > kMaxViews) return HTGS_ERR_INVALID_ARG;
    for (int v = 0; v < n_views; ++v) {
        htgs_status st = check_gaussians(views[v].gaussians, backward);
        if (st) return st;
        hv[v].n = views[v].gaussians->n;
        hv[v].cam = &views[v].camera;
    }
    return HTGS_OK;
}

// The device-side batch descriptor (passed by value to the kernels).
void make_batch(int n_views, const htgs_view *views, const Layout &L, bool backward, Batch &b) {
    memset(&b, 0, sizeof(b));
    b.n_views = n_views;
    b.n_rec = L.n_rec;
    b.total_tiles = L.tiles.n_tiles;
    long long rec = 0;
    int tile = 0;
    for (int v = 0; v < n_views; ++v) {
        const htgs_view &hv = views[v];
        ViewDesc &d = b.v[v];
        make_cam(&hv.camera, d.cam);
        const htgs_gaussians *g = hv.gaussians;
        d.means = g->means; d.log_scales = g->log_scales; d.quats = g->quats;
        d.logits = g->opacity_logits; d.sh = g->sh; d.filter_var = g->filter_var; d.baked = g->baked;
        d.n = g->n;
        d.sh_degree = g->sh_degree;
        d.rec_off = rec;
        d.tile_off = tile;
        d.tiles_x = (hv.camera.width + L.tiles.tile_w - 1) / L.tiles.tile_w;
        d.tiles_y = (hv.camera.height + L.tiles.tile_h - 1) / L.tiles.tile_h;
        d.image = hv.image;
        d.saved = hv.saved;
        if (backward) {
            d.dl_dimg = hv.dl_dimage;
            d.g_means = hv.grads->means; d.g_log_scales = hv.grads->log_scales;
            d.g_quats = hv.grads->quats; d.g_logits = hv.grads->opacity_logits; d.g_sh = hv.grads->sh;
            d.g_vis = hv.grads->visibility; d.g_dgrad = hv.grads->densify_grad;
            d.g_dcount = hv.grads->densify_count;
        } else {
            d.dl_dimg = nullptr;
            d.g_means = d.g_log_scales = d.g_quats = d.g_logits = d.g_sh = nullptr;
            d.g_vis = d.g_dgrad = d.g_dcount = nullptr;
        }
        rec += g->n;
        tile += d.tiles_x * d.tiles_y;
    }
}

// The kernels of one call are launched as programmatic dependents of their
// predecessors, unless the caller asked for timing events between the phases
// (an event recorded between two dependent kernels would not mark the
// boundary between them).
struct DependentLaunchScope {
    explicit DependentLaunchScope(const htgs_launch *launch) {
        bool events = false;
        if (launch)
            for (int i = 0; i < 6; ++i) events |= launch->events[i] != nullptr;
        set_dependent_launch(!events);
    }
    ~DependentLaunchScope() { set_dependent_launch(false); }
};

htgs_status render_batch_impl(int n_views, const htgs_view *views, const htgs_params *params,
                              const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                              int64_t capacity, void *stream);
htgs_status render_batch_backward_impl(int n_views, const htgs_view *views, const htgs_params *params,
                                       const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                                       int64_t capacity, void *stream);

htgs_status render_batch(int n_views, const htgs_view *views, const htgs_params *params,
                         const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                         int64_t capacity, void *stream) {
    DependentLaunchScope scope(launch);
    return render_batch_impl(n_views, views, params, launch, workspace, workspace_bytes, capacity, stream);
}

htgs_status render_batch_backward(int n_views, const htgs_view *views, const htgs_params *params,
                                  const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                                  int64_t capacity, void *stream) {
    DependentLaunchScope scope(launch);
    return render_batch_backward_impl(n_views, views, params, launch, workspace, workspace_bytes, capacity,
                                      stream);
}

htgs_status render_batch_impl(int n_views, const htgs_view *views, const htgs_params *params,
                              const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                              int64_t capacity, void *stream) {
    HostView hv[kMaxViews];
    htgs_status st = collect(n_views, views, hv);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace % kAlign)) return HTGS_ERR_INVALID_ARG;
    for (int v = 0; v < n_views; ++v)
        if (!views[v].image) return HTGS_ERR_INVALID_ARG;
    Layout L;
    st = make_layout(n_views, hv, params, launch, capacity, L);
    if (st) return st;
    if (workspace_bytes < L.end) return HTGS_ERR_WORKSPACE;
    static thread_local Batch b; // large; built on the host per call
    make_batch(n_views, views, L, false, b);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (cudaMemsetAsync(workspace, 0, L.zero_end, s) != cudaSuccess) return HTGS_ERR_CUDA;

    ParamArgs pa;
    make_prm(params, pa);
    int *status = at<int>(workspace, L.status);
    uint32_t *total = at<uint32_t>(workspace, L.total);

    mark(launch, 0, s);
    if (L.n_blocks > 0) {
        PreArgs pre{};
        pre.prm = pa; pre.tiles = L.tiles;
        pre.rec = at<float4>(workspace, L.rec);
        pre.rect = at<uint2>(workspace, L.rect);
        pre.cover = at<uint4>(workspace, L.cover);
        pre.count = at<uint32_t>(workspace, L.count);
        pre.block_sums = at<uint32_t>(workspace, L.block_sums);
        pre.stats = at<unsigned long long>(workspace, L.stats);
        if (L.sorted) {
            pre.dkey = at<uint32_t>(workspace, L.dkeys0);
            pre.dval = at<uint32_t>(workspace, L.dvals0);
            pre.dtotal = total + 1;
        }
        bool any_baked = false;
        for (int v = 0; v < n_views; ++v) any_baked |= views[v].gaussians->baked != nullptr;
        launch_preprocess(any_baked, L.n_blocks, b, pre, s);
    }
    mark(launch, 1, s);
    mark(launch, 2, s);
    BinArgs bin{};
    bin.n = L.n_rec; bin.n_blocks = L.n_blocks;
    bin.rect = at<uint2>(workspace, L.rect);
    bin.cover = at<uint4>(workspace, L.cover);
    bin.tile_w = L.tiles.tile_w; bin.tile_h = L.tiles.tile_h; bin.use_ellipse = L.tiles.cover == 0;
    bin.count = at<uint32_t>(workspace, L.count);
    bin.block_sums = at<uint32_t>(workspace, L.block_sums);
    if (L.sorted && L.n_blocks > 0) {
        // Records in order of view-space mean depth (stable, so equal depths
        // keep the record order); emitting in that order makes every tile's
        // list depth-ordered after the stable tile sort.
        SortArgs ds{};
        ds.capacity = L.n_rec; ds.total = total + 1; ds.passes = 4; ds.digit_bits = 8;
        ds.keys[0] = at<uint32_t>(workspace, L.dkeys0); ds.vals[0] = at<uint32_t>(workspace, L.dvals0);
        ds.keys[1] = at<uint32_t>(workspace, L.dkeys1); ds.vals[1] = at<uint32_t>(workspace, L.dvals1);
        ds.ghist = at<uint32_t>(workspace, L.d_ghist);
        ds.lookback = at<unsigned long long>(workspace, L.d_lookback);
        ds.tickets = at<uint32_t>(workspace, L.d_tickets);
        ds.n_sort_blocks = L.n_dsort_blocks; ds.status = status;
        const int db = launch_sort(ds, s);
        bin.perm = ds.vals[db];
        bin.count = at<uint32_t>(workspace, L.count_p);
        bin.block_sums = at<uint32_t>(workspace, L.block_sums_p);
        launch_permute_counts(L.n_rec, bin.perm, at<uint32_t>(workspace, L.count), at<uint32_t>(workspace, L.count_p),
                              at<uint32_t>(workspace, L.block_sums_p), s);
    }
    bin.status = status; bin.capacity = capacity;
    bin.keys = at<uint32_t>(workspace, L.keys0);
    bin.vals = at<uint32_t>(workspace, L.vals0);
    bin.total = total;
    uint32_t *sorted_vals = at<uint32_t>(workspace, sorted_buffer(L) ? L.vals1 : L.vals0);
    ScheduleArgs sc{};
    sc.total = total; sc.ranges = at<uint2>(workspace, L.ranges); sc.n_tiles = L.tiles.n_tiles;
    sc.no_split = L.sorted;  // early termination does not merge across chunks
    sc.slots_cap = L.slots_cap;
    sc.items = at<int4>(workspace, L.items);
    sc.n_items = at<uint32_t>(workspace, L.n_items);
    sc.status = status;
    // (The look-back test hook exercises the radix sort's bounded wait.)
    if (L.cs && !(launch && launch->test_lookback_stall)) {
        // Stable counting sort by tile: counts per (block, tile), their
        // prefix over blocks, tile ranges (in the schedule kernel), scatter.
        CsArgs ca{};
        ca.n = L.n_rec; ca.nb = L.csp.nb; ca.gauss = L.csp.gauss;
        ca.n_tiles = L.tiles.n_tiles; ca.tiles_x = b.v[0].tiles_x; ca.tiles_y = b.v[0].tiles_y;
        ca.band_rows = L.csp.band_rows; ca.n_bands = L.csp.n_bands;
        ca.perm = bin.perm; ca.rect = bin.rect; ca.count = bin.count;
        ca.cover = bin.cover; ca.tile_w = bin.tile_w; ca.tile_h = bin.tile_h; ca.use_ellipse = bin.use_ellipse;
        ca.hist = at<uint16_t>(workspace, L.cs_hist);
        ca.off = at<uint32_t>(workspace, L.cs_off);
        ca.tile_tot = at<uint32_t>(workspace, L.cs_tot);
        ca.ranges = sc.ranges; ca.vals = sorted_vals;
        ca.status = status; ca.capacity = capacity;
        launch_cs_count(ca, s);
        launch_cs_colscan(ca, s);
        sc.tile_tot = ca.tile_tot; sc.ranges_out = at<uint2>(workspace, L.ranges);
        sc.total_out = total; sc.capacity = capacity;
        launch_schedule(sc, s);
        launch_cs_emit(ca, s);
    } else {
        launch_scan_blocks(bin, s);
        launch_emit(b, bin, s);
        SortArgs so{};
        so.capacity = capacity; so.total = total; so.passes = L.passes; so.digit_bits = L.digit_bits;
        so.keys[0] = at<uint32_t>(workspace, L.keys0); so.vals[0] = at<uint32_t>(workspace, L.vals0);
        so.keys[1] = at<uint32_t>(workspace, L.keys1); so.vals[1] = at<uint32_t>(workspace, L.vals1);
        so.ghist = at<uint32_t>(workspace, L.ghist);
        so.lookback = at<unsigned long long>(workspace, L.lookback);
        so.tickets = at<uint32_t>(workspace, L.tickets);
        so.n_sort_blocks = L.n_sort_blocks; so.status = status;
        so.stall_first = (launch && launch->test_lookback_stall) ? 1 : 0;
        const int sb = launch_sort(so, s);
        if (so.vals[sb] != sorted_vals) return HTGS_ERR_CUDA;  // the layout's buffer choice is the sort's
        RangeArgs ra{};
        ra.total = total; ra.keys = so.keys[sb];
        ra.ranges = at<uint2>(workspace, L.ranges); ra.n_tiles = L.tiles.n_tiles;
        launch_ranges(ra, s);
        launch_schedule(sc, s);
    }

    BlendFwdArgs ba{};
    ba.rec = at<float4>(workspace, L.rec);
    ba.vals = sorted_vals;
    ba.ranges = at<uint2>(workspace, L.ranges);
    ba.items = sc.items; ba.n_items = sc.n_items; ba.max_items = L.max_items; ba.slots = L.slots_cap;
    ba.partials = at<float>(workspace, L.partials);
    ba.done = at<unsigned int>(workspace, L.done);
    ba.status = status;
    ba.work = at<unsigned int>(workspace, L.work);
    ba.tiles = L.tiles; ba.prm = pa;
    ba.stats = at<unsigned long long>(workspace, L.stats);
    const int ppt = (launch && launch->px_per_thread) ? launch->px_per_thread : 1;
    mark(launch, 3, s);
    mark(launch, 4, s);
    if (L.sorted ? !launch_blend_sorted_fwd(b, ba, s) : !launch_blend_fwd(b, ba, ppt, s)) return HTGS_ERR_NOT_SUPPORTED;
    mark(launch, 5, s);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}

htgs_status render_batch_backward_impl(int n_views, const htgs_view *views, const htgs_params *params,
                                       const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                                       int64_t capacity, void *stream) {
    HostView hv[kMaxViews];
    htgs_status st = collect(n_views, views, hv, true);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace % kAlign)) return HTGS_ERR_INVALID_ARG;
    for (int v = 0; v < n_views; ++v) {
        const htgs_view &w = views[v];
        const htgs_gaussians_grad *gr = w.grads;
        if (!w.saved || !w.dl_dimage || !gr) return HTGS_ERR_INVALID_ARG;
        if (w.gaussians->n > 0 && (!gr->means || !gr->log_scales || !gr->quats || !gr->opacity_logits || !gr->sh))
            return HTGS_ERR_INVALID_ARG;
    }
    Layout L;
    st = make_layout(n_views, hv, params, launch, capacity, L);
    if (st) return st;
    if (workspace_bytes < L.end) return HTGS_ERR_WORKSPACE;
    static thread_local Batch b;
    make_batch(n_views, views, L, true, b);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    // Views that share gradient buffers (several views of one scene) add
    // into them; those buffers start from zero.
    bool accumulate = false;
    for (int v = 0; v < n_views && !accumulate; ++v)
        for (int u = 0; u < v; ++u)
            if (views[u].grads->means == views[v].grads->means) { accumulate = true; break; }
    if (accumulate) {
        for (int v = 0; v < n_views; ++v) {
            bool first = true;
            for (int u = 0; u < v; ++u)
                if (views[u].grads->means == views[v].grads->means) first = false;
            const int64_t n = views[v].gaussians->n;
            if (!first || n == 0) continue;
            const htgs_gaussians_grad *gr = views[v].grads;
            const int nc = (views[v].gaussians->sh_degree + 1) * (views[v].gaussians->sh_degree + 1);
            if (cudaMemsetAsync(gr->means, 0, (size_t)n * 3 * sizeof(float), s) != cudaSuccess ||
                cudaMemsetAsync(gr->log_scales, 0, (size_t)n * 3 * sizeof(float), s) != cudaSuccess ||
                cudaMemsetAsync(gr->quats, 0, (size_t)n * 4 * sizeof(float), s) != cudaSuccess ||
                cudaMemsetAsync(gr->opacity_logits, 0, (size_t)n * sizeof(float), s) != cudaSuccess ||
                cudaMemsetAsync(gr->sh, 0, (size_t)n * nc * 3 * sizeof(float), s) != cudaSuccess)
                return HTGS_ERR_CUDA;
        }
    }
    // Gradient accumulators and the persistent kernel's work counter.
    if (cudaMemsetAsync(at<char>(workspace, L.bwd_work), 0, L.end - L.bwd_work, s) != cudaSuccess)
        return HTGS_ERR_CUDA;
    ParamArgs pa;
    make_prm(params, pa);
    const int sb = sorted_buffer(L);
    float *acc = at<float>(workspace, L.acc);

    BlendBwdArgs bb{};
    bb.rec = at<float4>(workspace, L.rec);
    bb.vals = at<uint32_t>(workspace, sb ? L.vals1 : L.vals0);
    bb.ranges = at<uint2>(workspace, L.ranges);
    bb.items = at<int4>(workspace, L.items);
    bb.n_items = at<uint32_t>(workspace, L.n_items);
    bb.max_items = L.max_items;
    bb.status = at<int>(workspace, L.status);
    bb.work = at<unsigned int>(workspace, L.bwd_work);
    bb.tiles = L.tiles; bb.prm = pa;
    bb.acc = acc;
    bool want_vis = false;
    for (int v = 0; v < n_views; ++v) want_vis = want_vis || views[v].grads->visibility;
    bb.vis = want_vis ? at<float>(workspace, L.vis) : nullptr;
    mark(launch, 0, s);
    if (L.sorted ? !launch_blend_sorted_bwd(b, bb, s) : !launch_blend_bwd(b, bb, s)) return HTGS_ERR_NOT_SUPPORTED;
    mark(launch, 1, s);
    mark(launch, 2, s);
    if (L.n_blocks > 0) {
        PreBwdArgs pb{};
        pb.prm = pa;
        pb.rec = at<float4>(workspace, L.rec);
        pb.rect = at<uint2>(workspace, L.rect);
        pb.acc = acc;
        pb.vis = bb.vis;
        pb.accumulate = accumulate ? 1 : 0;
        launch_k(preprocess_backward_kernel, L.n_blocks, kPreThreads, 0, s, b, pb);
    }
    mark(launch, 3, s);
    return cudaGetLastError() == cudaSuccess ? HTGS_OK : HTGS_ERR_CUDA;
}

htgs_view single_view(const htgs_gaussians *g, const htgs_camera *cam, float *image, float *saved) {
    htgs_view v;
    memset(&v, 0, sizeof(v));
    v.gaussians = g;
    if (cam) v.camera = *cam;
    v.image = image;
    v.saved = saved;
    return v;
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
    case HTGS_ERR_INTERNAL: return "device-side consistency check failed";
    default: return "unknown status";
    }
}

htgs_status htgs_workspace_size(int64_t n_gaussians, const htgs_camera *cam, const htgs_params *params,
                                const htgs_launch *launch, int64_t instance_capacity, size_t *fwd_bytes,
                                size_t *saved_bytes) {
    if (!camera_ok(cam)) return HTGS_ERR_INVALID_ARG;
    HostView hv{n_gaussians, cam};
    Layout L;
    htgs_status st = make_layout(1, &hv, params, launch, instance_capacity, L);
    if (st) return st;
    if (fwd_bytes) *fwd_bytes = L.end;
    if (saved_bytes) *saved_bytes = (size_t)(7 + params->K) * cam->width * cam->height * sizeof(float);
    return HTGS_OK;
}

htgs_status htgs_batch_workspace_size(int32_t n_views, const htgs_view *views, const htgs_params *params,
                                      const htgs_launch *launch, int64_t instance_capacity,
                                      size_t *workspace_bytes) {
    HostView hv[kMaxViews];
    htgs_status st = collect(n_views, views, hv);
    if (st) return st;
    Layout L;
    st = make_layout(n_views, hv, params, launch, instance_capacity, L);
    if (st) return st;
    if (workspace_bytes) *workspace_bytes = L.end;
    return HTGS_OK;
}

namespace {
void fill_layout(const Layout &L, const htgs_camera *cam, htgs_layout *out) {
    const int sb = sorted_buffer(L);
    out->rec = L.rec;
    out->rect = L.rect;
    out->count = L.count;
    out->sorted_keys = sb ? L.keys1 : L.keys0;
    out->sorted_vals = sb ? L.vals1 : L.vals0;
    out->ranges = L.ranges;
    out->acc = L.acc;
    out->n_tiles = L.tiles.n_tiles;
    out->tiles_x = (cam->width + L.tiles.tile_w - 1) / L.tiles.tile_w;
    out->tiles_y = (cam->height + L.tiles.tile_h - 1) / L.tiles.tile_h;
    out->tile_bits = L.tiles.tile_bits;
    out->items = L.items;
    out->n_items = L.n_items;
    out->partials = L.partials;
    out->max_items = L.max_items;
    out->slots = L.slots_cap;
}
} // namespace

htgs_status htgs_workspace_layout(int64_t n_gaussians, const htgs_camera *cam, const htgs_params *params,
                                  const htgs_launch *launch, int64_t instance_capacity, htgs_layout *out) {
    if (!out || !camera_ok(cam)) return HTGS_ERR_INVALID_ARG;
    HostView hv{n_gaussians, cam};
    Layout L;
    htgs_status st = make_layout(1, &hv, params, launch, instance_capacity, L);
    if (st) return st;
    fill_layout(L, cam, out);
    return HTGS_OK;
}

htgs_status htgs_batch_workspace_layout(int32_t n_views, const htgs_view *views, const htgs_params *params,
                                        const htgs_launch *launch, int64_t instance_capacity, htgs_layout *out) {
    if (!out) return HTGS_ERR_INVALID_ARG;
    HostView hv[kMaxViews];
    htgs_status st = collect(n_views, views, hv);
    if (st) return st;
    Layout L;
    st = make_layout(n_views, hv, params, launch, instance_capacity, L);
    if (st) return st;
    fill_layout(L, &views[0].camera, out);
    return HTGS_OK;
}

htgs_status htgs_render(const htgs_gaussians *g, const htgs_camera *cam, const htgs_params *params,
                        const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                        int64_t instance_capacity, float *saved, float *image, void *stream) {
    if (!camera_ok(cam)) return HTGS_ERR_INVALID_ARG;
    const htgs_view v = single_view(g, cam, image, saved);
    return render_batch(1, &v, params, launch, workspace, workspace_bytes, instance_capacity, stream);
}

htgs_status htgs_render_backward(const htgs_gaussians *g, const htgs_camera *cam,
                                 const htgs_params *params, const htgs_launch *launch, void *workspace,
                                 size_t workspace_bytes, int64_t instance_capacity, const float *saved,
                                 const float *dl_dimage, const htgs_gaussians_grad *grads, void *stream) {
    if (!camera_ok(cam)) return HTGS_ERR_INVALID_ARG;
    htgs_view v = single_view(g, cam, nullptr, const_cast<float *>(saved));
    v.dl_dimage = dl_dimage;
    v.grads = grads;
    return render_batch_backward(1, &v, params, launch, workspace, workspace_bytes, instance_capacity, stream);
}

htgs_status htgs_render_batch(int32_t n_views, const htgs_view *views, const htgs_params *params,
                              const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                              int64_t instance_capacity, void *stream) {
    return render_batch(n_views, views, params, launch, workspace, workspace_bytes, instance_capacity, stream);
}

htgs_status htgs_render_batch_backward(int32_t n_views, const htgs_view *views, const htgs_params *params,
                                       const htgs_launch *launch, void *workspace, size_t workspace_bytes,
                                       int64_t instance_capacity, void *stream) {
    return render_batch_backward(n_views, views, params, launch, workspace, workspace_bytes, instance_capacity,
                                 stream);
}

htgs_status htgs_bake(const htgs_gaussians *g, float *baked, void *stream) {
    if (!g || g->baked || !baked || !aligned16(baked)) return HTGS_ERR_INVALID_ARG;
    htgs_status st = check_gaussians(g);
    if (st) return st;
    if (g->n == 0) return HTGS_OK;
    BakeArgs a;
    a.means = g->means; a.log_scales = g->log_scales; a.quats = g->quats; a.logits = g->opacity_logits;
    a.sh = g->sh; a.filter_var = g->filter_var; a.baked = baked; a.n = g->n; a.sh_degree = g->sh_degree;
    const int64_t blocks = (g->n + kPreThreads - 1) / kPreThreads;
    bake_kernel<<<(unsigned)blocks, kPreThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
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
