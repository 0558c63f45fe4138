// kernels.cuh -- argument blocks and launch entry points of the kernels
// behind the C ABI. Host code in api.cu is the only caller.
//
// Every render is a batch of views (a single-view render is a batch of one).
// A view has its own camera, the scene it renders (several views may share
// one scene) and its outputs. Records are indexed per (view, Gaussian): view
// v owns records [rec_off, rec_off + n); tiles are numbered globally: view v
// owns tiles [tile_off, tile_off + tiles_x * tiles_y).
#pragma once

#include "common.cuh"

namespace htgs {

constexpr int kPreThreads = 256;     // preprocess / emit block size
constexpr int kSortThreads = 256;    // onesweep block size
constexpr int kSortItems = 16;       // keys per thread per onesweep block
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxRadixBits = 9;     // widest digit: keys of up to 18 bits sort in two passes
constexpr int kMaxRadix = 1 << kMaxRadixBits;
constexpr int kMaxPasses = 4;
constexpr int kMaxViews = HTGS_MAX_VIEWS;

// Blend work items. A tile whose instance list is longer than the chunk size
// C = max(kMinChunk, ceil(total / kChunkDiv)) is cut into m = ceil(count / C)
// contiguous chunks processed by different CTAs; the forward's chunks leave
// mergeable partial states in one of at most kMaxSlots slots. Items are
// ordered by decreasing chunk length so that the long ones start first.
constexpr uint32_t kMinChunk = 1024;
constexpr uint32_t kChunkDiv = 2048;
constexpr int kMaxSlots = 4096;
constexpr int kSchedThreads = 1024;
constexpr int kSchedBuckets = 64;

struct ViewDesc {
    CamArgs cam;
    const float *means, *log_scales, *quats, *logits, *sh;
    const float *filter_var;  // nullptr: no 3D filter
    const float *baked;       // nullptr, or the baked records (then means .. filter_var are not read)
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
    float *g_vis, *g_dgrad, *g_dcount;  // optional training statistics
    float *image;          // H x W x 3
    float *saved;          // (7 + K) planes of H*W, or nullptr
    const float *dl_dimg;  // H x W x 3 (backward)
    long long n;           // Gaussians of the scene
    long long rec_off;     // first record of this view
    int sh_degree;
    int tile_off;          // first global tile of this view
    int tiles_x, tiles_y;
};

// Passed by value (as a __grid_constant__ kernel parameter).
struct Batch {
    int n_views;
    int total_tiles;
    long long n_rec;
    ViewDesc v[kMaxViews];
};
static_assert(sizeof(Batch) <= 32764, "kernel parameter limit");

// View owning record i (records are grouped by view in increasing order).
__device__ __forceinline__ int view_of_record(const Batch &b, long long i) {
    int lo = 0, hi = b.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.v[mid].rec_off <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// View owning global tile t.
__device__ __forceinline__ int view_of_tile(const Batch &b, int t) {
    int lo = 0, hi = b.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.v[mid].tile_off <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct PreArgs {
    ParamArgs prm;
    TileArgs tiles;        // tile shape (counts per view are in the batch)
    uint32_t *dkey;        // sorted blending: n_rec mean-depth keys (float bits), or nullptr
    uint32_t *dval;        // sorted blending: n_rec record indices
    uint32_t *dtotal;      // sorted blending: receives n_rec (the depth sort's length)
    float4 *rec;           // n_rec * kRecF4
    uint2 *rect;           // n_rec: (tx0 | tx1 << 16, ty0 | ty1 << 16), view-local tiles
    uint4 *cover;          // n_rec * 2: the record's cover (see CoverRec)
    uint32_t *count;       // n_rec
    uint32_t *block_sums;  // ceil(n_rec / kPreThreads)
    unsigned long long *stats;
};

struct PreBwdArgs {
    ParamArgs prm;
    const float4 *rec;
    const uint2 *rect;
    const float *acc;      // n_rec * 16
    const float *vis;      // n_rec: largest blending weight of each record, or nullptr
    int accumulate;        // 1: several views share a scene, add into the gradients atomically
};

struct BinArgs {
    long long n;           // records
    int n_blocks;          // ceil(n / kPreThreads)
    const uint32_t *perm;  // emission order of the records (position -> record), or nullptr
    const uint2 *rect;
    const uint4 *cover;    // per record: its cover (see CoverRec)
    int tile_w, tile_h, use_ellipse;  // tile shape; TileArgs::cover == 0
    const uint32_t *count; // per position (permuted when perm is set)
    uint32_t *block_sums;  // in: per-block sums; out: exclusive block offsets
    int *status;
    int64_t capacity;
    uint32_t *keys, *vals; // emit targets: global tile id, record index
    uint32_t *total;       // device copy of the instance count (0 on overflow)
};

struct SortArgs {
    int64_t capacity;
    const uint32_t *total;
    int passes;
    int digit_bits;        // bits per pass (every pass the same), at most kMaxRadixBits
    uint32_t *keys[2], *vals[2];
    uint32_t *ghist;       // kMaxPasses * kMaxRadix
    unsigned long long *lookback;  // passes * n_sort_blocks * 2^digit_bits flag|count words
    uint32_t *tickets;     // kMaxPasses
    int n_sort_blocks;
    int *status;
    int stall_first;       // 1 only to test the bounded wait: pass 0's first block waits on a word nothing writes
};

struct RangeArgs {
    const uint32_t *total;
    const uint32_t *keys;
    uint2 *ranges;         // total_tiles
    int n_tiles;
};

// Work item: (global tile, chunk k of m, first partial-state slot of the tile).
struct ScheduleArgs {
    const uint32_t *total;
    const uint2 *ranges;
    int n_tiles;
    int no_split;          // 1: one item per tile (sorted blending)
    int slots_cap;         // partial-state slots available
    int4 *items;           // n_tiles + slots_cap
    uint32_t *n_items;
    int *status;           // a recorded failure (overflow, a wait that gave up): no items
    // Counting-sort binning: the per-tile instance counts. When set, the
    // kernel first writes ranges_out (exclusive scan of the counts) and
    // total_out (the instance total, 0 on overflow), checks the capacity and
    // records the total in the status slots.
    const uint32_t *tile_tot;
    uint2 *ranges_out;
    uint32_t *total_out;
    int64_t capacity;
};

// Counting-sort binning of a single view (tilesort.cu): blocks of `gauss`
// emission positions (kCsMinGauss .. kCsMaxGauss, so that per-block tile
// counts fit 16 bits), bands of whole tile rows of at most kCsBandTiles tiles.
constexpr int kCsWarps = 8;
constexpr int kCsThreads = 32 * kCsWarps;
constexpr int kCsBandTiles = 2048;   // shared memory: 5 x 4 B per band tile in cs_emit
constexpr int kCsMinGauss = 2048;
constexpr int kCsMaxGauss = 16384;
struct CsPlan {
    int band_rows, n_bands, gauss, nb;
};
struct CsArgs {
    long long n;           // emission positions (records)
    int nb, gauss;         // blocks of `gauss` positions
    int n_tiles, tiles_x, tiles_y;
    int band_rows, n_bands;
    const uint32_t *perm;  // position -> record, or nullptr
    const uint2 *rect;     // per record: (tx0 | tx1 << 16, ty0 | ty1 << 16), view-local tiles
    const uint4 *cover;    // per record: its cover (see CoverRec)
    int tile_w, tile_h, use_ellipse;  // tile shape; TileArgs::cover == 0
    const uint32_t *count; // per position: tiles covered
    uint16_t *hist;        // nb x n_tiles: instances of each tile in each block
    uint32_t *off;         // nb x n_tiles: instances of the tile in earlier blocks
    uint32_t *tile_tot;    // n_tiles
    const uint2 *ranges;   // n_tiles: [start, end) (written by the schedule kernel)
    uint32_t *vals;        // capacity: record ids in tile order
    int *status;
    int64_t capacity;
};

// A work item names an existing tile and a chunk k < m whose slots fit.
__device__ __forceinline__ bool item_ok(int4 w, int n_tiles, int slots) {
    return w.x >= 0 && w.x < n_tiles && w.z >= 1 && w.y >= 0 && w.y < w.z &&
           (w.z == 1 || (w.w >= 0 && w.w + w.z <= slots));
}

// Instance range [start, end) of chunk k of m of a tile's list.
__device__ __forceinline__ uint2 chunk_range(uint2 r, int k, int m) {
    if (m <= 1) return r;
    const uint32_t per = (r.y - r.x + (uint32_t)m - 1) / (uint32_t)m;
    const uint32_t a = min(r.x + (uint32_t)k * per, r.y);
    return make_uint2(a, min(a + per, r.y));
}

struct BlendFwdArgs {
    const float4 *rec;
    const uint32_t *vals;  // sorted record indices
    const uint2 *ranges;
    const int4 *items;
    const uint32_t *n_items;
    float *partials;       // slots * (6 + 2K) * tile pixels
    unsigned int *done;    // per split tile (at its first slot): chunks finished
    int max_items;         // bound on the item count (grid size cap)
    int slots;             // partial-state slots
    const int *status;
    unsigned int *work;    // persistent-kernel work counter (zeroed per render)
    TileArgs tiles;
    ParamArgs prm;
    unsigned long long *stats;
};

struct BlendBwdArgs {
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    const int4 *items;
    const uint32_t *n_items;
    int max_items;
    const int *status;
    unsigned int *work;
    TileArgs tiles;
    ParamArgs prm;
    float *acc;            // n_rec * 16
    float *vis;            // n_rec (largest blending weight, as int bits), or nullptr
};

// Baking of one scene (raw parameters in, HTGS_BAKED_FLOATS records out).
struct BakeArgs {
    const float *means, *log_scales, *quats, *logits, *sh, *filter_var;
    float *baked;
    long long n;
    int sh_degree;
};
__global__ void bake_kernel(BakeArgs a);
// The forward setup of every record; any_baked: some view renders baked records.
void launch_preprocess(bool any_baked, int blocks, const Batch &b, const PreArgs &a, cudaStream_t s);
__global__ void preprocess_backward_kernel(const __grid_constant__ Batch b, PreBwdArgs a);

// Binning: scan of per-block sums, then emit (global tile, record) instances.
void launch_scan_blocks(const BinArgs &a, cudaStream_t s);
void launch_emit(const Batch &b, const BinArgs &a, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by the low passes * digit_bits bits.
// Returns the buffer index (0 or 1) holding the result.
int launch_sort(const SortArgs &a, cudaStream_t s);
void launch_ranges(RangeArgs a, cudaStream_t s);
// Counts in the order perm gives and their per-block sums (for the scan).
void launch_permute_counts(long long n, const uint32_t *perm, const uint32_t *count, uint32_t *count_p,
                           uint32_t *block_sums, cudaStream_t s);
// Blend work items from the tile ranges (one CTA).
void launch_schedule(const ScheduleArgs &a, cudaStream_t s);
// Band and block sizes of the counting sort; false where it does not apply
// (several views, or a tile row longer than a band).
bool cs_plan(int n_views, int tiles_x, int tiles_y, long long n, CsPlan &p);
void launch_cs_count(const CsArgs &a, cudaStream_t s);
void launch_cs_colscan(const CsArgs &a, cudaStream_t s);
void launch_cs_emit(const CsArgs &a, cudaStream_t s);

// Persistent blend kernels over the batch's (view, tile) items; return false
// when (K, tile shape, px/thread) has no compiled instance.
bool launch_blend_fwd(const Batch &b, const BlendFwdArgs &a, int px_per_thread, cudaStream_t s);
bool launch_blend_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s);
// The same for mean-depth-sorted blending (one item per tile).
bool launch_blend_sorted_fwd(const Batch &b, const BlendFwdArgs &a, cudaStream_t s);
bool launch_blend_sorted_bwd(const Batch &b, const BlendBwdArgs &a, cudaStream_t s);

// Programmatic dependent launch for the kernels of one render call: while
// it is on (set_dependent_launch, per host thread), launch_k starts each
// kernel with cudaLaunchAttributeProgrammaticStreamSerialization, so that
// its CTAs may become resident while the previous kernel's last CTAs run;
// every kernel begins with dependent_entry(), which waits for the previous
// kernel to complete before touching memory. Off, launch_k is a plain launch.
void set_dependent_launch(bool on);
bool dependent_launch();

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
    if (!dependent_launch()) {
        kernel<<<grid, block, smem, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// CTAs per SM the persistent kernels are launched with (occupancy query).
int persistent_grid(const void *kernel, int threads, size_t dyn_smem, int items);
// Raises a kernel's dynamic shared-memory limit to `bytes` (once per device).
bool allow_dynamic_smem(const void *kernel, size_t bytes);

} // namespace htgs
