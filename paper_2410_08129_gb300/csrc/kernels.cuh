// kernels.cuh -- argument blocks and launch entry points of the kernels
// behind the C ABI. Host code in api.cu is the only caller.
#pragma once

#include "common.cuh"

namespace htgs {

constexpr int kPreThreads = 256;     // preprocess / emit block size
constexpr int kSortThreads = 256;    // onesweep block size
constexpr int kSortItems = 16;       // keys per thread per onesweep block
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 4;

struct PreArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n;
    int sh_degree;
    CamArgs cam;
    ParamArgs prm;
    TileArgs tiles;
    float4 *rec;          // n * 6
    uint2 *rect;          // n: (tx0 | tx1 << 16, ty0 | ty1 << 16)
    uint32_t *count;      // n
    uint32_t *block_sums; // ceil(n / kPreThreads)
    unsigned long long *stats;
};

struct PreBwdArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n;
    int sh_degree;
    CamArgs cam;
    ParamArgs prm;
    const float4 *rec;
    const uint2 *rect;
    const float *acc;     // n * 16
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
};

struct BinArgs {
    int64_t n;
    int n_blocks;               // ceil(n / kPreThreads)
    const uint2 *rect;
    const uint32_t *count;
    uint32_t *block_sums;       // in: per-block sums; out: exclusive block offsets
    int *status;
    int64_t capacity;
    TileArgs tiles;
    uint32_t *keys, *vals;      // emit targets
    uint32_t *total;            // device copy of the instance count (clamped use)
};

struct SortArgs {
    int64_t capacity;
    const uint32_t *total;
    int passes;
    uint32_t *keys[2], *vals[2];
    uint32_t *ghist;            // kMaxPasses * kRadix
    uint32_t *lookback;         // passes * n_sort_blocks * kRadix
    uint32_t *tickets;          // kMaxPasses
    int n_sort_blocks;
    int *status;
};

struct RangeArgs {
    const uint32_t *total;
    const uint32_t *keys;
    int shift;                  // key >> shift = tile id
    uint2 *ranges;              // n_tiles
    int64_t capacity;
    int n_tiles;
};

struct BlendFwdArgs {
    const float4 *rec;
    const uint32_t *vals;       // sorted gids
    const uint2 *ranges;
    const int *status;
    TileArgs tiles;
    ParamArgs prm;
    int width, height;
    float *image;               // H x W x 3
    float *saved;               // (7 + K) planes of H*W, or nullptr
    unsigned long long *stats;
};

struct BlendBwdArgs {
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *ranges;
    const int *status;
    TileArgs tiles;
    ParamArgs prm;
    int width, height;
    const float *saved;
    const float *dl_dimg;
    float *acc;                 // n * 16
    int64_t n;                  // Gaussians (bounds the saved core ids)
};

__global__ void preprocess_kernel(PreArgs a);
__global__ void preprocess_backward_kernel(PreBwdArgs a);

// Binning: scan of per-block sums, then emit (tile key, gid) instances.
void launch_scan_blocks(const BinArgs &a, cudaStream_t s);
void launch_emit(const BinArgs &a, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by the low `passes * 8` bits.
// Returns the buffer index (0 or 1) holding the result.
int launch_sort(const SortArgs &a, cudaStream_t s);
void launch_ranges(RangeArgs a, int n_tiles, cudaStream_t s);

// Blend kernels; return false when (K, tile shape, px/thread) has no instance.
bool launch_blend_fwd(const BlendFwdArgs &a, int px_per_thread, cudaStream_t s);
bool launch_blend_bwd(const BlendBwdArgs &a, int px_per_thread, cudaStream_t s);

} // namespace htgs
