// tilesort.cu -- tile binning of a single view as one stable counting sort
// by tile id (arXiv 2410.08129, Sec. 4.3: one instance per covered
// (Gaussian, tile), keyed by the tile id only; no global depth sort).
//
// The instances of a record are the tiles of its cover (per tile row of its
// rectangle, the span its cutoff ellipse reaches), so no (key, value) list is
// materialised: positions are computed from the covers.
// Emission positions (records, or their mean-depth order for sorted
// blending) are cut into blocks of `gauss` consecutive positions, and the
// tile rows into bands of at most kCsBandTiles tiles. A CTA works on one
// (block, band) pair and sees only the rows of each cover inside its band.
//
//   cs_count    per (block, band): how many of the block's records cover each
//               tile of the band (shared-memory atomics), written to a row of
//               uint16 counts per block
//   cs_colscan  per tile: exclusive prefix of those counts over the blocks and
//               the tile's total
//   (schedule)  one CTA scans the tile totals into [start, end) ranges and the
//               instance total, checks the capacity and builds the blend work
//               items (binning.cu)
//   cs_emit     per (block, band): each of the kCsWarps warps takes a slice of
//               the block's positions, counts its instances per tile in a
//               16-bit counter of its own, the counters are prefixed across
//               warps per tile, and each warp walks its instances again in
//               emission order, 32 at a time; instances of one tile within
//               such a chunk are ranked by __match_any_sync in lane order. The
//               record id lands at
//               start[t] + earlier blocks + earlier warps + earlier chunks + rank,
//               so every tile's list keeps emission order: the lists a stable
//               radix sort of (tile, record) keys gives, in four launches and
//               one write per instance.
#include "common.cuh"
#include "kernels.cuh"

namespace htgs {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One emission position, restricted to the band: its cover and the cover's
// rows [lo, hi] inside the band (lo > hi: none), and its record.
struct PosInfo {
    uint32_t lo, hi, rec;
    RowCover cov;
};

__device__ __forceinline__ PosInfo band_part(const CsArgs &a, uint32_t count, uint2 r, uint32_t rec, int band_r0,
                                             int band_r1) {
    PosInfo q;
    q.lo = 1u; q.hi = 0u; q.rec = rec;
    q.cov = row_cover(make_uint2(1u, 0u), 0.f, 0.f, 0.f, 0.f, 0.f, false);
    if (count) {
        const int ty0 = (int)(r.y & 0xffffu), ty1 = (int)(r.y >> 16);
        const int lo = max(ty0, band_r0), hi = min(ty1, band_r1 - 1);
        if (lo <= hi) {
            q.cov = load_cover(a.cover, rec, a.use_ellipse != 0);
            q.lo = (uint32_t)lo;
            q.hi = (uint32_t)hi;
        }
    }
    return q;
}

// The warp's positions [first, first + per_warp), kCsUnroll steps of 32 at a
// time: the counts and rectangles of all of them are loaded first (their
// loads are independent, so their latencies overlap), then fn(q) runs for
// each step in order with the band part of the lane's position.
constexpr int kCsUnroll = 4;

template <class Fn>
__device__ __forceinline__ void for_warp_positions(const CsArgs &a, long long first, int per_warp, int lane,
                                                   int band_r0, int band_r1, Fn &&fn) {
    for (int s0 = 0; s0 < per_warp && first + s0 < a.n; s0 += 32 * kCsUnroll) {
        uint32_t cnt[kCsUnroll], rec[kCsUnroll];
        uint2 rct[kCsUnroll];
#pragma unroll
        for (int u = 0; u < kCsUnroll; ++u) {
            const long long p = first + s0 + 32 * u + lane;
            const bool ok = s0 + 32 * u < per_warp && p < a.n;
            rec[u] = ok ? (a.perm ? a.perm[p] : (uint32_t)p) : 0u;
            cnt[u] = ok ? a.count[p] : 0u;
        }
        // (A record that covers no tile may hold any rectangle: it is not used.)
#pragma unroll
        for (int u = 0; u < kCsUnroll; ++u) rct[u] = a.rect[rec[u]];
#pragma unroll
        for (int u = 0; u < kCsUnroll; ++u) {
            if (s0 + 32 * u < per_warp && first + s0 + 32 * u < a.n)
                fn(band_part(a, cnt[u], rct[u], rec[u], band_r0, band_r1));
        }
    }
}

// Calls f(valid, band_tile, record) for the band instances of the warp's 32
// positions (one per lane, in lane order), 32 instances per call, in emission
// order: position by position, each position's tiles row by row. Every lane
// makes the same number of calls (padding slots with valid = false).
template <class F>
__device__ __forceinline__ void warp_instances(const CsArgs &a, const PosInfo &q, int lane, int band_r0, F &&f) {
    if (__ballot_sync(kFull, q.lo <= q.hi) == 0) return;  // no row of these positions in the band
    warp_cover_instances(q.cov, q.lo, q.hi, lane, a.tile_w, a.tile_h,
                         [&](bool valid, uint32_t, uint32_t ty, uint32_t tx, uint32_t owner) {
                             const uint32_t rec = __shfl_sync(kFull, q.rec, (int)owner);
                             f(valid, (ty - (uint32_t)band_r0) * (uint32_t)a.tiles_x + tx, rec);
                         });
}

struct Band {
    int r0, r1;  // tile rows [r0, r1)
    int t0, nt;  // first tile, tiles in the band
};

__device__ __forceinline__ Band band_of(const CsArgs &a, int s) {
    Band B;
    B.r0 = s * a.band_rows;
    B.r1 = min(a.tiles_y, B.r0 + a.band_rows);
    B.t0 = B.r0 * a.tiles_x;
    B.nt = (B.r1 - B.r0) * a.tiles_x;
    return B;
}

__global__ void __launch_bounds__(kCsThreads) cs_count_kernel(CsArgs a) {
    dependent_entry();
    __shared__ uint32_t s_hist[kCsBandTiles];
    const Band B = band_of(a, blockIdx.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < B.nt; t += kCsThreads) s_hist[t] = 0;
    __syncthreads();
    const int per_warp = a.gauss / kCsWarps;
    const long long first = (long long)blockIdx.x * a.gauss + (long long)warp * per_warp;
    for_warp_positions(a, first, per_warp, lane, B.r0, B.r1, [&](const PosInfo &q) {
        warp_instances(a, q, lane, B.r0, [&](bool valid, uint32_t tile, uint32_t) {
            if (valid && tile < (uint32_t)B.nt) atomicAdd(&s_hist[tile], 1u);
        });
    });
    __syncthreads();
    uint16_t *row = a.hist + (size_t)blockIdx.x * a.n_tiles + B.t0;
    for (int t = threadIdx.x; t < B.nt; t += kCsThreads) row[t] = (uint16_t)s_hist[t];
}

// Column scan: CTA c owns tiles [32 c, 32 c + 32); warp g of kColGroups
// scans rows [g R, g R + R) with R = ceil(nb / kColGroups).
constexpr int kColGroups = 8;

__global__ void __launch_bounds__(32 * kColGroups) cs_colscan_kernel(CsArgs a) {
    dependent_entry();
    __shared__ uint32_t s_part[kColGroups][32];
    const int T = a.n_tiles, nb = a.nb;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + lane;
    const int R = (nb + kColGroups - 1) / kColGroups;
    const int r0 = g * R, r1 = min(nb, r0 + R);
    uint32_t sum = 0;
    if (t < T) {
#pragma unroll 4
        for (int r = r0; r < r1; ++r) sum += a.hist[(size_t)r * T + t];
    }
    s_part[g][lane] = sum;
    __syncthreads();
    uint32_t run = 0;
    for (int k = 0; k < g; ++k) run += s_part[k][lane];
    if (g == kColGroups - 1 && t < T) a.tile_tot[t] = run + sum;
    if (t < T) {
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
            const size_t i = (size_t)r * T + t;
            const uint32_t v = a.hist[i];
            a.off[i] = run;
            run += v;
        }
    }
}

__global__ void __launch_bounds__(kCsThreads) cs_emit_kernel(CsArgs a) {
    dependent_entry();
    // s_base[t]: global position of this block's first instance of band tile t.
    // s_wc[h][t]: 16-bit counters of warps 2h (low half) and 2h + 1 (high
    // half): first the warp's count of tile t, then its running position
    // within the block's part of the tile.
    __shared__ uint32_t s_base[kCsBandTiles];
    __shared__ uint32_t s_wc[kCsWarps / 2][kCsBandTiles];
    if (a.status[kStError] != 0) return;  // overflow (or an earlier failure): nothing to place
    const Band B = band_of(a, blockIdx.y);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < B.nt; t += kCsThreads) {
#pragma unroll
        for (int h = 0; h < kCsWarps / 2; ++h) s_wc[h][t] = 0;
    }
    __syncthreads();
    const int per_warp = a.gauss / kCsWarps;
    const long long first = (long long)blockIdx.x * a.gauss + (long long)warp * per_warp;
    uint32_t *const wc = s_wc[warp >> 1];
    const uint32_t shift = (warp & 1) ? 16u : 0u;
    for_warp_positions(a, first, per_warp, lane, B.r0, B.r1, [&](const PosInfo &q) {
        warp_instances(a, q, lane, B.r0, [&](bool valid, uint32_t tile, uint32_t) {
            if (valid && tile < (uint32_t)B.nt) atomicAdd(&wc[tile], 1u << shift);
        });
    });
    __syncthreads();
    // Per tile: exclusive prefix of the warps' counts, in warp order.
    const uint32_t *off_row = a.off + (size_t)blockIdx.x * a.n_tiles + B.t0;
    for (int t = threadIdx.x; t < B.nt; t += kCsThreads) {
        uint32_t run = 0, any = 0;
#pragma unroll
        for (int h = 0; h < kCsWarps / 2; ++h) {
            const uint32_t v = s_wc[h][t];
            any |= v;
            const uint32_t lo = v & 0xffffu, hi = v >> 16;
            s_wc[h][t] = run | ((run + lo) << 16);
            run += lo + hi;
        }
        if (any) s_base[t] = a.ranges[B.t0 + t].x + off_row[t];
    }
    __syncthreads();
    const uint32_t cap = a.capacity < 0xffffffffll ? (uint32_t)a.capacity : 0xffffffffu;
    for_warp_positions(a, first, per_warp, lane, B.r0, B.r1, [&](const PosInfo &q) {
        warp_instances(a, q, lane, B.r0, [&](bool valid, uint32_t tile, uint32_t rec) {
            const bool ok = valid && tile < (uint32_t)B.nt;
            const uint32_t vmask = __ballot_sync(kFull, ok);
            if (ok) {
                const uint32_t peers = __match_any_sync(vmask, tile);
                const uint32_t below = peers & lanemask_lt();
                const uint32_t cur = (wc[tile] >> shift) & 0xffffu;
                const uint32_t pos = s_base[tile] + cur + (uint32_t)__popc(below);
                if (pos < cap) a.vals[pos] = rec;
                __syncwarp(vmask);
                if (below == 0) atomicAdd(&wc[tile], (uint32_t)__popc(peers) << shift);
            }
            __syncwarp();
        });
    });
}

}  // namespace

bool cs_plan(int n_views, int tiles_x, int tiles_y, long long n, CsPlan &p) {
    if (n_views != 1 || tiles_x <= 0 || tiles_y <= 0 || tiles_x > kCsBandTiles || n <= 0) return false;
    // Rows per band: what fits kCsBandTiles, at most a quarter of the rows
    // (at least four bands where the image has the rows for them).
    p.band_rows = kCsBandTiles / tiles_x;
    if (p.band_rows > (tiles_y + 3) / 4) p.band_rows = (tiles_y + 3) / 4;
    p.n_bands = (tiles_y + p.band_rows - 1) / p.band_rows;
    // The largest block (the fewer blocks, the smaller the count matrix)
    // that still gives about four (block, band) CTAs per SM of a 152-SM GPU.
    p.gauss = kCsMinGauss;
    for (int g = kCsMaxGauss; g > kCsMinGauss; g >>= 1)
        if ((long long)((n + g - 1) / g) * p.n_bands >= 600) {
            p.gauss = g;
            break;
        }
    p.nb = (int)((n + p.gauss - 1) / p.gauss);
    return true;
}

void launch_cs_count(const CsArgs &a, cudaStream_t s) {
    if (a.nb > 0) launch_k(cs_count_kernel, dim3(a.nb, a.n_bands), kCsThreads, 0, s, a);
}

void launch_cs_colscan(const CsArgs &a, cudaStream_t s) {
    launch_k(cs_colscan_kernel, (a.n_tiles + 31) / 32, 32 * kColGroups, 0, s, a);
}

void launch_cs_emit(const CsArgs &a, cudaStream_t s) {
    if (a.nb > 0) launch_k(cs_emit_kernel, dim3(a.nb, a.n_bands), kCsThreads, 0, s, a);
}

}  // namespace htgs
