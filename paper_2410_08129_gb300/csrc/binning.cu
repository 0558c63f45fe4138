// binning.cu -- tile binning and sorting (arXiv 2410.08129, Sec. 4.3: one
// instance per covered (Gaussian, tile) keyed by the tile id, with no global
// depth sort).
//
//   scan_blocks  exclusive scan of the preprocess block sums; overflow check
//   emit         (tile key, gid) for each tile a Gaussian covers (per tile row
//                of its rectangle, the span its cutoff ellipse reaches),
//                load-balanced across the lanes of a warp
//   histogram    digit histograms of every radix pass in one read of the keys
//   onesweep     one stable scatter per digit (the key bits split evenly into
//                the fewest passes of at most 9 bits); the block prefix comes
//                from a decoupled look-back whose waits are bounded, and each
//                block orders its items by digit in shared memory first so
//                that its stores are runs of consecutive addresses
//   ranges       [start, end) of every tile in the sorted keys
#include <mutex>
#include <set>
#include <utility>

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

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Exclusive scan of the per-block instance counts (one CTA).
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(BinArgs a) {
    dependent_entry();
    __shared__ uint64_t warp_tot[kScanThreads / 32];
    const int nb = a.n_blocks;
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per;
    uint64_t local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) local += a.block_sums[b0 + k];
    // Block-wide exclusive scan of `local`.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t v = warp_tot[lane];
        uint64_t vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(kFull, vi, o);
            if (lane >= o) vi += t;
        }
        warp_tot[lane] = vi - v;
    }
    __syncthreads();
    uint64_t run = warp_tot[warp] + incl - local;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) {
            uint32_t c = a.block_sums[b0 + k];
            a.block_sums[b0 + k] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
            run += c;
        }
    if (threadIdx.x == kScanThreads - 1) {
        const uint64_t total = run;
        a.status[kStInstLo] = (int)(uint32_t)(total & 0xffffffffull);
        a.status[kStInstHi] = (int)(uint32_t)(total >> 32);
        if (total > (uint64_t)a.capacity) {
            set_error(a.status, HTGS_ERR_OVERFLOW);
            a.total[0] = 0;
        } else {
            a.total[0] = (uint32_t)total;
        }
    }
}

// ---------------------------------------------------------------------------
// Emit: the instances of a Gaussian are its cover's tiles, row by row.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPreThreads) emit_kernel(const __grid_constant__ Batch b, BinArgs a) {
    dependent_entry();
    __shared__ uint32_t warp_tot[kPreThreads / 32];
    if (a.status[kStError] == HTGS_ERR_OVERFLOW) return;
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t c = i < a.n ? a.count[i] : 0u;
    // The record emitted at position i (the identity unless an order is given).
    const uint32_t rec = i < a.n ? (a.perm ? a.perm[i] : (uint32_t)i) : 0u;
    // The record's view: its tile numbering (row length and first global tile).
    uint32_t vtx = 0, vtoff = 0;
    if (c) {
        const ViewDesc &V = b.v[view_of_record(b, rec)];
        vtx = (uint32_t)V.tiles_x;
        vtoff = (uint32_t)V.tile_off;
    }
    uint32_t wtot;
    warp_excl_scan(c, lane, &wtot);
    if (lane == 0) warp_tot[warp] = wtot;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += warp_tot[w];
    const uint64_t base = (uint64_t)a.block_sums[blockIdx.x] + woff;
    // The lane's own cover (only read for a record that emits something).
    const RowCover cov = c ? load_cover(a.cover, rec, a.use_ellipse != 0)
                           : row_cover(make_uint2(1u, 0u), 0.f, 0.f, 0.f, 0.f, 0.f, false);
    const uint32_t lo = c ? cov.ty0 : 1u, hi = c ? cov.ty1 : 0u;
    const uint64_t cap = (uint64_t)a.capacity;
    // The warp deals out its (record, row) pairs 32 at a time; each lane
    // writes the span of its row (rows are a few tiles wide, so the lanes
    // stay nearly in step and neighbouring lanes write neighbouring slots).
    uint32_t run = 0;
    warp_cover_rows(cov, lo, hi, lane, a.tile_w, a.tile_h,
                    [&](bool, uint32_t owner, uint32_t row, uint32_t s0, uint32_t w) {
                        uint32_t tot;
                        const uint32_t off = run + warp_excl_scan(w, lane, &tot);
                        const uint32_t ltx = __shfl_sync(kFull, vtx, (int)owner);
                        const uint32_t ltoff = __shfl_sync(kFull, vtoff, (int)owner);
                        const uint32_t lrec = __shfl_sync(kFull, rec, (int)owner);
                        const uint32_t key0 = ltoff + row * ltx + s0;
                        for (uint32_t t = 0; t < w; ++t) {
                            // (off + t < wtot: never past this warp's share of the list.)
                            const uint64_t pos = base + off + t;
                            if (off + t < wtot && pos < cap) {
                                a.keys[pos] = key0 + t;
                                a.vals[pos] = lrec;
                            }
                        }
                        run += tot;
                    });
    // The spans are the ones the preprocess counted (same steps, same
    // inputs); a mismatch would leave slots unwritten, so it is reported
    // and the blend is skipped.
    if (lane == 0 && run != wtot) set_error(a.status, HTGS_ERR_INTERNAL);
}

// ---------------------------------------------------------------------------
// Radix sort: digit histograms for all passes in one read.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) histogram_kernel(SortArgs a) {
    dependent_entry();
    __shared__ uint32_t h[kMaxPasses * kMaxRadix];
    const int R = 1 << a.digit_bits;
    for (int k = threadIdx.x; k < a.passes * kMaxRadix; k += kSortThreads) h[k] = 0;
    __syncthreads();
    const uint32_t total = *a.total;
    const uint32_t *keys = a.keys[0];
    // Eight consecutive keys per thread (two 16-byte loads; the key array is
    // 16-byte aligned), loaded before any of their counts is added.
    const uint32_t step = gridDim.x * kSortThreads * 8;
    for (uint32_t i0 = (blockIdx.x * kSortThreads + threadIdx.x) * 8; i0 < total; i0 += step) {
        uint32_t k[8];
        if (i0 + 8 <= total) {
            const uint4 lo = *reinterpret_cast<const uint4 *>(keys + i0);
            const uint4 hi = *reinterpret_cast<const uint4 *>(keys + i0 + 4);
            k[0] = lo.x; k[1] = lo.y; k[2] = lo.z; k[3] = lo.w;
            k[4] = hi.x; k[5] = hi.y; k[6] = hi.z; k[7] = hi.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) k[j] = i0 + j < total ? keys[i0 + j] : 0u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (i0 + j >= total) break;
            for (int p = 0; p < a.passes; ++p)
                atomicAdd(&h[p * kMaxRadix + ((k[j] >> (p * a.digit_bits)) & (uint32_t)(R - 1))], 1u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < a.passes * kMaxRadix; k += kSortThreads)
        if (h[k]) atomicAdd(&a.ghist[k], h[k]);
}

// ---------------------------------------------------------------------------
// One stable scatter pass. Blocks take tickets in launch order so that every
// block they wait on is already resident; waits are bounded.
// ---------------------------------------------------------------------------
// Look-back word: status in the top two bits, digit count below (64-bit so
// that counts up to the 2^31 - 1 instance limit fit beside the flags).
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kCountMask = (1ull << 62) - 1;
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint32_t kSpinLimit = 1u << 22;

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(SortArgs a, int pass, int src) {
    dependent_entry();
    // s_whist (per-warp digit counts, then their prefixes) and s_k (the block's
    // keys in digit order) are alive at different times and share storage.
    __shared__ uint32_t s_kw[kSortTile > kSortWarps * kMaxRadix ? kSortTile : kSortWarps * kMaxRadix];
    __shared__ uint32_t s_v[kSortTile];
    __shared__ uint32_t s_base[kMaxRadix];    // global position of the block's first item of each digit
    __shared__ uint32_t s_scan[kMaxRadix];    // global exclusive digit offsets
    __shared__ uint32_t s_cnt[kMaxRadix];     // block digit counts
    __shared__ uint32_t s_bstart[kMaxRadix];  // block-local exclusive digit offsets
    __shared__ uint32_t s_wsum[kSortWarps];
    __shared__ int s_ticket;
    uint32_t(*s_whist)[kMaxRadix] = reinterpret_cast<uint32_t(*)[kMaxRadix]>(s_kw);
    uint32_t *s_k = s_kw;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int R = 1 << a.digit_bits;  // digits of this sort: 2 .. kMaxRadix
    const uint32_t total = *a.total;
    const uint32_t used = (total + kSortTile - 1) / kSortTile;
    const int shift = pass * a.digit_bits;
    const uint32_t dmask = (uint32_t)(R - 1);
    const uint32_t *kin = a.keys[src], *vin = a.vals[src];
    uint32_t *kout = a.keys[src ^ 1], *vout = a.vals[src ^ 1];
    constexpr int kPerMax = kMaxRadix / kSortThreads;
    const int per = (R + kSortThreads - 1) / kSortThreads;

    // Exclusive scan of in[0, R) into out[0, R); thread tid owns digits
    // [tid * per, tid * per + per). Block-wide (uses s_wsum).
    auto block_scan = [&](const uint32_t *in, uint32_t *out) {
        const int d0 = tid * per;
        uint32_t v[kPerMax], loc = 0;
#pragma unroll
        for (int i = 0; i < kPerMax; ++i) {
            v[i] = (i < per && d0 + i < R) ? in[d0 + i] : 0u;
            loc += v[i];
        }
        uint32_t incl = loc;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t off = incl - loc;
        for (int w = 0; w < warp; ++w) off += s_wsum[w];
#pragma unroll
        for (int i = 0; i < kPerMax; ++i) {
            if (i < per && d0 + i < R) out[d0 + i] = off;
            off += v[i];
        }
        __syncthreads();
    };
    block_scan(a.ghist + pass * kMaxRadix, s_scan);

    // Persistent: the block sorts tiles of kSortTile keys in ticket order
    // until every tile is taken (a tile's look-back waits only on smaller
    // tickets, which blocks already running hold).
    for (;;) {
    if (tid == 0) s_ticket = (int)atomicAdd(&a.tickets[pass], 1u);
    for (int k = tid; k < kSortWarps * kMaxRadix; k += kSortThreads) (&s_whist[0][0])[k] = 0;
    __syncthreads();
    const int t = s_ticket;
    if ((uint32_t)t >= used) break;

    // Stable per-warp ranking: item order is (warp, iteration, lane).
    const uint32_t wbase = (uint32_t)t * kSortTile + (uint32_t)warp * 32 * kSortItems;
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = wbase + it * 32 + lane;
        const bool valid = idx < total;
        key[it] = valid ? kin[idx] : 0u;
        val[it] = valid ? vin[idx] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = wbase + it * 32 + lane;
        const bool valid = idx < total;
        const uint32_t vmask = __ballot_sync(kFull, valid);
        uint32_t r = 0;
        if (valid) {
            const uint32_t d = (key[it] >> shift) & dmask;
            const uint32_t peers = __match_any_sync(vmask, d);
            const uint32_t below = peers & lanemask_lt();
            const uint32_t prev = s_whist[warp][d];
            r = prev + __popc(below);
            __syncwarp(vmask);
            if (below == 0) s_whist[warp][d] = prev + __popc(peers);
        }
        __syncwarp();
        rank[it] = r;
    }
    __syncthreads();

    // Per digit: prefix over warps, block count, decoupled look-back.
    for (int d = tid; d < R; d += kSortThreads) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_whist[w][d];
            s_whist[w][d] = run;
            run += c;
        }
        s_cnt[d] = run;
        unsigned long long *lb = a.lookback + ((size_t)pass * a.n_sort_blocks) * R;
        unsigned long long excl = 0;
        if (t == 0) {
            if (pass == 0 && a.stall_first) {
                // Test of the bounded wait: the word after the look-back
                // array is zeroed with it and never written. The limit is an
                // eighth of the others', so the blocks waiting on this one
                // still see its counts and the sort completes correctly.
                const unsigned long long *never = a.lookback + (size_t)a.passes * a.n_sort_blocks * R;
                uint32_t spins = 0;
                while ((ld_relaxed(never) & ~kCountMask) == 0) {
                    if (++spins > kSpinLimit / 8) {
                        set_error(a.status, HTGS_ERR_TIMEOUT);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                }
            }
            st_relaxed(&lb[d], kFlagInc | run);
        } else {
            st_relaxed(&lb[(size_t)t * R + d], kFlagAgg | run);
            int pred = t - 1;
            uint32_t spins = 0;
            while (pred >= 0) {
                const unsigned long long v = ld_relaxed(&lb[(size_t)pred * R + d]);
                const unsigned long long flag = v & ~kCountMask;
                if (flag == 0) {
                    if (++spins > kSpinLimit) {
                        set_error(a.status, HTGS_ERR_TIMEOUT);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                    continue;
                }
                excl += v & kCountMask;
                if (flag == kFlagInc) break;
                --pred;
            }
            st_relaxed(&lb[(size_t)t * R + d], kFlagInc | ((excl + run) & kCountMask));
        }
        s_base[d] = s_scan[d] + (uint32_t)excl;
    }
    __syncthreads();
    block_scan(s_cnt, s_bstart);

    // Block-local positions in digit order, then the keys and values are
    // placed there (s_k reuses the per-warp counters' storage) and written
    // out in runs of equal digits, so consecutive threads store to
    // consecutive addresses.
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t d = (key[it] >> shift) & dmask;
        rank[it] += s_bstart[d] + s_whist[warp][d];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const uint32_t idx = wbase + it * 32 + lane;
        if (idx < total && rank[it] < (uint32_t)kSortTile) {
            s_k[rank[it]] = key[it];
            s_v[rank[it]] = val[it];
        }
    }
    __syncthreads();
    const uint32_t n_here = min((uint32_t)kSortTile, total - (uint32_t)t * kSortTile);
    for (uint32_t i = tid; i < n_here; i += kSortThreads) {
        const uint32_t k = s_k[i];
        const uint32_t d = (k >> shift) & dmask;
        const uint32_t pos = s_base[d] + (i - s_bstart[d]);
        if (pos < total) {  // always true unless a bounded wait gave up
            kout[pos] = k;
            vout[pos] = s_v[i];
        }
    }
    __syncthreads();  // the next tile reuses the shared arrays
    } // next tile
}

// ---------------------------------------------------------------------------
// Tile ranges from the sorted keys.
// ---------------------------------------------------------------------------
// Each thread takes kRangeKeys consecutive keys (two 16-byte loads) and
// their two neighbours, all loaded before any is compared; a neighbour past
// either end reads as a key no tile has.
constexpr int kRangeKeys = 8;
static_assert(kRangeKeys == 8, "two uint4 loads per thread");

__global__ void ranges_kernel(RangeArgs a) {
    dependent_entry();
    const uint32_t total = *a.total;
    const uint32_t none = 0xffffffffu;
    const uint32_t step = gridDim.x * blockDim.x * kRangeKeys;
    for (uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * kRangeKeys; i0 < total; i0 += step) {
        uint32_t k[kRangeKeys + 2];  // keys i0 - 1 .. i0 + kRangeKeys
        k[0] = i0 > 0 ? a.keys[i0 - 1] : none;
        if (i0 + kRangeKeys <= total) {
            // i0 is a multiple of 8 and the key array 16-byte aligned.
            const uint4 lo = *reinterpret_cast<const uint4 *>(a.keys + i0);
            const uint4 hi = *reinterpret_cast<const uint4 *>(a.keys + i0 + 4);
            k[1] = lo.x; k[2] = lo.y; k[3] = lo.z; k[4] = lo.w;
            k[5] = hi.x; k[6] = hi.y; k[7] = hi.z; k[8] = hi.w;
        } else {
#pragma unroll
            for (int j = 0; j < kRangeKeys; ++j) k[1 + j] = i0 + j < total ? a.keys[i0 + j] : none;
        }
        k[kRangeKeys + 1] = i0 + kRangeKeys < total ? a.keys[i0 + kRangeKeys] : none;
#pragma unroll
        for (int j = 0; j < kRangeKeys; ++j) {
            const uint32_t t = k[1 + j];
            if (t >= (uint32_t)a.n_tiles) continue;  // also past the end
            if (k[j] != t) a.ranges[t].x = i0 + j;
            if (k[j + 2] != t) a.ranges[t].y = i0 + j + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Blend work items (one CTA): chunk the long tile lists, then bucket the
// items by chunk length (two buckets per octave, longest first).
// ---------------------------------------------------------------------------
constexpr int kSchedUnroll = 4;  // tiles per thread and step of the schedule kernel

__device__ __forceinline__ int length_bucket(uint32_t len) {
    if (len == 0) return kSchedBuckets - 1;
    const int l = 31 - __clz(len);
    const int sub = l > 0 ? (int)((len >> (l - 1)) & 1u) : 0;
    return (kSchedBuckets - 2) - min(2 * l + sub, kSchedBuckets - 2);
}

__global__ void __launch_bounds__(kSchedThreads) schedule_kernel(ScheduleArgs a) {
    dependent_entry();
    __shared__ uint32_t s_cnt[kSchedBuckets];
    __shared__ uint32_t s_pos[kSchedBuckets];
    __shared__ uint32_t s_slots;
    __shared__ unsigned long long s_wt[kSchedThreads / 32];
    const int tid = threadIdx.x;
    if (a.tile_tot) {
        // Counting-sort binning: tile ranges and the instance total from the
        // per-tile counts. Thread tid owns tiles [tid * per, tid * per + per).
        const int T = a.n_tiles, lane = tid & 31, warp = tid >> 5;
        const int per = (T + kSchedThreads - 1) / kSchedThreads;
        const int t0 = tid * per;
        unsigned long long loc = 0;
        for (int k = 0; k < per; ++k)
            if (t0 + k < T) loc += a.tile_tot[t0 + k];
        unsigned long long incl = loc;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long x = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) s_wt[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long v = s_wt[lane];
            unsigned long long vi = v;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long x = __shfl_up_sync(kFull, vi, o);
                if (lane >= o) vi += x;
            }
            s_wt[lane] = vi - v;
        }
        __syncthreads();
        unsigned long long run = s_wt[warp] + incl - loc;
        for (int k = 0; k < per; ++k)
            if (t0 + k < T) {
                const uint32_t c = a.tile_tot[t0 + k];
                a.ranges_out[t0 + k] = make_uint2((uint32_t)run, (uint32_t)(run + c));
                run += c;
            }
        if (tid == kSchedThreads - 1) {
            a.status[kStInstLo] = (int)(uint32_t)(run & 0xffffffffull);
            a.status[kStInstHi] = (int)(uint32_t)(run >> 32);
            if (run > (unsigned long long)a.capacity) {
                set_error(a.status, HTGS_ERR_OVERFLOW);
                *a.total_out = 0;
            } else {
                *a.total_out = (uint32_t)run;
            }
        }
        __syncthreads();
    }
    // After a recorded failure the tile ranges may not describe the list
    // (keys a bounded wait left unsorted): schedule nothing.
    if (a.status[kStError] != 0) {
        if (tid == 0) *a.n_items = 0;
        return;
    }
    const uint64_t total = *a.total;
    uint64_t chunk = (total + kChunkDiv - 1) / kChunkDiv;
    if (chunk < kMinChunk) chunk = kMinChunk;
    // Every split tile uses m < 2 count / chunk slots: keep the sum within the cap.
    const uint64_t need = (2 * total + (uint64_t)a.slots_cap - 1) / (uint64_t)max(a.slots_cap, 1);
    if (chunk < need) chunk = need;
    auto parts = [&](uint32_t cnt) -> int {
        return (!a.no_split && cnt > chunk) ? (int)((cnt + chunk - 1) / chunk) : 1;
    };
    for (int b = tid; b < kSchedBuckets; b += kSchedThreads) s_cnt[b] = 0;
    if (tid == 0) s_slots = 0;
    __syncthreads();
    // Each thread takes kSchedUnroll tiles per step and loads their ranges
    // before any of its shared-memory atomics, so that the loads overlap.
    const int T = a.n_tiles;
    auto load_counts = [&](int t0, uint32_t (&cnt)[kSchedUnroll]) {
#pragma unroll
        for (int u = 0; u < kSchedUnroll; ++u) {
            const int t = t0 + u * kSchedThreads;
            const uint2 r = t < T ? a.ranges[t] : make_uint2(0u, 0u);
            cnt[u] = r.y - r.x;
        }
    };
    for (int t0 = tid; t0 < T; t0 += kSchedThreads * kSchedUnroll) {
        uint32_t cnt[kSchedUnroll];
        load_counts(t0, cnt);
#pragma unroll
        for (int u = 0; u < kSchedUnroll; ++u) {
            if (t0 + u * kSchedThreads >= T) break;
            const int m = parts(cnt[u]);
            atomicAdd(&s_cnt[length_bucket((cnt[u] + m - 1) / (uint32_t)m)], (uint32_t)m);
        }
    }
    __syncthreads();
    // Bucket offsets: an exclusive scan of the 64 bucket counts by one warp,
    // two buckets per lane.
    static_assert(kSchedBuckets == 64, "two buckets per lane of one warp");
    if (tid < 32) {
        const uint32_t c0 = s_cnt[2 * tid], c1 = s_cnt[2 * tid + 1];
        uint32_t incl = c0 + c1;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, incl, o);
            if (tid >= o) incl += x;
        }
        const uint32_t excl = incl - (c0 + c1);
        s_pos[2 * tid] = excl;
        s_pos[2 * tid + 1] = excl + c0;
        if (tid == 31) *a.n_items = incl;
    }
    __syncthreads();
    for (int t0 = tid; t0 < T; t0 += kSchedThreads * kSchedUnroll) {
        uint32_t cnt[kSchedUnroll];
        load_counts(t0, cnt);
#pragma unroll
        for (int u = 0; u < kSchedUnroll; ++u) {
            const int t = t0 + u * kSchedThreads;
            if (t >= T) break;
            const int m = parts(cnt[u]);
            const int slot0 = m > 1 ? (int)atomicAdd(&s_slots, (uint32_t)m) : 0;
            const uint32_t pos = atomicAdd(&s_pos[length_bucket((cnt[u] + m - 1) / (uint32_t)m)], (uint32_t)m);
            for (int k = 0; k < m; ++k) a.items[pos + k] = make_int4(t, k, m, slot0);
        }
    }
}

// Counts in emission order and their per-block sums.
__global__ void __launch_bounds__(kPreThreads) permute_counts_kernel(long long n, const uint32_t *perm,
                                                                     const uint32_t *count, uint32_t *count_p,
                                                                     uint32_t *block_sums) {
    dependent_entry();
    __shared__ uint32_t warp_sums[kPreThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    uint32_t c = 0;
    if (i < n) {
        const uint32_t r = perm[i];
        c = r < (uint64_t)n ? count[r] : 0u;
        count_p[i] = c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kPreThreads / 32; ++w) tot += warp_sums[w];
        block_sums[blockIdx.x] = tot;
    }
}

} // namespace

void launch_permute_counts(long long n, const uint32_t *perm, const uint32_t *count, uint32_t *count_p,
                           uint32_t *block_sums, cudaStream_t s) {
    const int blocks = (int)((n + kPreThreads - 1) / kPreThreads);
    if (blocks > 0) launch_k(permute_counts_kernel, blocks, kPreThreads, 0, s, n, perm, count, count_p, block_sums);
}

void launch_schedule(const ScheduleArgs &a, cudaStream_t s) {
    launch_k(schedule_kernel, 1, kSchedThreads, 0, s, a);
}

void launch_scan_blocks(const BinArgs &a, cudaStream_t s) {
    launch_k(scan_blocks_kernel, 1, kScanThreads, 0, s, a);
}

void launch_emit(const Batch &b, const BinArgs &a, cudaStream_t s) {
    if (a.n_blocks > 0) launch_k(emit_kernel, a.n_blocks, kPreThreads, 0, s, b, a);
}

int launch_sort(const SortArgs &a, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int hist_blocks = std::min<int64_t>((int64_t)sms * 4, (a.capacity + kSortThreads - 1) / kSortThreads + 1);
    launch_k(histogram_kernel, hist_blocks, kSortThreads, 0, s, a);
    // Enough blocks to fill the GPU; each takes tiles until none is left.
    static int per_sm = 0;
    if (per_sm == 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel, kSortThreads, 0) !=
                            cudaSuccess || per_sm < 1))
        per_sm = 1;
    const int grid = std::min<int64_t>(a.n_sort_blocks, (int64_t)sms * per_sm);
    int src = 0;
    for (int p = 0; p < a.passes; ++p) {
        launch_k(onesweep_kernel, grid, kSortThreads, 0, s, a, p, src);
        src ^= 1;
    }
    return src;
}

void launch_ranges(RangeArgs a, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    launch_k(ranges_kernel, sms * 8, 256, 0, s, a);  // 2.5M keys per sweep
}

namespace {
thread_local bool t_dependent_launch = false;
}

void set_dependent_launch(bool on) { t_dependent_launch = on; }
bool dependent_launch() { return t_dependent_launch; }

bool allow_dynamic_smem(const void *kernel, size_t bytes) {
    // Once per (kernel, device): the attribute persists, and repeating the
    // call on every launch (possibly inside a stream capture) is avoidable.
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    done.insert({kernel, dev});
    return true;
}

int persistent_grid(const void *kernel, int threads, size_t dyn_smem, int items) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long grid = (long long)sms * per_sm;
    return (int)(grid < items ? grid : (items > 0 ? items : 1));
}

} // namespace htgs
