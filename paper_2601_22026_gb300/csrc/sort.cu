// Tile binning: pair emission, stable sort by (tile id, depth), per-tile
// ranges.
//
// 3DGS (which the fitted peripheral model is, Section 4.2) renders by sorting
// every (Gaussian, covered tile) pair by (tile id, depth) once per image and
// compositing each tile's range front to back. Every pair of one Gaussian
// record carries the same depth, so the sort is done in two stages:
//   1. reduce_kernel / scan_kernel: a spin-free reduce-then-scan over the
//      per-record tile counts gives the total pair count (kept on the device;
//      checked against capacity) and the number of binned records.
//   2. compact_kernel: the binned records, in record order, as 64-bit keys
//      (tile count << 32 | depth bits) with the record index as value; also
//      the depth-digit histograms, and clears the look-back tables and ranges.
//   3. onesweep_kernel x 4 over the depth bits: a stable counting pass per
//      8-bit digit in the Onesweep style (Adinets & Merrill 2022): each CTA
//      ranks a 4096-key partition in shared memory, publishes its digit
//      counts, obtains its global digit offsets by decoupled look-back over
//      earlier partitions (every wait bounded: on expiry the status word gets
//      GSFIT_ERR_TIMEOUT), and writes its keys digit-run by digit-run so
//      stores coalesce. Records are now in (depth, record index) order.
//   4. reduce_sorted_kernel / scan_blocks_kernel / emit_kernel: pair offsets
//      in that order, then the pairs (tile id << 32 | depth, Gaussian index),
//      with the tile-digit histograms.
//   5. onesweep_kernel over the significant tile-id bits only (two passes for
//      up to 65536 tiles): being stable, it leaves equal tile ids in (depth,
//      record index) order, the unique order by (key, view, index).
//   6. ranges_kernel: [first, last+1) of each tile from adjacent keys.
// Sorting records instead of pairs by depth moves 24 bytes per record per
// depth pass instead of 24 bytes per pair (a record covers several tiles).
// Counts never leave the device, so the sequence can be captured in a CUDA
// graph; launches are sized by capacity and idle CTAs exit at once.
#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;  // records per block
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kPart = kSortThreads * kSortItems;  // keys per partition
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 1u << 31;
constexpr uint32_t kValMask = kFlagAgg - 1u;
constexpr int kSpinLimit = 1 << 20;  // x ~100 ns sleeps: about a tenth of a second
constexpr int kHistBlocks = 1024;

constexpr int kDepthPasses = 4;  // 8-bit digits over the 32 depth bits

struct SortCtl {
    uint32_t n_sort;      // pairs to sort (0 when the capacity was exceeded)
    uint32_t n_rec;       // binned records to sort (0 when the capacity was exceeded)
    unsigned long long total;  // exact pair count
    uint32_t part_counter[kMaxPasses];
    uint32_t hist[kMaxPasses][kRadix];  // depth passes, then tile passes
    uint32_t order_hist[32];  // tiles per log2(list length + 1) bucket
    uint32_t order_fill[32];
};

// Block-wide exclusive scan of one value per thread (blockDim == 256).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t s = s_warp[w];
        if (w < wid) wpre += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + incl - x;
}

// Per block of kScanChunk records: pair count and binned-record count.
__global__ void __launch_bounds__(kScanThreads) reduce_kernel(const uint32_t* __restrict__ tiles, long long n_rec,
                                                              uint32_t* __restrict__ pair_sums,
                                                              uint32_t* __restrict__ rec_sums) {
    __shared__ uint32_t s_warp[8];
    const long long base = (long long)blockIdx.x * kScanChunk;
    uint32_t acc = 0, cnt = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long r = base + (long long)j * kScanThreads + threadIdx.x;
        const uint32_t t = r < n_rec ? tiles[r] : 0u;
        acc += t;
        cnt += t > 0u;
    }
    uint32_t total;
    block_excl_scan(acc, s_warp, total);
    if (threadIdx.x == 0) pair_sums[blockIdx.x] = total;
    block_excl_scan(cnt, s_warp, total);
    if (threadIdx.x == 0) rec_sums[blockIdx.x] = total;
}

// In-place exclusive scan of n_blocks block sums by one 1024-thread block;
// returns the total (to thread 0).
__device__ unsigned long long scan_block_sums(uint32_t* __restrict__ sums, int n_blocks) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += 1024) {
        const int b = base + threadIdx.x;
        const unsigned long long x = b < n_blocks ? sums[b] : 0ull;
        unsigned long long incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        unsigned long long wpre = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < wid) wpre += s_warp[w];
            tot += s_warp[w];
        }
        const unsigned long long carry = s_carry;
        if (b < n_blocks) sums[b] = (uint32_t)(carry + wpre + incl - x);
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    return s_carry;
}

// Single block: scans of both block-sum arrays, totals, capacity check, and
// reset of the sort control block.
__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ pair_sums, uint32_t* __restrict__ rec_sums,
                                                    int n_blocks, SortCtl* __restrict__ ctl,
                                                    uint32_t* __restrict__ n_instances, long long capacity,
                                                    int32_t* __restrict__ status) {
    for (int k = threadIdx.x; k < kMaxPasses * kRadix; k += blockDim.x) (&ctl->hist[0][0])[k] = 0u;
    if (threadIdx.x < kMaxPasses) ctl->part_counter[threadIdx.x] = 0u;
    if (threadIdx.x < 32) {
        ctl->order_hist[threadIdx.x] = 0u;
        ctl->order_fill[threadIdx.x] = 0u;
    }
    const unsigned long long total = scan_block_sums(pair_sums, n_blocks);
    const unsigned long long recs = scan_block_sums(rec_sums, n_blocks);
    if (threadIdx.x == 0) {
        ctl->total = total;
        *n_instances = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
        if (total > (unsigned long long)capacity) {
            ctl->n_sort = 0u;
            ctl->n_rec = 0u;
            *status = GSFIT_ERR_CAPACITY;
        } else {
            ctl->n_sort = (uint32_t)total;
            ctl->n_rec = (uint32_t)recs;
        }
    }
}

// Single block: in-place exclusive scan of the sorted records' block sums.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* __restrict__ sums, int n_blocks) {
    scan_block_sums(sums, n_blocks);
}

// Binned records in record order as (tile count << 32 | depth bits, record
// index), with the depth-digit histograms; clears the look-back tables and
// the tile ranges for this sort.
__global__ void __launch_bounds__(kScanThreads) compact_kernel(const uint32_t* __restrict__ tiles,
                                                               const float4* __restrict__ xyd, long long n_rec,
                                                               const uint32_t* __restrict__ rec_sums,
                                                               SortCtl* __restrict__ ctl,
                                                               unsigned long long* __restrict__ rkeys,
                                                               uint32_t* __restrict__ rvals,
                                                               uint32_t* __restrict__ lookback, long long lookback_words,
                                                               uint32_t* __restrict__ ranges, long long range_words) {
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_hist[kDepthPasses][kRadix];
    for (int k = threadIdx.x; k < kDepthPasses * kRadix; k += blockDim.x) (&s_hist[0][0])[k] = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long k = tid; k < lookback_words; k += stride) lookback[k] = 0u;
    for (long long k = tid; k < range_words; k += stride) ranges[k] = 0u;
    __syncthreads();
    if (ctl->n_rec == 0u) return;  // nothing binned, or the capacity was exceeded
    const long long base = (long long)blockIdx.x * kScanChunk;
    uint32_t offset = rec_sums[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        const long long r = base + (long long)j * kScanThreads + threadIdx.x;
        const uint32_t t = r < n_rec ? tiles[r] : 0u;
        uint32_t row_total;
        const uint32_t ex = block_excl_scan(t > 0u ? 1u : 0u, s_warp, row_total);
        if (t > 0u) {
            const uint32_t depth = __float_as_uint(xyd[r].z);
            rkeys[offset + ex] = ((unsigned long long)t << 32) | depth;
            rvals[offset + ex] = (uint32_t)r;
#pragma unroll
            for (int p = 0; p < kDepthPasses; ++p) atomicAdd(&s_hist[p][(depth >> (8 * p)) & 0xff], 1u);
        }
        offset += row_total;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kDepthPasses * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[k];
        if (c) atomicAdd(&ctl->hist[0][0] + k, c);
    }
}

// Pair counts of the depth-sorted records, per block of kScanChunk.
__global__ void __launch_bounds__(kScanThreads) reduce_sorted_kernel(const unsigned long long* __restrict__ rkeys,
                                                                     const SortCtl* __restrict__ ctl,
                                                                     uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[8];
    const uint32_t n = ctl->n_rec;
    const long long base = (long long)blockIdx.x * kScanChunk;
    uint32_t acc = 0;
    if (base < n) {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const long long m = base + (long long)j * kScanThreads + threadIdx.x;
            if (m < n) acc += (uint32_t)(rkeys[m] >> 32);
        }
    }
    uint32_t total;
    block_excl_scan(acc, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Pairs of the depth-sorted records, in that order, with the tile-digit
// histograms of the n_tile_passes tile passes.
__global__ void __launch_bounds__(kScanThreads) emit_kernel(const unsigned long long* __restrict__ rkeys,
                                                            const uint32_t* __restrict__ rvals,
                                                            const float4* __restrict__ xyd, int n, int n_views,
                                                            const gsfit_camera* __restrict__ cams_g,
                                                            const uint32_t* __restrict__ sums,
                                                            SortCtl* __restrict__ ctl, int n_tile_passes,
                                                            unsigned long long* __restrict__ keys,
                                                            uint32_t* __restrict__ vals) {
    extern __shared__ gsfit_camera cams[];
    __shared__ uint32_t s_warp[8];
    __shared__ uint32_t s_hist[kMaxPasses - kDepthPasses][kRadix];
    load_cameras(cams, cams_g, n_views);
    for (int k = threadIdx.x; k < n_tile_passes * kRadix; k += blockDim.x) (&s_hist[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t n_recs = ctl->n_rec;
    const long long base = (long long)blockIdx.x * kScanChunk;
    if (base >= n_recs) return;
    uint32_t offset = sums[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        const long long m = base + (long long)j * kScanThreads + threadIdx.x;
        const bool ok = m < n_recs;
        const unsigned long long rk = ok ? rkeys[m] : 0ull;
        const uint32_t t = (uint32_t)(rk >> 32);
        uint32_t row_total;
        const uint32_t ex = block_excl_scan(t, s_warp, row_total);
        if (t > 0u) {
            const uint32_t r = rvals[m];
            const int v = (int)(r / (uint32_t)n);
            const int i = (int)(r - (uint32_t)v * (uint32_t)n);
            const gsfit_camera& cam = cams[v];
            const float4 p = xyd[r];
            const int txn = tiles_x_of(cam);
            const Rect rc = tile_rect(p.x, p.y, p.w, txn, tiles_y_of(cam), tile_of(cam));
            const unsigned long long depth = rk & 0xffffffffull;
            uint32_t o = offset + ex;
            for (int ty = rc.y0; ty < rc.y1; ++ty)
                for (int tx = rc.x0; tx < rc.x1; ++tx) {
                    const uint32_t tile = (uint32_t)(cam.tile_offset + ty * txn + tx);
                    keys[o] = ((unsigned long long)tile << 32) | depth;
                    vals[o] = (uint32_t)i;
                    ++o;
                    for (int q = 0; q < n_tile_passes; ++q) atomicAdd(&s_hist[q][(tile >> (8 * q)) & 0xff], 1u);
                }
        }
        offset += row_total;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_tile_passes * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[k];
        if (c) atomicAdd(&ctl->hist[kDepthPasses][0] + k, c);
    }
}

// Waits until a look-back word carries a flag (aggregate or inclusive prefix)
// and returns it in f; false, with GSFIT_ERR_TIMEOUT in the status word, after
// `limit` polls of ~100 ns.
__device__ __forceinline__ bool lookback_poll(const uint32_t* word, uint32_t& f, int32_t* status, int limit) {
    for (int spins = 0;; ++spins) {
        f = *reinterpret_cast<const volatile uint32_t*>(word);
        if (f & (kFlagInc | kFlagAgg)) return true;
        if (spins >= limit) {
            if (status) atomicExch(status, GSFIT_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(100);
    }
}

// Diagnostic: polls a look-back word nothing will ever set.
__global__ void lookback_selftest_kernel(const uint32_t* word, int limit, int32_t* status) {
    uint32_t f;
    lookback_poll(word, f, status, limit);
}

struct OnesweepSmem {
    unsigned long long keys[kPart];
    uint32_t vals[kPart];
    uint32_t vals_in[kPart];  // this partition's values in input order
    uint32_t warp_hist[kSortWarps][kRadix + 1];  // bin kRadix collects padding keys
    uint32_t local_start[kRadix];
    uint32_t glob_off[kRadix];  // global position of local index j is glob_off[d] + j
    uint32_t scan_warp[8];
    uint32_t part;
};

// One stable counting pass over the 8-bit digit at bit `shift` of *n_ptr keys;
// `pass` indexes the histogram and partition counter of this launch.
__global__ void __launch_bounds__(kSortThreads, 3) onesweep_kernel(const unsigned long long* __restrict__ keys_in,
                                                                const uint32_t* __restrict__ vals_in,
                                                                unsigned long long* __restrict__ keys_out,
                                                                uint32_t* __restrict__ vals_out,
                                                                SortCtl* __restrict__ ctl, int pass, int shift,
                                                                const uint32_t* __restrict__ n_ptr,
                                                                uint32_t* __restrict__ lookback,
                                                                int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem& S = *reinterpret_cast<OnesweepSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t n = *n_ptr;
    const uint32_t n_parts = (n + kPart - 1) / kPart;
    if (threadIdx.x == 0) S.part = atomicAdd(&ctl->part_counter[pass], 1u);
    for (int k = threadIdx.x; k < kSortWarps * (kRadix + 1); k += kSortThreads) (&S.warp_hist[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t part = S.part;
    if (part >= n_parts) return;
    const uint32_t base = part * kPart;
    const uint32_t valid = min((uint32_t)kPart, n - base);

    // Load (warp-striped, coalesced) and rank within the warp per digit. Keys
    // stay in registers; values wait in shared memory in input order.
    unsigned long long k_reg[kSortItems];
    uint32_t r_reg[kSortItems];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t idx = (uint32_t)wid * (32 * kSortItems) + j * 32 + lane;
        const bool ok = idx < valid;
        k_reg[j] = ok ? keys_in[base + idx] : ~0ull;
        if (ok) S.vals_in[idx] = vals_in[base + idx];
    }
    // digit of item j; items past the end go to bin kRadix
    auto digit = [&](int j) -> uint32_t {
        const uint32_t idx = (uint32_t)wid * (32 * kSortItems) + j * 32 + lane;
        return idx < valid ? (uint32_t)((k_reg[j] >> shift) & 0xff) : (uint32_t)kRadix;
    };
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = digit(j);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t cnt = S.warp_hist[wid][d];
        __syncwarp();
        const int leader = 31 - __clz(peers);
        if (lane == leader) S.warp_hist[wid][d] = cnt + __popc(peers);
        __syncwarp();
        r_reg[j] = cnt + __popc(peers & lt_mask);
    }
    __syncthreads();

    // Per digit: prefix over warps, block count, block-local digit start.
    const int d = threadIdx.x;  // kSortThreads == kRadix
    uint32_t dcount = 0;
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = S.warp_hist[w][d];
        S.warp_hist[w][d] = dcount;
        dcount += c;
    }
    // publish this partition's aggregate before looking back
    uint32_t* lb = lookback;  // this pass's table
    if (part == 0) {
        atomicExch(&lb[d], kFlagInc | dcount);
    } else {
        atomicExch(&lb[(size_t)part * kRadix + d], kFlagAgg | dcount);
    }
    uint32_t tot;
    const uint32_t lstart = block_excl_scan(dcount, S.scan_warp, tot);
    S.local_start[d] = lstart;

    // decoupled look-back over earlier partitions for digit d
    uint32_t excl = 0;
    if (part > 0) {
        int p = (int)part - 1;
        while (p >= 0) {
            uint32_t f;
            if (!lookback_poll(&lb[(size_t)p * kRadix + d], f, status, kSpinLimit)) break;  // timed out
            excl += f & kValMask;
            if (f & kFlagInc) break;
            --p;  // an aggregate: keep looking back
        }
        atomicExch(&lb[(size_t)part * kRadix + d], kFlagInc | (excl + dcount));
    }
    // global exclusive offset of digit d over all keys of this pass
    uint32_t htot;
    const uint32_t gexcl = block_excl_scan(ctl->hist[pass][d], S.scan_warp, htot);
    S.glob_off[d] = gexcl + excl - lstart;
    __syncthreads();

    // scatter into shared memory in digit order (stable: warp, item, lane order)
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t dd = digit(j);
        if (dd < (uint32_t)kRadix) {
            const uint32_t pos = S.local_start[dd] + S.warp_hist[wid][dd] + r_reg[j];
            S.keys[pos] = k_reg[j];
            S.vals[pos] = S.vals_in[(uint32_t)wid * (32 * kSortItems) + j * 32 + lane];
        }
    }
    __syncthreads();
    // write runs of equal digits to consecutive global addresses
    for (uint32_t j = threadIdx.x; j < valid; j += kSortThreads) {
        const unsigned long long key = S.keys[j];
        const uint32_t dd = (uint32_t)((key >> shift) & 0xff);
        const uint32_t o = S.glob_off[dd] + j;
        if (o < n) {  // always true unless a look-back wait ran out
            keys_out[o] = key;
            vals_out[o] = S.vals[j];
        }
    }
}

__global__ void __launch_bounds__(256) ranges_kernel(const unsigned long long* __restrict__ keys,
                                                     const SortCtl* __restrict__ ctl,
                                                     uint32_t* __restrict__ ranges, uint32_t total_tiles) {
    const uint32_t n = ctl->n_sort;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint32_t t = (uint32_t)(keys[k] >> 32);
        if (t >= total_tiles) continue;  // only after a failed sort
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)k;
        if (k + 1 == n || (uint32_t)(keys[k + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(k + 1);
    }
}

// Heavy-first tile order: tiles bucketed by floor(log2(list length + 1)),
// buckets in decreasing order, tiles within a bucket in any order.
__device__ __forceinline__ int length_bucket(const uint32_t* ranges, int t) {
    const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
    return 31 - __clz(len + 1u);
}

__global__ void __launch_bounds__(256) order_hist_kernel(const uint32_t* __restrict__ ranges, int total_tiles,
                                                         SortCtl* __restrict__ ctl) {
    __shared__ uint32_t h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x)
        atomicAdd(&h[length_bucket(ranges, t)], 1u);
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&ctl->order_hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void __launch_bounds__(256) order_scatter_kernel(const uint32_t* __restrict__ ranges, int total_tiles,
                                                            SortCtl* __restrict__ ctl,
                                                            uint32_t* __restrict__ tile_order) {
    __shared__ uint32_t off[32];
    if (threadIdx.x == 0) {
        uint32_t o = 0;
        for (int b = 31; b >= 0; --b) {
            off[b] = o;
            o += ctl->order_hist[b];
        }
    }
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x) {
        const int b = length_bucket(ranges, t);
        tile_order[off[b] + atomicAdd(&ctl->order_fill[b], 1u)] = (uint32_t)t;
    }
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct SortLayout {
    size_t pair_sums, rec_sums, sorted_sums, ctl, lookback, keys_alt, vals_alt, rkeys[2], rvals[2], total;
    int n_blocks, tile_passes;
    long long max_parts, max_rec_parts, lookback_words;
};

int tile_passes_for(int total_tiles) {
    int bits = 0;
    while ((1ll << bits) < (long long)total_tiles) ++bits;  // tile ids 0 .. total_tiles-1
    return bits == 0 ? 1 : (bits + 7) / 8;
}

SortLayout layout(long long n_rec, long long capacity, int total_tiles) {
    SortLayout L;
    L.n_blocks = (int)((n_rec + kScanChunk - 1) / kScanChunk);
    if (L.n_blocks < 1) L.n_blocks = 1;
    L.tile_passes = tile_passes_for(total_tiles);
    L.max_parts = (capacity + kPart - 1) / kPart;
    if (L.max_parts < 1) L.max_parts = 1;
    L.max_rec_parts = (n_rec + kPart - 1) / kPart;
    if (L.max_rec_parts < 1) L.max_rec_parts = 1;
    L.lookback_words = ((long long)kDepthPasses * L.max_rec_parts + (long long)L.tile_passes * L.max_parts) * kRadix;
    const size_t cap = (size_t)(capacity > 0 ? capacity : 1), nr = (size_t)(n_rec > 0 ? n_rec : 1);
    size_t o = 0;
    L.pair_sums = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.n_blocks);
    L.rec_sums = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.n_blocks);
    L.sorted_sums = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.n_blocks);
    L.ctl = o; o = align_up(o + sizeof(SortCtl));
    L.lookback = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.lookback_words);
    L.keys_alt = o; o = align_up(o + sizeof(unsigned long long) * cap);
    L.vals_alt = o; o = align_up(o + sizeof(uint32_t) * cap);
    for (int b = 0; b < 2; ++b) {
        L.rkeys[b] = o; o = align_up(o + sizeof(unsigned long long) * nr);
        L.rvals[b] = o; o = align_up(o + sizeof(uint32_t) * nr);
    }
    L.total = o;
    return L;
}

// Opt-in to more than 48 KB of dynamic shared memory, once per device.
int enable_onesweep_smem(size_t smem) {
    static bool done[64] = {false};
    int dev = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GSFIT_ERR_CUDA;
    if (!done[dev]) {
        GSFIT_CUDA_CHECK(cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        done[dev] = true;
    }
    return GSFIT_OK;
}

}  // namespace

bool valid_proj(const gsfit_proj* p);

}  // namespace gsfit

using namespace gsfit;

extern "C" size_t gsfit_bin_sort_workspace_size(int64_t n_records, int64_t capacity, int32_t total_tiles) {
    if (n_records < 0 || capacity < 0 || total_tiles < 1) return 0;
    return layout(n_records, capacity, total_tiles).total;
}

extern "C" int gsfit_bin_sort(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                              int32_t total_tiles, void* ws, size_t ws_bytes, uint64_t* keys, uint32_t* vals,
                              int64_t capacity, uint32_t* n_instances, uint32_t* ranges, uint32_t* tile_order,
                              int32_t* status, cudaStream_t stream) {
    if (!valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || n < 1 || total_tiles < 1 ||
        !ws || !keys || !vals || !n_instances || !ranges || !status || capacity < 1 ||
        capacity >= (int64_t)kFlagAgg)
        return GSFIT_ERR_INVALID_ARG;
    const long long n_rec = (long long)n * n_views;
    if (n_rec >= (long long)0xffffffffll) return GSFIT_ERR_INVALID_ARG;  // record indices are 32-bit
    const SortLayout L = layout(n_rec, capacity, total_tiles);
    if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) % 256) != 0) return GSFIT_ERR_INVALID_ARG;
    char* base = static_cast<char*>(ws);
    uint32_t* pair_sums = reinterpret_cast<uint32_t*>(base + L.pair_sums);
    uint32_t* rec_sums = reinterpret_cast<uint32_t*>(base + L.rec_sums);
    uint32_t* sorted_sums = reinterpret_cast<uint32_t*>(base + L.sorted_sums);
    SortCtl* ctl = reinterpret_cast<SortCtl*>(base + L.ctl);
    uint32_t* lookback = reinterpret_cast<uint32_t*>(base + L.lookback);
    unsigned long long* keys_alt = reinterpret_cast<unsigned long long*>(base + L.keys_alt);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(base + L.vals_alt);
    unsigned long long* rk[2] = {reinterpret_cast<unsigned long long*>(base + L.rkeys[0]),
                                 reinterpret_cast<unsigned long long*>(base + L.rkeys[1])};
    uint32_t* rv[2] = {reinterpret_cast<uint32_t*>(base + L.rvals[0]), reinterpret_cast<uint32_t*>(base + L.rvals[1])};
    unsigned long long* keys_out = reinterpret_cast<unsigned long long*>(keys);
    const size_t smem = sizeof(OnesweepSmem);
    const int rc = enable_onesweep_smem(smem);
    if (rc != GSFIT_OK) return rc;

    reduce_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(proj->tiles, n_rec, pair_sums, rec_sums);
    GSFIT_LAUNCH_CHECK();
    scan_kernel<<<1, 1024, 0, stream>>>(pair_sums, rec_sums, L.n_blocks, ctl, n_instances, capacity, status);
    GSFIT_LAUNCH_CHECK();
    compact_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(proj->tiles, reinterpret_cast<const float4*>(proj->xyd),
                                                            n_rec, rec_sums, ctl, rk[0], rv[0], lookback,
                                                            L.lookback_words, ranges, 2ll * total_tiles);
    GSFIT_LAUNCH_CHECK();
    // depth passes over the records (an even number: the result is back in buffer 0)
    uint32_t* lb = lookback;
    for (int p = 0; p < kDepthPasses; ++p) {
        onesweep_kernel<<<(unsigned)L.max_rec_parts, kSortThreads, smem, stream>>>(
            rk[p & 1], rv[p & 1], rk[(p + 1) & 1], rv[(p + 1) & 1], ctl, p, 8 * p, &ctl->n_rec, lb, status);
        GSFIT_LAUNCH_CHECK();
        lb += (size_t)L.max_rec_parts * kRadix;
    }
    reduce_sorted_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(rk[0], ctl, sorted_sums);
    GSFIT_LAUNCH_CHECK();
    scan_blocks_kernel<<<1, 1024, 0, stream>>>(sorted_sums, L.n_blocks);
    GSFIT_LAUNCH_CHECK();
    // pairs go to the buffer that, after the tile passes' ping-pong, leaves the result in keys/vals
    const bool emit_to_alt = (L.tile_passes % 2) == 1;
    unsigned long long* k_cur = emit_to_alt ? keys_alt : keys_out;
    uint32_t* v_cur = emit_to_alt ? vals_alt : vals;
    unsigned long long* k_nxt = emit_to_alt ? keys_out : keys_alt;
    uint32_t* v_nxt = emit_to_alt ? vals : vals_alt;
    emit_kernel<<<L.n_blocks, kScanThreads, sizeof(gsfit_camera) * n_views, stream>>>(
        rk[0], rv[0], reinterpret_cast<const float4*>(proj->xyd), n, n_views, cams, sorted_sums, ctl, L.tile_passes,
        k_cur, v_cur);
    GSFIT_LAUNCH_CHECK();
    for (int q = 0; q < L.tile_passes; ++q) {
        onesweep_kernel<<<(unsigned)L.max_parts, kSortThreads, smem, stream>>>(
            k_cur, v_cur, k_nxt, v_nxt, ctl, kDepthPasses + q, 32 + 8 * q, &ctl->n_sort, lb, status);
        GSFIT_LAUNCH_CHECK();
        lb += (size_t)L.max_parts * kRadix;
        std::swap(k_cur, k_nxt);
        std::swap(v_cur, v_nxt);
    }
    ranges_kernel<<<kHistBlocks, 256, 0, stream>>>(keys_out, ctl, ranges, (uint32_t)total_tiles);
    GSFIT_LAUNCH_CHECK();
    if (tile_order) {
        const int ob = min(152, (total_tiles + 255) / 256);
        order_hist_kernel<<<ob, 256, 0, stream>>>(ranges, total_tiles, ctl);
        GSFIT_LAUNCH_CHECK();
        order_scatter_kernel<<<ob, 256, 0, stream>>>(ranges, total_tiles, ctl, tile_order);
        GSFIT_LAUNCH_CHECK();
    }
    return GSFIT_OK;
}

extern "C" int gsfit_selftest_lookback_timeout(uint32_t* word, int32_t polls, int32_t* status, cudaStream_t stream) {
    if (!word || !status || polls < 1) return GSFIT_ERR_INVALID_ARG;
    lookback_selftest_kernel<<<1, 32, 0, stream>>>(word, polls, status);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
