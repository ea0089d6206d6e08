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
//      stores coalesce. A pass whose digit is the same for every key (the
//      histogram has one bucket holding them all, as the top depth byte is
//      when all depths share a binary exponent) is the identity permutation:
//      its CTAs exit at once and the records stay in their buffer (each later
//      kernel derives the buffer from the histograms). Records are now in
//      (depth, record index) order.
//   4. reduce_sorted_kernel / scan_blocks_kernel / emit_kernel: pair offsets
//      in that order (per block of records, and per 128-record segment within
//      it), then the pairs (tile id << 32 | depth, Gaussian index), with the
//      tile-digit histograms; a resident grid of warps takes the segments in
//      turn and deals each row's pairs out to its lanes 32 at a time, so
//      stores coalesce whatever the splat sizes.
//   5. onesweep_kernel over the significant tile-id bits only (two passes for
//      up to 65536 tiles): being stable, it leaves equal tile ids in (depth,
//      record index) order, the unique order by (key, view, index).
//   6. ranges_kernel: [first, last+1) of each tile from adjacent keys, and
//      the heavy-first tile order for the compositing kernels.
// Sorting records instead of pairs by depth moves 24 bytes per record per
// depth pass instead of 24 bytes per pair (a record covers several tiles).
// Counts never leave the device, so the sequence can be captured in a CUDA
// graph; launches are sized by capacity (or, for the emission, by the SM
// count) and idle CTAs exit at once.
#include <algorithm>

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

constexpr int kDepthPasses = 4;  // 8-bit digits over the 32 depth bits

struct SortCtl {
    uint32_t n_sort;      // pairs to sort (0 when the capacity was exceeded)
    uint32_t n_rec;       // binned records to sort (0 when the capacity was exceeded)
    unsigned long long total;  // exact pair count
    uint32_t part_counter[kMaxPasses];
    uint32_t hist[kMaxPasses][kRadix];  // depth passes, then tile passes
    uint32_t order_hist[128];  // tiles per work bucket (tile order)
    uint32_t order_fill[128];
    uint32_t depth_buf;  // buffer of the depth-sorted records (set by reduce_sorted_kernel)
};

// The buffer (0 or 1) holding the depth-sorted records after depth passes
// [0, p) (blockDim == kRadix, called by the whole block): a pass whose digit
// is the same for all n keys is the identity permutation and is skipped; every
// other pass moves the records to the other buffer.
__device__ __forceinline__ int depth_buffer(const SortCtl* ctl, int p, uint32_t n) {
    int b = 0;
    for (int q = 0; q < p; ++q) b ^= __syncthreads_or(ctl->hist[q][threadIdx.x] == n) ? 0 : 1;
    return b;
}

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
    if (threadIdx.x < kOrderBuckets) {
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
// the tile ranges for this sort. Warp w of a block takes the block's records
// [32 kScanItems w, 32 kScanItems (w + 1)) as kScanItems rows of 32 and
// places each row's binned records with a ballot; one block-wide step orders
// the warps.
__global__ void __launch_bounds__(kScanThreads) compact_kernel(const uint32_t* __restrict__ tiles,
                                                               const float4* __restrict__ xyd, long long n_rec,
                                                               const uint32_t* __restrict__ rec_sums,
                                                               SortCtl* __restrict__ ctl,
                                                               unsigned long long* __restrict__ rkeys,
                                                               uint32_t* __restrict__ rvals,
                                                               uint32_t* __restrict__ lookback, long long lookback_words,
                                                               uint32_t* __restrict__ ranges, long long range_words) {
    __shared__ uint32_t s_wtot[kScanThreads / 32];
    __shared__ uint32_t s_hist[kDepthPasses][kRadix];
    for (int k = threadIdx.x; k < kDepthPasses * kRadix; k += blockDim.x) (&s_hist[0][0])[k] = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long k = tid; k < lookback_words; k += stride) lookback[k] = 0u;
    for (long long k = tid; k < range_words; k += stride) ranges[k] = 0u;
    __syncthreads();
    if (ctl->n_rec == 0u) return;  // nothing binned, or the capacity was exceeded
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long wbase = (long long)blockIdx.x * kScanChunk + (long long)wid * (32 * kScanItems);
    const float* depth_of = reinterpret_cast<const float*>(xyd) + 2;  // .z of record r at 4 r
    bool bin[kScanItems];
    uint32_t depth[kScanItems];
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long r = wbase + 32 * j + lane;
        bin[j] = r < n_rec && __ldg(tiles + r) > 0u;
        mine += bin[j];
    }
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long r = wbase + 32 * j + lane;
        depth[j] = bin[j] ? __float_as_uint(__ldg(depth_of + 4 * r)) : 0u;
    }
    const uint32_t wtot = __reduce_add_sync(0xffffffffu, mine);
    if (lane == 0) s_wtot[wid] = wtot;
    __syncthreads();
    uint32_t offset = rec_sums[blockIdx.x];
    for (int w = 0; w < wid; ++w) offset += s_wtot[w];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const uint32_t m = __ballot_sync(0xffffffffu, bin[j]);
        if (bin[j]) {
            const long long r = wbase + 32 * j + lane;
            const uint32_t o = offset + __popc(m & lt);
            rkeys[o] = ((unsigned long long)__ldg(tiles + r) << 32) | depth[j];
            rvals[o] = (uint32_t)r;
#pragma unroll
            for (int p = 0; p < kDepthPasses; ++p) atomicAdd(&s_hist[p][(depth[j] >> (8 * p)) & 0xff], 1u);
        }
        offset += __popc(m);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kDepthPasses * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[k];
        if (c) atomicAdd(&ctl->hist[0][0] + k, c);
    }
}

// The emit kernel's unit of work: kEmitSeg consecutive depth-sorted records,
// taken by one warp as rows of 32.
constexpr int kEmitSeg = 128;
constexpr int kSegsPerChunk = kScanChunk / kEmitSeg;
static_assert(kSegsPerChunk == 32 && kScanItems * 2 == kSegsPerChunk, "one segment per half row of a chunk load");
constexpr int kEmitBlocksPerSm = 5;

// Pair counts of the depth-sorted records: per block of kScanChunk (the
// total, scanned over blocks afterwards) and the exclusive offset of each
// kEmitSeg-record segment within its block. Records are loaded block-striped,
// so row j of the load holds segments 2j (warps 0-3) and 2j + 1 (warps 4-7).
__global__ void __launch_bounds__(kScanThreads) reduce_sorted_kernel(const unsigned long long* __restrict__ rkeys0,
                                                                     const unsigned long long* __restrict__ rkeys1,
                                                                     const SortCtl* __restrict__ ctl,
                                                                     uint32_t* __restrict__ sums,
                                                                     uint32_t* __restrict__ seg_off) {
    __shared__ uint32_t s_part[kScanItems][kScanThreads / 32];
    const uint32_t n = ctl->n_rec;
    const int buf = depth_buffer(ctl, kDepthPasses, n);
    const unsigned long long* rkeys = buf ? rkeys1 : rkeys0;
    if (blockIdx.x == 0 && threadIdx.x == 0) const_cast<SortCtl*>(ctl)->depth_buf = (uint32_t)buf;
    const long long base = (long long)blockIdx.x * kScanChunk;
    if (base >= n) {  // block-uniform: an empty block's sum is still scanned
        if (threadIdx.x == 0) sums[blockIdx.x] = 0u;
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long m = base + (long long)j * kScanThreads + threadIdx.x;
        const uint32_t c = m < n ? (uint32_t)(rkeys[m] >> 32) : 0u;
        const uint32_t w = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) s_part[j][wid] = w;
    }
    __syncthreads();
    if (wid == 0) {
        const int j = lane >> 1, h = 4 * (lane & 1);  // segment `lane` = half h / 4 of load row j
        const uint32_t seg = s_part[j][h] + s_part[j][h + 1] + s_part[j][h + 2] + s_part[j][h + 3];
        uint32_t incl = seg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        seg_off[(size_t)blockIdx.x * kSegsPerChunk + lane] = incl - seg;
        if (lane == 31) sums[blockIdx.x] = incl;
    }
}

// Pairs of the depth-sorted records, in that order, with the tile-digit
// histograms of the n_tile_passes tile passes. A resident grid: every warp
// takes kEmitSeg-record segments in turn (global warp index, then strided by
// the grid's warp count), so the work has no wave tail whatever the record
// count, and each block adds its histograms to the global ones once. A
// segment is taken as 4 rows of 32 records (one per lane); a row's pairs are
// dealt out to the lanes 32 at a time (pair k goes to lane k mod 32, which
// finds the record owning it by binary search over the row's inclusive
// counts), so every store is coalesced and a large splat does not hold up the
// other lanes. The next row's record gather is issued before the current row
// is dealt out.
// A pair's key: (tile << 32) | depth bits, or the tile id alone when the
// tile passes sort 32-bit keys.
template <typename K>
__device__ __forceinline__ K pair_key(uint32_t tile, uint32_t depth);
template <>
__device__ __forceinline__ unsigned long long pair_key<unsigned long long>(uint32_t tile, uint32_t depth) {
    return ((unsigned long long)tile << 32) | depth;
}
template <>
__device__ __forceinline__ uint32_t pair_key<uint32_t>(uint32_t tile, uint32_t) {
    return tile;
}

template <typename K>
__global__ void __launch_bounds__(kScanThreads, kEmitBlocksPerSm) emit_kernel(
    const unsigned long long* __restrict__ rkeys0, const uint32_t* __restrict__ rvals0,
    const unsigned long long* __restrict__ rkeys1, const uint32_t* __restrict__ rvals1,
    const float4* __restrict__ xyd, int n, int n_views, const gsfit_camera* __restrict__ cams_g,
    const uint32_t* __restrict__ sums, const uint32_t* __restrict__ seg_off, SortCtl* __restrict__ ctl,
    int n_tile_passes, K* __restrict__ keys, uint32_t* __restrict__ vals) {
    constexpr int kRows = kEmitSeg / 32;
    extern __shared__ gsfit_camera cams[];
    __shared__ uint32_t s_hist[kMaxPasses - kDepthPasses][kRadix];
    const uint32_t n_recs = ctl->n_rec;
    const long long n_segs = ((long long)n_recs + kEmitSeg - 1) / kEmitSeg;
    const long long warps = (long long)gridDim.x * (kScanThreads / 32);
    const bool second = ctl->depth_buf != 0u;
    const unsigned long long* rkeys = second ? rkeys1 : rkeys0;
    const uint32_t* rvals = second ? rvals1 : rvals0;
    if ((long long)blockIdx.x * (kScanThreads / 32) >= n_segs) return;  // block-uniform
    load_cameras(cams, cams_g, n_views);
    for (int k = threadIdx.x; k < n_tile_passes * kRadix; k += blockDim.x) (&s_hist[0][0])[k] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (long long seg = (long long)blockIdx.x * (kScanThreads / 32) + (threadIdx.x >> 5); seg < n_segs;
         seg += warps) {
        const long long sbase = seg * kEmitSeg;
        uint32_t offset = __ldg(sums + seg / kSegsPerChunk) + __ldg(seg_off + seg);
        unsigned long long key[kRows];
        uint32_t rec[kRows];
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const long long m = sbase + 32 * j + lane;
            const bool ok = m < (long long)n_recs;
            key[j] = ok ? __ldg(rkeys + m) : 0ull;
            rec[j] = ok ? __ldg(rvals + m) : 0u;
        }
        float4 p_next = (key[0] >> 32) > 0ull ? __ldg(xyd + rec[0]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
            const uint32_t c = (uint32_t)(key[j] >> 32);
            uint32_t inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t row = __shfl_sync(0xffffffffu, inc, 31);
            const float4 p = p_next;
            if (j + 1 < kRows && (key[j + 1] >> 32) > 0ull) p_next = __ldg(xyd + rec[j + 1]);
            if (row == 0u) continue;  // warp-uniform
            // this lane's record: first tile id, tiles across the camera, rect width, depth, Gaussian index
            uint32_t t0 = 0u, txn = 0u, rw = 1u, depth = 0u, gi = 0u;
            if (c > 0u) {
                const uint32_t r = rec[j];
                const uint32_t v = r / (uint32_t)n;
                gi = r - v * (uint32_t)n;
                const gsfit_camera& cam = cams[v];
                const int tx = tiles_x_of(cam);
                const Rect rc = tile_rect(p.x, p.y, p.w, tx, tiles_y_of(cam), tile_of(cam));
                txn = (uint32_t)tx;
                rw = (uint32_t)max(rc.x1 - rc.x0, 1);
                t0 = (uint32_t)(cam.tile_offset + rc.y0 * tx + rc.x0);
                depth = (uint32_t)key[j];
            }
            const uint32_t excl = inc - c;
            for (uint32_t k0 = 0; k0 < row; k0 += 32) {
                const uint32_t k = k0 + (uint32_t)lane;
                int owner = 0;  // lanes whose inclusive count is <= k
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t x = __shfl_sync(0xffffffffu, inc, owner + step - 1);
                    if (x <= k) owner += step;
                }
                const uint32_t o_t0 = __shfl_sync(0xffffffffu, t0, owner);
                const uint32_t o_txn = __shfl_sync(0xffffffffu, txn, owner);
                const uint32_t o_rw = __shfl_sync(0xffffffffu, rw, owner);
                const uint32_t o_depth = __shfl_sync(0xffffffffu, depth, owner);
                const uint32_t o_gi = __shfl_sync(0xffffffffu, gi, owner);
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, owner);
                if (k < row) {
                    const uint32_t q = k - o_excl;  // row-major position in the owner's rect
                    uint32_t dy = (uint32_t)((float)q * __frcp_rn((float)o_rw));
                    if (dy * o_rw > q) --dy;  // exact floor(q / rw) after the float estimate
                    else if ((dy + 1u) * o_rw <= q) ++dy;
                    const uint32_t tile = o_t0 + dy * o_txn + (q - dy * o_rw);
                    keys[offset + k] = pair_key<K>(tile, o_depth);
                    vals[offset + k] = o_gi;
                    for (int p = 0; p < n_tile_passes; ++p) atomicAdd(&s_hist[p][(tile >> (8 * p)) & 0xff], 1u);
                }
            }
            offset += row;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_tile_passes * kRadix; k += blockDim.x) {
        const uint32_t c = (&s_hist[0][0])[k];
        if (c) atomicAdd(&ctl->hist[kDepthPasses][0] + k, c);
    }
}

// Exclusive prefix of digit d over partitions [0, p], looked up kLookWindow
// partitions per round trip: the window's words are read together and
// consumed newest first while they carry a flag, up to the first inclusive
// prefix. A window whose newest word carries no flag is polled again after
// ~100 ns, at most `limit` times in a row (then GSFIT_ERR_TIMEOUT). With
// p = 0 only lb[d] is read.
constexpr int kLookWindow = 8;
__device__ __forceinline__ void lookback_window(const uint32_t* lb, int p, int d, uint32_t& excl,
                                                int32_t* status, int limit = kSpinLimit) {
    int idle = 0;
    while (p >= 0) {
        uint32_t f[kLookWindow];
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w)
            f[w] = p - w >= 0 ? *reinterpret_cast<const volatile uint32_t*>(&lb[(size_t)(p - w) * kRadix + d])
                              : 0u;
        int used = 0;
        bool inc = false;
#pragma unroll
        for (int w = 0; w < kLookWindow; ++w) {
            if (used == w && p - w >= 0 && (f[w] & (kFlagInc | kFlagAgg))) {
                excl += f[w] & kValMask;
                inc = (f[w] & kFlagInc) != 0u;
                used = inc ? kLookWindow + 1 : w + 1;  // stop consuming after an inclusive prefix
            }
        }
        if (inc) return;
        if (used == 0) {
            if (++idle > limit) {
                if (status) atomicExch(status, GSFIT_ERR_TIMEOUT);
                return;
            }
            __nanosleep(100);
        } else {
            idle = 0;
            p -= used;
        }
    }
}

// Diagnostic: polls a look-back word nothing will ever set.
__global__ void lookback_selftest_kernel(const uint32_t* word, int limit, int32_t* status) {
    uint32_t excl = 0;
    lookback_window(word, 0, 0, excl, status, limit);  // partition 0's word of digit 0: word[0] only
}

// K: the key type, 64-bit (the depth passes' (tile count, depth) records, and
// the tile passes when the sorted keys are an output) or 32-bit (the tile
// passes over tile ids alone).
template <typename K>
struct OnesweepSmem {
    K keys[kPart];
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
template <typename K>
__global__ void __launch_bounds__(kSortThreads, 3) onesweep_kernel(K* keys_a, uint32_t* vals_a, K* keys_b,
                                                                uint32_t* vals_b,
                                                                SortCtl* __restrict__ ctl, int pass, int shift,
                                                                const uint32_t* __restrict__ n_ptr,
                                                                uint32_t* __restrict__ lookback,
                                                                int32_t* __restrict__ status, int depth_pass) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem<K>& S = *reinterpret_cast<OnesweepSmem<K>*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t n = *n_ptr;
    const uint32_t n_parts = (n + kPart - 1) / kPart;
    const uint32_t hist_d = ctl->hist[pass][threadIdx.x];  // this pass's count of digit threadIdx.x
    if (threadIdx.x == 0) S.part = atomicAdd(&ctl->part_counter[pass], 1u);
    for (int k = threadIdx.x; k < kSortWarps * (kRadix + 1); k += kSortThreads) (&S.warp_hist[0][0])[k] = 0u;
    // one digit value holding every key: the stable pass is the identity permutation
    const bool identity = __syncthreads_or(hist_d == n) != 0;
    // input a, output b; a depth pass reads where the last pass that moved the
    // records left them (buffer a or b), and an identity depth pass leaves them there
    bool swap = false;
    if (depth_pass) {
        if (identity) return;
        swap = depth_buffer(ctl, pass, n) != 0;
    }
    const K* __restrict__ keys_in = swap ? keys_b : keys_a;
    const uint32_t* __restrict__ vals_in = swap ? vals_b : vals_a;
    K* __restrict__ keys_out = swap ? keys_a : keys_b;
    uint32_t* __restrict__ vals_out = swap ? vals_a : vals_b;
    const uint32_t part = S.part;
    if (part >= n_parts) return;
    const uint32_t base = part * kPart;
    const uint32_t valid = min((uint32_t)kPart, n - base);
    if (identity) {  // block-uniform: copy the partition in place of ranking it
        K kc[kSortItems];
        uint32_t vc[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t idx = (uint32_t)j * kSortThreads + threadIdx.x;
            if (idx < valid) {
                kc[j] = keys_in[base + idx];
                vc[j] = vals_in[base + idx];
            }
        }
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t idx = (uint32_t)j * kSortThreads + threadIdx.x;
            if (idx < valid) {
                keys_out[base + idx] = kc[j];
                vals_out[base + idx] = vc[j];
            }
        }
        return;
    }

    // Load (warp-striped, coalesced) and rank within the warp per digit. Keys
    // stay in registers; values wait in shared memory in input order.
    K k_reg[kSortItems];
    uint32_t r_reg[kSortItems];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t idx = (uint32_t)wid * (32 * kSortItems) + j * 32 + lane;
        const bool ok = idx < valid;
        k_reg[j] = ok ? keys_in[base + idx] : static_cast<K>(~static_cast<K>(0));
        if (ok) S.vals_in[idx] = vals_in[base + idx];
    }
    // global exclusive offset of digit threadIdx.x over all keys of this pass
    // (while the loads are in flight)
    uint32_t htot;
    S.glob_off[threadIdx.x] = block_excl_scan(hist_d, S.scan_warp, htot);
    // digit of item j; items past the end go to bin kRadix
    auto digit = [&](int j) -> uint32_t {
        const uint32_t idx = (uint32_t)wid * (32 * kSortItems) + j * 32 + lane;
        return idx < valid ? (uint32_t)((k_reg[j] >> shift) & 0xff) : (uint32_t)kRadix;
    };
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t d = digit(j);
        // lanes holding the same digit: one ballot per digit bit (bit 8 marks
        // padding), a constant cost where match.any grows with the number of
        // distinct digits in the warp
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const uint32_t vote = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? vote : ~vote;
        }
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
        lookback_window(lb, (int)part - 1, d, excl, status);
        atomicExch(&lb[(size_t)part * kRadix + d], kFlagInc | (excl + dcount));
    }
    S.glob_off[d] += excl - lstart;
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
        const K key = S.keys[j];
        const uint32_t dd = (uint32_t)((key >> shift) & 0xff);
        const uint32_t o = S.glob_off[dd] + j;
        if (o < n) {  // always true unless a look-back wait ran out
            keys_out[o] = key;
            vals_out[o] = S.vals[j];
        }
    }
}

// [first, last + 1) of each tile from adjacent sorted keys. A resident grid
// strides over chunks of 256 kRangeItems keys, kRangeItems per thread
// (block-striped), with all of a chunk's loads issued before any compare.
constexpr int kRangeItems = 4;
constexpr int kRangeBlocksPerSm = 8;
// hi: the sorted keys' tile ids, one every `stride` words (the upper word of
// each 64-bit key, or each 32-bit key).
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ hi, int stride,
                                                     const SortCtl* __restrict__ ctl,
                                                     uint32_t* __restrict__ ranges, uint32_t total_tiles) {
    const uint32_t n = ctl->n_sort;
    for (long long base = (long long)blockIdx.x * (256 * kRangeItems) + threadIdx.x; base < n;
         base += (long long)gridDim.x * (256 * kRangeItems)) {
        uint32_t t[kRangeItems], prev[kRangeItems], next[kRangeItems];
#pragma unroll
        for (int i = 0; i < kRangeItems; ++i) {
            const long long k = base + 256 * i;
            t[i] = k < n ? __ldg(hi + stride * k) : 0xffffffffu;
            prev[i] = k < n && k > 0 ? __ldg(hi + stride * (k - 1)) : 0xffffffffu;
            next[i] = k + 1 < n ? __ldg(hi + stride * (k + 1)) : 0xffffffffu;
        }
#pragma unroll
        for (int i = 0; i < kRangeItems; ++i) {
            const long long k = base + 256 * i;
            if (k >= n || t[i] >= total_tiles) continue;  // past the end, or only after a failed sort
            if (k == 0 || prev[i] != t[i]) ranges[2 * (size_t)t[i]] = (uint32_t)k;
            if (k + 1 == n || next[i] != t[i]) ranges[2 * (size_t)t[i] + 1] = (uint32_t)(k + 1);
        }
    }
}

// Heavy-first tile order: tiles bucketed by their expected work, buckets in
// decreasing order, tiles within a bucket in any order. A tile's work is the
// number of list entries its compositing walks: up to the furthest
// contributor the previous forward pass recorded in this order buffer (a
// quarter octave predicts a tile's time far better than its list length:
// correlation 0.96 against 0.76 on the bench workload, where the scene moves
// little from one iteration to the next), capped at the current list length,
// or the list length where none was recorded (the first iteration, a tile
// that was empty). Bucket 0 holds exactly the empty tiles, the others are
// 1 + the quarter octave of the work (at most kOrderBuckets - 1).
__device__ __forceinline__ int work_bucket(const uint32_t* ranges, const uint32_t* prev, int t) {
    const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
    if (len == 0u) return 0;
    const uint32_t k = prev[t];
    return min(kOrderBuckets - 1, 1 + quarter_octave(k != 0u && k < len ? k : len));
}

__global__ void __launch_bounds__(256) order_hist_kernel(const uint32_t* __restrict__ ranges, int total_tiles,
                                                         const uint32_t* __restrict__ prev, SortCtl* __restrict__ ctl) {
    __shared__ uint32_t h[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x)
        atomicAdd(&h[work_bucket(ranges, prev, t)], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) atomicAdd(&ctl->order_hist[threadIdx.x], h[threadIdx.x]);
}

// Also writes, after the permutation, the number of non-empty tiles (bucket
// 0 holds exactly the empty ones, placed last), and zeroes each tile's
// furthest-contributor word, which the forward pass raises.
__global__ void __launch_bounds__(256) order_scatter_kernel(const uint32_t* __restrict__ ranges, int total_tiles,
                                                            SortCtl* __restrict__ ctl,
                                                            uint32_t* __restrict__ tile_order) {
    __shared__ uint32_t off[kOrderBuckets];
    if (threadIdx.x == 0) {
        uint32_t o = 0;
        for (int b = kOrderBuckets - 1; b >= 0; --b) {
            off[b] = o;
            o += ctl->order_hist[b];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tile_order[total_tiles] = (uint32_t)total_tiles - ctl->order_hist[0];
    // per 256 tiles: bucket counts in shared memory, then one global
    // reservation per (block, bucket)
    __shared__ uint32_t cnt[kOrderBuckets], res[kOrderBuckets];
    const uint32_t* prev = tile_order + total_tiles + 1;  // each tile's word is read here before it is zeroed
    for (int t0 = blockIdx.x * blockDim.x; t0 < total_tiles; t0 += gridDim.x * blockDim.x) {
        if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0u;
        __syncthreads();
        const int t = t0 + threadIdx.x;
        const int b = t < total_tiles ? work_bucket(ranges, prev, t) : 0;
        const uint32_t local = t < total_tiles ? atomicAdd(&cnt[b], 1u) : 0u;
        __syncthreads();
        if (threadIdx.x < kOrderBuckets && cnt[threadIdx.x])
            res[threadIdx.x] = atomicAdd(&ctl->order_fill[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (t < total_tiles) {
            tile_order[off[b] + res[b] + local] = (uint32_t)t;
            tile_order[total_tiles + 1 + t] = 0u;
        }
        __syncthreads();
    }
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct SortLayout {
    size_t pair_sums, rec_sums, sorted_sums, seg_off, ctl, lookback, keys_alt, vals_alt, rkeys[2], rvals[2], total;
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
    L.seg_off = o; o = align_up(o + sizeof(uint32_t) * (size_t)L.n_blocks * kSegsPerChunk);
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

// Opt-in to more than 48 KB of dynamic shared memory, once per device and context.
template <typename K>
int enable_onesweep_smem() {
    static ContextOnce once;
    return opt_in_smem(once, onesweep_kernel<K>, sizeof(OnesweepSmem<K>));
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
        !ws || !vals || !n_instances || !ranges || !status || capacity < 1 ||
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
    const bool narrow = keys == nullptr;  // the tile passes sort 32-bit tile ids; no keys are written
    const size_t smem = sizeof(OnesweepSmem<unsigned long long>), smem32 = sizeof(OnesweepSmem<uint32_t>);
    int rc = enable_onesweep_smem<unsigned long long>();
    if (rc == GSFIT_OK && narrow) rc = enable_onesweep_smem<uint32_t>();
    if (rc != GSFIT_OK) return rc;

    reduce_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(proj->tiles, n_rec, pair_sums, rec_sums);
    GSFIT_LAUNCH_CHECK();
    scan_kernel<<<1, 1024, 0, stream>>>(pair_sums, rec_sums, L.n_blocks, ctl, n_instances, capacity, status);
    GSFIT_LAUNCH_CHECK();
    compact_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(proj->tiles, reinterpret_cast<const float4*>(proj->xyd),
                                                            n_rec, rec_sums, ctl, rk[0], rv[0], lookback,
                                                            L.lookback_words, ranges, 2ll * total_tiles);
    GSFIT_LAUNCH_CHECK();
    // depth passes over the records, between buffers 0 and 1 (which one holds the
    // result depends on how many passes were identities; the kernels after them check)
    uint32_t* lb = lookback;
    for (int p = 0; p < kDepthPasses; ++p) {
        onesweep_kernel<unsigned long long><<<(unsigned)L.max_rec_parts, kSortThreads, smem, stream>>>(
            rk[0], rv[0], rk[1], rv[1], ctl, p, 8 * p, &ctl->n_rec, lb, status, 1);
        GSFIT_LAUNCH_CHECK();
        lb += (size_t)L.max_rec_parts * kRadix;
    }
    uint32_t* seg_off = reinterpret_cast<uint32_t*>(base + L.seg_off);
    reduce_sorted_kernel<<<L.n_blocks, kScanThreads, 0, stream>>>(rk[0], rk[1], ctl, sorted_sums, seg_off);
    GSFIT_LAUNCH_CHECK();
    scan_blocks_kernel<<<1, 1024, 0, stream>>>(sorted_sums, L.n_blocks);
    GSFIT_LAUNCH_CHECK();
    // pairs go to the buffer that, after the tile passes' ping-pong, leaves the result in keys/vals
    const bool emit_to_alt = (L.tile_passes % 2) == 1;
    uint32_t* v_cur = emit_to_alt ? vals_alt : vals;
    uint32_t* v_nxt = emit_to_alt ? vals : vals_alt;
    int dev = 0, sms = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long segs = (long long)L.n_blocks * kSegsPerChunk;
    const unsigned emit_grid = (unsigned)std::min<long long>((long long)kEmitBlocksPerSm * sms, (segs + 7) / 8);
    const unsigned range_grid = (unsigned)std::min<long long>((long long)kRangeBlocksPerSm * sms,
                                                              (capacity + 256 * kRangeItems - 1) / (256 * kRangeItems));
    if (narrow) {  // 32-bit keys in the two halves of the alternate key buffer
        uint32_t* k_cur = reinterpret_cast<uint32_t*>(keys_alt);
        uint32_t* k_nxt = k_cur + capacity;
        emit_kernel<uint32_t><<<emit_grid, kScanThreads, sizeof(gsfit_camera) * n_views, stream>>>(
            rk[0], rv[0], rk[1], rv[1], reinterpret_cast<const float4*>(proj->xyd), n, n_views, cams, sorted_sums,
            seg_off, ctl, L.tile_passes, k_cur, v_cur);
        GSFIT_LAUNCH_CHECK();
        for (int q = 0; q < L.tile_passes; ++q) {
            onesweep_kernel<uint32_t><<<(unsigned)L.max_parts, kSortThreads, smem32, stream>>>(
                k_cur, v_cur, k_nxt, v_nxt, ctl, kDepthPasses + q, 8 * q, &ctl->n_sort, lb, status, 0);
            GSFIT_LAUNCH_CHECK();
            lb += (size_t)L.max_parts * kRadix;
            std::swap(k_cur, k_nxt);
            std::swap(v_cur, v_nxt);
        }
        ranges_kernel<<<range_grid, 256, 0, stream>>>(k_cur, 1, ctl, ranges, (uint32_t)total_tiles);
        GSFIT_LAUNCH_CHECK();
    } else {
        unsigned long long* k_cur = emit_to_alt ? keys_alt : keys_out;
        unsigned long long* k_nxt = emit_to_alt ? keys_out : keys_alt;
        emit_kernel<unsigned long long><<<emit_grid, kScanThreads, sizeof(gsfit_camera) * n_views, stream>>>(
            rk[0], rv[0], rk[1], rv[1], reinterpret_cast<const float4*>(proj->xyd), n, n_views, cams, sorted_sums,
            seg_off, ctl, L.tile_passes, k_cur, v_cur);
        GSFIT_LAUNCH_CHECK();
        for (int q = 0; q < L.tile_passes; ++q) {
            onesweep_kernel<unsigned long long><<<(unsigned)L.max_parts, kSortThreads, smem, stream>>>(
                k_cur, v_cur, k_nxt, v_nxt, ctl, kDepthPasses + q, 32 + 8 * q, &ctl->n_sort, lb, status, 0);
            GSFIT_LAUNCH_CHECK();
            lb += (size_t)L.max_parts * kRadix;
            std::swap(k_cur, k_nxt);
            std::swap(v_cur, v_nxt);
        }
        ranges_kernel<<<range_grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t*>(keys_out) + 1, 2, ctl, ranges,
                                                      (uint32_t)total_tiles);
        GSFIT_LAUNCH_CHECK();
    }
    if (tile_order) {
        const int ob = min(152, (total_tiles + 255) / 256);
        order_hist_kernel<<<ob, 256, 0, stream>>>(ranges, total_tiles, tile_order + total_tiles + 1, ctl);
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
