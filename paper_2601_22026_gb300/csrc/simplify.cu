// Simplification of a Gaussian set by importance (the abbreviated
// regeneration of Section 4.2 simplifies after 95 steps; the rule read here is
// importance = accumulated blend weight, keep the `keep` most important).
//
// The threshold is found without sorting: importance values are non-negative
// floats, so their bit patterns order like the values. A 65536-bin histogram
// of the high 16 bits locates the bin holding the keep-th largest value, a
// second histogram of the low 16 bits inside that bin locates the value
// itself; every Gaussian at or above it is kept (ties at the threshold are
// all kept). The kept Gaussians are then compacted in index order with a
// reduce-then-scan (per-block counts, one scan block, per-block rescans).
#include <algorithm>

#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kBins = 65536;
constexpr int kChunk = 4096;  // Gaussians per block in the compaction
constexpr int kThreads = 256;

struct SimplifyCtl {
    uint32_t bin;        // high 16 bits of the threshold
    uint32_t above;      // Gaussians in higher bins
    uint32_t threshold;  // bit pattern of the threshold importance
    uint32_t n_out;
};

__device__ __forceinline__ uint32_t imp_bits(float x) {
    return x > 0.0f ? __float_as_uint(x) : 0u;  // -0, NaN and negatives count as 0
}

__global__ void __launch_bounds__(kThreads) clear_kernel(uint32_t* __restrict__ w, int words) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < words; k += gridDim.x * blockDim.x) w[k] = 0u;
}

__global__ void __launch_bounds__(kThreads) hist_hi_kernel(const float* __restrict__ imp, int n,
                                                           uint32_t* __restrict__ hist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&hist[imp_bits(imp[i]) >> 16], 1u);
}

__global__ void __launch_bounds__(kThreads) hist_lo_kernel(const float* __restrict__ imp, int n,
                                                           const SimplifyCtl* __restrict__ ctl,
                                                           uint32_t* __restrict__ hist) {
    const uint32_t bin = ctl->bin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t b = imp_bits(imp[i]);
        if ((b >> 16) == bin) atomicAdd(&hist[b & 0xffffu], 1u);
    }
}

// One 1024-thread block: the largest bin b with base (already counted above)
// + (count in bins >= b) >= keep, and the count in bins > b (plus base); bin
// 0xffffffff if even all bins fall short. Threads own 64 consecutive bins.
// Every thread returns the same values.
__device__ void select_bin(const uint32_t* __restrict__ hist, uint32_t keep, uint32_t base, uint32_t& bin_out,
                           uint32_t& above_out) {
    __shared__ uint32_t s_sum[1024];
    __shared__ uint32_t s_pick, s_above;
    const int t = threadIdx.x;
    uint32_t local = 0;
    for (int k = 0; k < 64; ++k) local += hist[64 * t + k];
    s_sum[t] = local;
    if (t == 0) {
        s_pick = 0xffffffffu;
        s_above = base;
    }
    __syncthreads();
    // suffix sums over threads (Hillis-Steele, from the top)
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t add = t + o < 1024 ? s_sum[t + o] : 0u;
        __syncthreads();
        s_sum[t] += add;
        __syncthreads();
    }
    const uint32_t incl = base + s_sum[t];                             // in bins >= 64 t
    const uint32_t excl = t + 1 < 1024 ? base + s_sum[t + 1] : base;  // in bins >= 64 (t + 1)
    if (excl < keep && incl >= keep) {  // exactly one thread
        uint32_t acc = excl;
        for (int k = 63; k >= 0; --k) {
            const uint32_t c = hist[64 * t + k];
            if (acc + c >= keep) {
                s_pick = (uint32_t)(64 * t + k);
                s_above = acc;
                break;
            }
            acc += c;
        }
    }
    __syncthreads();
    bin_out = s_pick;
    above_out = s_above;
}

__global__ void __launch_bounds__(1024) select_hi_kernel(const uint32_t* __restrict__ hist, uint32_t keep,
                                                         SimplifyCtl* __restrict__ ctl) {
    uint32_t bin = 0, above = 0;
    select_bin(hist, keep, 0u, bin, above);
    if (threadIdx.x == 0) {
        const bool all = bin == 0xffffffffu;  // fewer than keep Gaussians: keep all
        ctl->bin = all ? 0u : bin;
        ctl->above = all ? 0u : above;
    }
}

__global__ void __launch_bounds__(1024) select_lo_kernel(const uint32_t* __restrict__ hist, uint32_t keep,
                                                         SimplifyCtl* __restrict__ ctl) {
    uint32_t lo = 0, above = 0;
    const uint32_t bin = ctl->bin;
    select_bin(hist, keep, ctl->above, lo, above);
    if (threadIdx.x == 0) ctl->threshold = (bin << 16) | (lo == 0xffffffffu ? 0u : lo);
}

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
    for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t s = s_warp[w];
        if (w < wid) wpre += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + incl - x;
}

__global__ void __launch_bounds__(kThreads) count_kernel(const float* __restrict__ imp, int n,
                                                         const SimplifyCtl* __restrict__ ctl,
                                                         uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const uint32_t t = ctl->threshold;
    uint32_t c = 0;
    for (int k = 0; k < kChunk / kThreads; ++k) {
        const int i = blockIdx.x * kChunk + k * kThreads + threadIdx.x;
        if (i < n && imp_bits(imp[i]) >= t) ++c;
    }
    uint32_t total;
    block_excl_scan(c, s_warp, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_kernel(uint32_t* __restrict__ sums, int n_blocks,
                                                    SimplifyCtl* __restrict__ ctl, uint32_t* __restrict__ n_out) {
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_warp[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0u;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += 1024) {
        const int b = base + threadIdx.x;
        const uint32_t x = b < n_blocks ? sums[b] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        uint32_t wpre = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < wid) wpre += s_warp[w];
            tot += s_warp[w];
        }
        const uint32_t carry = s_carry;
        if (b < n_blocks) sums[b] = carry + wpre + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->n_out = s_carry;
        *n_out = s_carry;
    }
}

__global__ void __launch_bounds__(kThreads) scatter_kernel(const float4* __restrict__ params, int n, int n_planes,
                                                           const float* __restrict__ imp,
                                                           const SimplifyCtl* __restrict__ ctl,
                                                           const uint32_t* __restrict__ block_sums,
                                                           float4* __restrict__ out) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const uint32_t t = ctl->threshold;
    uint32_t offset = block_sums[blockIdx.x];
    for (int k = 0; k < kChunk / kThreads; ++k) {
        const int i = blockIdx.x * kChunk + k * kThreads + threadIdx.x;
        const uint32_t keep = (i < n && imp_bits(imp[i]) >= t) ? 1u : 0u;
        uint32_t row;
        const uint32_t ex = block_excl_scan(keep, s_warp, row);
        if (keep) {
            const size_t m = offset + ex;
            for (int p = 0; p < n_planes; ++p) out[(size_t)p * n + m] = params[(size_t)p * n + i];
        }
        offset += row;
    }
}

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" size_t gsfit_simplify_workspace_size(int32_t n) {
    if (n < 1) return 0;
    const size_t blocks = (size_t)(n + kChunk - 1) / kChunk;
    return sizeof(uint32_t) * (2 * (size_t)kBins + blocks) + 256;
}

extern "C" int gsfit_simplify(const float* params, int32_t n, int32_t n_planes, const float* importance,
                              int32_t keep, float* params_out, uint32_t* n_out, void* ws, size_t ws_bytes,
                              cudaStream_t stream) {
    if (!params || !importance || !params_out || !n_out || !ws || n < 1 || n_planes < 1 || n_planes > 16 ||
        keep < 1 || ws_bytes < gsfit_simplify_workspace_size(n) || (reinterpret_cast<uintptr_t>(params) % 16) ||
        (reinterpret_cast<uintptr_t>(params_out) % 16) || (reinterpret_cast<uintptr_t>(ws) % 16) ||
        params_out == params)
        return GSFIT_ERR_INVALID_ARG;
    uint32_t* hist_hi = static_cast<uint32_t*>(ws);
    uint32_t* hist_lo = hist_hi + kBins;
    const int n_blocks = (n + kChunk - 1) / kChunk;
    uint32_t* block_sums = hist_lo + kBins;
    SimplifyCtl* ctl = reinterpret_cast<SimplifyCtl*>(block_sums + ((n_blocks + 3) & ~3));
    const int grid = (int)std::min<long long>(((long long)n + kThreads - 1) / kThreads, 4096);
    clear_kernel<<<256, kThreads, 0, stream>>>(hist_hi, 2 * kBins);
    GSFIT_LAUNCH_CHECK();
    hist_hi_kernel<<<grid, kThreads, 0, stream>>>(importance, n, hist_hi);
    GSFIT_LAUNCH_CHECK();
    select_hi_kernel<<<1, 1024, 0, stream>>>(hist_hi, (uint32_t)keep, ctl);
    GSFIT_LAUNCH_CHECK();
    hist_lo_kernel<<<grid, kThreads, 0, stream>>>(importance, n, ctl, hist_lo);
    GSFIT_LAUNCH_CHECK();
    select_lo_kernel<<<1, 1024, 0, stream>>>(hist_lo, (uint32_t)keep, ctl);
    GSFIT_LAUNCH_CHECK();
    count_kernel<<<n_blocks, kThreads, 0, stream>>>(importance, n, ctl, block_sums);
    GSFIT_LAUNCH_CHECK();
    scan_kernel<<<1, 1024, 0, stream>>>(block_sums, n_blocks, ctl, n_out);
    GSFIT_LAUNCH_CHECK();
    scatter_kernel<<<n_blocks, kThreads, 0, stream>>>(reinterpret_cast<const float4*>(params), n, n_planes,
                                                      importance, ctl, block_sums, reinterpret_cast<float4*>(params_out));
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
