// Front-to-back compositing of the tile lists and its back-to-front adjoint.
//
// The peripheral model is rendered and trained as 3DGS with an alpha output
// for alpha supervision (Section 4.2). Per pixel, over its tile's sorted
// range: power = -1/2 (a' dx^2 + c' dy^2) - b' dx dy (skip if > 0), alpha =
// min(0.99, o exp(power)) (skip if < 1/255), stop before T would drop below
// 1e-4, C = sum c alpha T + T_N bg, A = 1 - T_N.
//
// Design: one 256-thread CTA per 16 x 16 tile, one pixel per thread; warp w
// owns an 8 x 4 pixel box (two boxes across, four down). Tiles are launched in
// the heavy-first order gsfit_bin_sort produces, so the longest lists do not
// form the tail of the grid. The CTA stages the tile's records in batches of
// 256 (one coalesced record per thread); each warp then compacts, with a
// ballot, the batch entries whose opacity-aware extent can reach alpha >=
// 1/255 somewhere in its box (a conservative test: every pixel of the box
// would skip the others anyway) and walks only those. The adjoint copies the
// next batch with cp.async while it works on the current one (the forward, which
// often stops early, stages one batch at a time). The adjoint
// keeps no per-(pixel, Gaussian) state: it restarts from the stored final
// transmittance and contributor count and recovers T_i = T_{i+1} / (1 -
// alpha_i) walking backwards, and sums the nine per-Gaussian gradient terms of
// the warp with a transposed butterfly (12 shuffles instead of 45) that
// leaves each total in its own lane, so one predicated scalar-atomic
// instruction of nine lanes accumulates them.
#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kRenderThreads = kTilePixels;  // one pixel per thread
constexpr int kRenderWarps = kRenderThreads / 32;
constexpr int kBatch = kRenderThreads;       // records staged per batch
constexpr float kCullMargin = 0.02f;         // slack (units of the quadratic form) of the warp cull

// This thread's pixel: warp w covers the 8 x 4 box at (8 (w mod 2), 4 (w / 2))
// of the tile, lane l its pixel (l mod 8, l / 8).
struct TileCtx {
    int view, px, py;
    bool inside;
    long long pix, plane, rgb_base;
    float box_cx, box_cy;  // centre of the warp's box of pixel centres
};

__device__ __forceinline__ TileCtx tile_ctx(const gsfit_camera* cams, int n_views, int t) {
    TileCtx c;
    c.view = view_of_tile(cams, n_views, t);
    const gsfit_camera& cam = cams[c.view];
    const int local = t - cam.tile_offset;
    const int txn = tiles_x_of(cam);
    const int ty = local / txn, tx = local - ty * txn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int bx = (w & 1) * 8, by = (w >> 1) * 4;
    c.px = tx * kTile + bx + (lane & 7);
    c.py = ty * kTile + by + (lane >> 3);
    c.inside = c.px < cam.width && c.py < cam.height;
    c.plane = (long long)cam.width * cam.height;
    c.pix = (long long)cam.pixel_offset + (long long)c.py * cam.width + c.px;
    c.rgb_base = 3ll * cam.pixel_offset + (long long)c.py * cam.width + c.px;
    c.box_cx = (float)(tx * kTile + bx) + 3.5f;
    c.box_cy = (float)(ty * kTile + by) + 1.5f;
    return c;
}

// Half-extents of the region where a splat can reach alpha >= 1/255:
// o exp(-q/2) >= 1/255  <=>  q <= 2 ln(255 o), q the conic's quadratic form;
// the ellipse q <= t has half-widths sqrt(t Sigma'_xx), sqrt(t Sigma'_yy).
// Negative extents mark a splat that cannot reach the threshold anywhere.
__device__ __forceinline__ float2 alpha_extent(float4 co) {
    const float t = 2.0f * __logf(255.0f * co.w) + kCullMargin;
    if (!(t > 0.0f)) return make_float2(-1.f, -1.f);
    const float det = co.x * co.z - co.y * co.y;
    if (!(det > 0.0f)) return make_float2(1e30f, 1e30f);  // degenerate conic: never cull
    const float ex = sqrtf(t * co.z / det), ey = sqrtf(t * co.x / det);
    return make_float2(ex * 1.001f + 0.05f, ey * 1.001f + 0.05f);
}

// One batch of staged records (shared memory).
struct Batch {
    float2 xy[kBatch];
    float2 ext[kBatch];
    float4 co[kBatch];
    float4 col[kBatch];
    uint32_t g[kBatch];
};

// This thread stages list entry idx (if < end) into slot threadIdx.x.
__device__ __forceinline__ void stage(Batch& S, uint32_t idx, uint32_t end, const uint32_t* __restrict__ vals,
                                      const float4* __restrict__ xyd, const float4* __restrict__ conic,
                                      const float4* __restrict__ rgb, size_t rec0, int n) {
    const int t = threadIdx.x;
    uint32_t g = 0xffffffffu;
    if (idx < end) {
        g = __ldg(vals + idx);
        if (g >= (uint32_t)n) g = 0xffffffffu;  // only after a failed sort: never blended
    }
    if (g != 0xffffffffu) {
        const size_t k = rec0 + g;
        const float4 p = __ldg(xyd + k);
        const float4 co = __ldg(conic + k);
        S.xy[t] = make_float2(p.x, p.y);
        S.co[t] = co;
        S.col[t] = __ldg(rgb + k);
        S.ext[t] = alpha_extent(co);
    } else {
        S.ext[t] = make_float2(-1.f, -1.f);
    }
    S.g[t] = g;
}

// Can entry j reach alpha >= 1/255 at a pixel centre of this warp's box?
__device__ __forceinline__ bool box_hit(const Batch& S, int j, const TileCtx& c) {
    const float2 p = S.xy[j];
    const float2 e = S.ext[j];
    return e.x >= 0.0f && fabsf(p.x - c.box_cx) <= 3.5f + e.x && fabsf(p.y - c.box_cy) <= 1.5f + e.y;
}

// Double-buffered staging (adjoint): while the warps work on one batch,
// cp.async copies the next batch's 16-byte records (gathered by Gaussian index) into
// the other buffer; only the index of the batch after that occupies a
// register. Entries past the list end, or with an out-of-range index (which
// only a failed sort produces), are never copied and are culled.
struct Batch2 {
    float4 xyd[2][kBatch];
    float4 co[2][kBatch];
    float4 col[2][kBatch];
    float2 ext[2][kBatch];
    uint32_t g[2][kBatch];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ uint32_t load_index(uint32_t idx, uint32_t end, const uint32_t* __restrict__ vals, int n) {
    if (idx >= end) return 0xffffffffu;
    const uint32_t g = __ldg(vals + idx);
    return g < (uint32_t)n ? g : 0xffffffffu;
}

// This thread's copies of record g into slot threadIdx.x of buffer b.
__device__ __forceinline__ void issue_rec(Batch2& S, int b, uint32_t g, const float4* __restrict__ xyd,
                                          const float4* __restrict__ conic, const float4* __restrict__ rgb,
                                          size_t rec0) {
    if (g != 0xffffffffu) {
        const size_t k = rec0 + g;
        const int t = threadIdx.x;
        cp_async16(&S.xyd[b][t], xyd + k);
        cp_async16(&S.co[b][t], conic + k);
        cp_async16(&S.col[b][t], rgb + k);
    }
}

// After this thread's copies into buffer b have landed: its slot's extents.
__device__ __forceinline__ void finish_rec(Batch2& S, int b, uint32_t g) {
    const int t = threadIdx.x;
    S.ext[b][t] = g != 0xffffffffu ? alpha_extent(S.co[b][t]) : make_float2(-1.f, -1.f);
    S.g[b][t] = g;
}

__device__ __forceinline__ bool box_hit2(const Batch2& S, int b, int j, const TileCtx& c) {
    const float4 p = S.xyd[b][j];
    const float2 e = S.ext[b][j];
    return e.x >= 0.0f && fabsf(p.x - c.box_cx) <= 3.5f + e.x && fabsf(p.y - c.box_cy) <= 1.5f + e.y;
}

__global__ void __launch_bounds__(kRenderThreads) render_fwd_kernel(
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgb, int n,
    const gsfit_camera* __restrict__ cams_g, int n_views, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ tile_order, const float* __restrict__ bg,
    float* __restrict__ out_rgb,
    float* __restrict__ out_alpha, float* __restrict__ out_T, uint32_t* __restrict__ out_nc) {
    extern __shared__ gsfit_camera cams[];
    __shared__ Batch S;
    __shared__ uint8_t s_list[kRenderWarps][kBatch];
    load_cameras(cams, cams_g, n_views);
    __syncthreads();
    const int t = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileCtx c = tile_ctx(cams, n_views, t);
    const uint2 range = ranges[t];
    const size_t rec0 = (size_t)c.view * n;
    const float fx = (float)c.px, fy = (float)c.py;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !c.inside;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        stage(S, b0 + threadIdx.x, range.y, vals, xyd, conic, rgb, rec0, n);
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
        // this warp's entries of the batch, in list order
        int nw = 0;
        if (!__all_sync(0xffffffffu, done)) {
#pragma unroll
            for (int k = 0; k < kBatch / 32; ++k) {
                const int j = 32 * k + lane;
                const bool hit = j < cnt && box_hit(S, j, c);
                const uint32_t m = __ballot_sync(0xffffffffu, hit);
                if (hit) s_list[w][nw + __popc(m & lt)] = (uint8_t)j;
                nw += __popc(m);
            }
        }
        __syncwarp();
        for (int i = 0; i < nw; ++i) {
            const int j = s_list[w][i];
            if (!done) {
                const float2 p = S.xy[j];
                const float4 co = S.co[j];
                const float power = splat_power(co, fx - p.x, fy - p.y);
                if (power <= 0.0f) {
                    const float alpha = fminf(kAlphaClamp, co.w * __expf(power));
                    if (alpha >= kAlphaSkip) {
                        const float test_T = T * (1.0f - alpha);
                        if (test_T < kTStop) {
                            done = true;
                        } else {
                            const float4 col = S.col[j];
                            const float wgt = alpha * T;
                            C0 += col.x * wgt;
                            C1 += col.y * wgt;
                            C2 += col.z * wgt;
                            T = test_T;
                            last = b0 - range.x + (uint32_t)j + 1u;  // one past this list position
                        }
                    }
                }
            }
            if (__all_sync(0xffffffffu, done)) break;
        }
    }
    if (c.inside) {
        const float* bgv = bg + 3 * c.view;
        out_rgb[c.rgb_base] = C0 + T * bgv[0];
        out_rgb[c.rgb_base + c.plane] = C1 + T * bgv[1];
        out_rgb[c.rgb_base + 2 * c.plane] = C2 + T * bgv[2];
        out_alpha[c.pix] = 1.0f - T;
        out_T[c.pix] = T;
        out_nc[c.pix] = last;
    }
}

// Transposed butterfly sum of nine values over the warp (12 shuffles): at each
// level the two partner lanes split their remaining values in halves, each
// keeping one half and adding its partner's copy of it. Afterwards the lane
// pair (l, l ^ 1) holds the warp total of value reduce9_slot(l).
__device__ __forceinline__ float reduce9(const float* v, int lane) {
    const bool b1 = lane & 16, b2 = lane & 8, b3 = lane & 4, b4 = lane & 2;
    float w1[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float lo = v[k], hi = (k < 4) ? v[5 + k] : 0.f;
        const float r = __shfl_xor_sync(0xffffffffu, b1 ? lo : hi, 16);
        w1[k] = (b1 ? hi : lo) + r;
    }
    float w2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = w1[k], hi = (k < 2) ? w1[3 + k] : 0.f;
        const float r = __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 8);
        w2[k] = (b2 ? hi : lo) + r;
    }
    float w3[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float lo = w2[k], hi = (k < 1) ? w2[2 + k] : 0.f;
        const float r = __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 4);
        w3[k] = (b3 ? hi : lo) + r;
    }
    const float r4 = __shfl_xor_sync(0xffffffffu, b4 ? w3[0] : w3[1], 2);
    const float w4 = (b4 ? w3[1] : w3[0]) + r4;
    return w4 + __shfl_xor_sync(0xffffffffu, w4, 1);
}

// Index of the value whose total lane `lane` holds after reduce9 (-1: none, or
// the odd lane of a pair).
__device__ __forceinline__ int reduce9_slot(int lane) {
    const int b1 = (lane >> 4) & 1, b2 = (lane >> 3) & 1, b3 = (lane >> 2) & 1, b4 = (lane >> 1) & 1;
    const int s2 = 2 * b3 + b4;  // slot after level 2 (of 3)
    if (s2 >= 3) return -1;
    const int s1 = 3 * b2 + s2;  // slot after level 1 (of 5 or 4)
    if (s1 >= 5) return -1;
    const int idx = 5 * b1 + s1;
    if (idx >= 9) return -1;
    return (lane & 1) ? -1 : idx;
}

// Back-to-front state of one pixel.
struct PixBwd {
    float T, TN, S0, S1, S2, dC0, dC1, dC2, dA;
    uint32_t last;
};

// Adjoint of one blend at one pixel (list position pos < last), accumulating
// the nine per-Gaussian terms g9 = dL/d(u, v, opacity, a', b', c', r, g, b);
// returns whether the Gaussian was blended here.
__device__ __forceinline__ bool pix_bwd_step(PixBwd& q, uint32_t pos, float4 co, float4 col, float bg0, float bg1,
                                             float bg2, float dx, float dy, float* g9) {
    if (pos >= q.last) return false;
    const float power = splat_power(co, dx, dy);
    if (power > 0.0f) return false;
    const float G = __expf(power);
    const float a = co.w * G;
    const float alpha = fminf(kAlphaClamp, a);
    if (alpha < kAlphaSkip) return false;
    const float one_m = 1.0f - alpha;
    const float inv = 1.0f / one_m;
    q.T *= inv;  // transmittance in front of this Gaussian
    const float wT = alpha * q.T;
    g9[6] = q.dC0 * wT;
    g9[7] = q.dC1 * wT;
    g9[8] = q.dC2 * wT;
    // dC/dalpha = T c - (S + T_N bg) / (1 - alpha); dA/dalpha = T_N / (1 - alpha)
    const float dalpha = (q.dA * q.TN + q.dC0 * (q.T * col.x * one_m - (q.S0 + q.TN * bg0)) +
                          q.dC1 * (q.T * col.y * one_m - (q.S1 + q.TN * bg1)) +
                          q.dC2 * (q.T * col.z * one_m - (q.S2 + q.TN * bg2))) * inv;
    q.S0 += col.x * wT;
    q.S1 += col.y * wT;
    q.S2 += col.z * wT;
    if (a <= kAlphaClamp) {  // the clamped alpha depends on neither opacity nor power
        const float dpow = dalpha * alpha;
        g9[2] = dalpha * G;
        g9[0] = dpow * (co.x * dx + co.y * dy);
        g9[1] = dpow * (co.z * dy + co.y * dx);
        g9[3] = -0.5f * dpow * dx * dx;
        g9[4] = -dpow * dx * dy;
        g9[5] = -0.5f * dpow * dy * dy;
    }
    return true;
}

__global__ void __launch_bounds__(kRenderThreads) render_bwd_kernel(
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgb, int n,
    const gsfit_camera* __restrict__ cams_g, int n_views, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ tile_order, const float* __restrict__ bg,
    const float* __restrict__ T_final,
    const uint32_t* __restrict__ n_contrib, const float* __restrict__ dL_drgb, const float* __restrict__ dL_dalpha,
    float* __restrict__ grad2d) {
    extern __shared__ gsfit_camera cams[];
    __shared__ Batch2 S;
    __shared__ uint8_t s_list[kRenderWarps][kBatch];
    __shared__ uint32_t s_max;
    load_cameras(cams, cams_g, n_views);
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    const int t = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileCtx c = tile_ctx(cams, n_views, t);
    const uint2 range = ranges[t];
    const size_t rec0 = (size_t)c.view * n;
    const float fx = (float)c.px, fy = (float)c.py;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const float bg0 = bg[3 * c.view], bg1 = bg[3 * c.view + 1], bg2 = bg[3 * c.view + 2];
    const int slot = reduce9_slot(lane);
    const int slot_off = slot + slot / 3;  // floats (du dv do _ | da db dc _ | dr dg db _ | ....) of a record

    PixBwd q;
    q.T = 1.f; q.last = 0; q.dC0 = q.dC1 = q.dC2 = q.dA = 0.f;
    if (c.inside) {
        q.T = T_final[c.pix];
        q.last = n_contrib[c.pix];
        q.dC0 = dL_drgb[c.rgb_base];
        q.dC1 = dL_drgb[c.rgb_base + c.plane];
        q.dC2 = dL_drgb[c.rgb_base + 2 * c.plane];
        q.dA = dL_dalpha[c.pix];
    }
    q.TN = q.T;
    q.S0 = q.S1 = q.S2 = 0.f;
    // the warp's furthest contributor bounds its walk; the block's bounds the batches
    uint32_t wmax = q.last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const uint32_t end = range.x + min(s_max, range.y - range.x);

    // batches walk backwards, [b0, b1) with b1 - b0 <= kBatch, the last first;
    // the next one (towards the list start) is copied while this one runs
    uint32_t b1 = end;
    uint32_t b0 = (b1 - range.x > (uint32_t)kBatch) ? b1 - kBatch : range.x;
    uint32_t g_cur = load_index(b0 + threadIdx.x, b1, vals, n);
    issue_rec(S, 0, g_cur, xyd, conic, rgb, rec0);
    cp_async_commit();
    uint32_t pb1 = b0, pb0 = (pb1 - range.x > (uint32_t)kBatch) ? pb1 - kBatch : range.x;
    uint32_t g_next = pb1 > range.x ? load_index(pb0 + threadIdx.x, pb1, vals, n) : 0xffffffffu;
    int buf = 0;
    while (b1 > range.x) {
        __syncthreads();  // the other buffer is free again
        uint32_t nb1 = pb1, nb0 = pb0, g_after = 0xffffffffu;
        if (pb1 > range.x) {
            issue_rec(S, buf ^ 1, g_next, xyd, conic, rgb, rec0);
            cp_async_commit();
            nb1 = pb0;
            nb0 = (nb1 - range.x > (uint32_t)kBatch) ? nb1 - kBatch : range.x;
            g_after = nb1 > range.x ? load_index(nb0 + threadIdx.x, nb1, vals, n) : 0xffffffffu;
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        finish_rec(S, buf, g_cur);
        __syncthreads();
        const int cnt = (int)(b1 - b0);
        int nw = 0;
#pragma unroll
        for (int k = 0; k < kBatch / 32; ++k) {
            const int j = 32 * k + lane;
            const bool hit = j < cnt && (b0 - range.x + (uint32_t)j) < wmax && box_hit2(S, buf, j, c);
            const uint32_t m = __ballot_sync(0xffffffffu, hit);
            if (hit) s_list[w][nw + __popc(m & lt)] = (uint8_t)j;
            nw += __popc(m);
        }
        __syncwarp();
        for (int i = nw - 1; i >= 0; --i) {
            const int j = s_list[w][i];
            const float4 p = S.xyd[buf][j];
            const float4 co = S.co[buf][j];
            const float4 col = S.col[buf][j];
            float g9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const bool hit = pix_bwd_step(q, b0 + (uint32_t)j - range.x, co, col, bg0, bg1, bg2, fx - p.x,
                                          fy - p.y, g9);
            if (__any_sync(0xffffffffu, hit)) {
                const float tot = reduce9(g9, lane);
                if (slot >= 0) atomicAdd(grad2d + 16 * (rec0 + S.g[buf][j]) + slot_off, tot);
            }
        }
        b1 = pb1;
        b0 = pb0;
        pb1 = nb1;
        pb0 = nb0;
        g_cur = g_next;
        g_next = g_after;
        buf ^= 1;
    }
    cp_async_wait<0>();  // no copy may outlive the block
}

// Diagnostic: blended pairs, with the forward's skip rules, up to each
// pixel's contributor count (one pixel per thread, batches as above, no cull).
__global__ void __launch_bounds__(kRenderThreads) render_count_kernel(
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgb, int n,
    const gsfit_camera* __restrict__ cams_g, int n_views, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ tile_order, const uint32_t* __restrict__ n_contrib,
    unsigned long long* __restrict__ count) {
    extern __shared__ gsfit_camera cams[];
    __shared__ Batch S;
    load_cameras(cams, cams_g, n_views);
    __syncthreads();
    const int t = tile_order ? (int)tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileCtx c = tile_ctx(cams, n_views, t);
    const uint2 range = ranges[t];
    const size_t rec0 = (size_t)c.view * n;
    const uint32_t last = c.inside ? n_contrib[c.pix] : 0u;
    unsigned long long mine = 0;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kBatch) {
        __syncthreads();
        stage(S, b0 + threadIdx.x, range.y, vals, xyd, conic, rgb, rec0, n);
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, range.y - b0);
        for (int j = 0; j < cnt; ++j) {
            if (S.g[j] == 0xffffffffu || b0 - range.x + (uint32_t)j >= last) continue;
            const float power = splat_power(S.co[j], (float)c.px - S.xy[j].x, (float)c.py - S.xy[j].y);
            if (power > 0.0f) continue;
            if (fminf(kAlphaClamp, S.co[j].w * __expf(power)) >= kAlphaSkip) ++mine;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

}  // namespace

bool valid_proj(const gsfit_proj* p);
bool valid_gaussians(const gsfit_gaussians* g);
int project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V, float* grad2d,
                float* grads, cudaStream_t s);

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_render_fwd(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                                int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                                const uint32_t* tile_order, const float* bg, float* rgb, float* alpha,
                                float* T_final, uint32_t* n_contrib, cudaStream_t stream) {
    if (!valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || n < 1 || total_tiles < 1 ||
        !vals || !ranges || !bg || !rgb || !alpha || !T_final || !n_contrib)
        return GSFIT_ERR_INVALID_ARG;
    render_fwd_kernel<<<total_tiles, kRenderThreads, sizeof(gsfit_camera) * n_views, stream>>>(
        reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), n, cams, n_views, vals, reinterpret_cast<const uint2*>(ranges),
        tile_order, bg, rgb, alpha, T_final, n_contrib);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

extern "C" int gsfit_blend_bwd(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                               int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                               const uint32_t* tile_order, const float* bg, const float* T_final,
                               const uint32_t* n_contrib, const float* dL_drgb, const float* dL_dalpha, float* grad2d,
                               cudaStream_t stream) {
    if (!valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || n < 1 || total_tiles < 1 ||
        !vals || !ranges || !bg || !T_final || !n_contrib || !dL_drgb || !dL_dalpha || !grad2d ||
        (reinterpret_cast<uintptr_t>(grad2d) % 16) != 0)
        return GSFIT_ERR_INVALID_ARG;
    render_bwd_kernel<<<total_tiles, kRenderThreads, sizeof(gsfit_camera) * n_views, stream>>>(
        reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), n, cams, n_views, vals, reinterpret_cast<const uint2*>(ranges),
        tile_order, bg, T_final, n_contrib, dL_drgb, dL_dalpha, grad2d);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

extern "C" int gsfit_project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                                 int32_t n_views, float* grad2d, float* grads, cudaStream_t stream) {
    if (!valid_gaussians(g) || !valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || !grad2d ||
        !grads || (reinterpret_cast<uintptr_t>(grad2d) % 16) != 0 || (reinterpret_cast<uintptr_t>(grads) % 16) != 0)
        return GSFIT_ERR_INVALID_ARG;
    return project_bwd(g, proj, cams, n_views, grad2d, grads, stream);
}

extern "C" int gsfit_render_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                                int32_t n_views, int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                                const uint32_t* tile_order, const float* bg, const float* T_final,
                                const uint32_t* n_contrib, const float* dL_drgb, const float* dL_dalpha, float* grad2d,
                                float* grads, cudaStream_t stream) {
    if (!valid_gaussians(g)) return GSFIT_ERR_INVALID_ARG;
    const int rc = gsfit_blend_bwd(proj, cams, n_views, g->n, total_tiles, vals, ranges, tile_order, bg, T_final,
                                   n_contrib, dL_drgb, dL_dalpha, grad2d, stream);
    if (rc != GSFIT_OK) return rc;
    return gsfit_project_bwd(g, proj, cams, n_views, grad2d, grads, stream);
}

extern "C" int gsfit_render_count(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                                  int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                                  const uint32_t* tile_order, const uint32_t* n_contrib, unsigned long long* count,
                                  cudaStream_t stream) {
    if (!valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || n < 1 || total_tiles < 1 ||
        !vals || !ranges || !n_contrib || !count)
        return GSFIT_ERR_INVALID_ARG;
    render_count_kernel<<<total_tiles, kRenderThreads, sizeof(gsfit_camera) * n_views, stream>>>(
        reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), n, cams, n_views, vals, reinterpret_cast<const uint2*>(ranges),
        tile_order, n_contrib, count);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
