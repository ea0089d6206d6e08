// Front-to-back compositing of the tile lists and its back-to-front adjoint.
//
// The peripheral model is rendered and trained as 3DGS with an alpha output
// for alpha supervision (Section 4.2). Per pixel, over its tile's sorted
// range: power = -1/2 (a' dx^2 + c' dy^2) - b' dx dy (skip if > 0), alpha =
// min(0.99, o exp(power)) (skip if < 1/255), stop before T would drop below
// 1e-4, C = sum c alpha T + T_N bg, A = 1 - T_N.
//
// Design: one 256-thread CTA per 16 x 16 tile (one pixel per thread); the
// tile's records are staged through shared memory in batches of 256 (one
// coalesced 48-byte record per thread), then every thread walks the batch.
// The adjoint keeps no per-(pixel, Gaussian) state: it restarts from the
// stored final transmittance and contributor count and recovers T_i =
// T_{i+1} / (1 - alpha_i) walking the list backwards; the nine per-Gaussian
// gradient terms are summed across the warp with shuffles (all lanes visit the
// same Gaussian in lock-step) before one set of float4 atomics per warp.
#include "common.cuh"

namespace gsfit {

namespace {

struct TileCtx {
    int view, px, py, W, H;
    bool inside;
    long long pix, plane, rgb_base;
};

__device__ __forceinline__ TileCtx tile_ctx(const gsfit_camera* cams, int n_views, int t) {
    TileCtx c;
    c.view = view_of_tile(cams, n_views, t);
    const gsfit_camera& cam = cams[c.view];
    const int local = t - cam.tile_offset;
    const int txn = tiles_x_of(cam);
    const int ty = local / txn, tx = local - ty * txn;
    c.px = tx * kTile + (threadIdx.x % kTile);
    c.py = ty * kTile + (threadIdx.x / kTile);
    c.W = cam.width;
    c.H = cam.height;
    c.inside = c.px < c.W && c.py < c.H;
    c.plane = (long long)c.W * c.H;
    c.pix = (long long)cam.pixel_offset + (long long)c.py * c.W + c.px;
    c.rgb_base = 3ll * cam.pixel_offset + (long long)c.py * c.W + c.px;
    return c;
}

__global__ void __launch_bounds__(kTilePixels) render_fwd_kernel(
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgb, int n,
    const gsfit_camera* __restrict__ cams_g, int n_views, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const float* __restrict__ bg, float* __restrict__ out_rgb,
    float* __restrict__ out_alpha, float* __restrict__ out_T, uint32_t* __restrict__ out_nc) {
    extern __shared__ gsfit_camera cams[];
    __shared__ float2 s_xy[kTilePixels];
    __shared__ float4 s_co[kTilePixels];
    __shared__ float4 s_rgb[kTilePixels];
    load_cameras(cams, cams_g, n_views);
    __syncthreads();
    const int t = blockIdx.x;
    const TileCtx c = tile_ctx(cams, n_views, t);
    const uint2 range = ranges[t];
    const size_t rec0 = (size_t)c.view * n;
    const float fx = (float)c.px, fy = (float)c.py;

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t contributor = 0, last = 0;
    bool done = !c.inside;
    for (uint32_t b0 = range.x; b0 < range.y; b0 += kTilePixels) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < range.y) {
            const uint32_t g = vals[idx];
            if (g < (uint32_t)n) {
                const size_t r = rec0 + g;
                const float4 p = xyd[r];
                s_xy[threadIdx.x] = make_float2(p.x, p.y);
                s_co[threadIdx.x] = conic[r];
                s_rgb[threadIdx.x] = rgb[r];
            } else {  // only after a failed sort: a splat that is never blended
                s_xy[threadIdx.x] = make_float2(0.f, 0.f);
                s_co[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_rgb[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kTilePixels, range.y - b0);
        for (int j = 0; j < cnt && !done; ++j) {
            ++contributor;
            const float2 xy = s_xy[j];
            const float4 co = s_co[j];
            const float dx = fx - xy.x, dy = fy - xy.y;
            const float power = splat_power(co, dx, dy);
            if (power > 0.0f) continue;
            const float alpha = fminf(kAlphaClamp, co.w * __expf(power));
            if (alpha < kAlphaSkip) continue;
            const float test_T = T * (1.0f - alpha);
            if (test_T < kTStop) {
                done = true;
                break;
            }
            const float4 col = s_rgb[j];
            const float w = alpha * T;
            C0 += col.x * w;
            C1 += col.y * w;
            C2 += col.z * w;
            T = test_T;
            last = contributor;
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

__global__ void __launch_bounds__(kTilePixels) render_bwd_kernel(
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgb, int n,
    const gsfit_camera* __restrict__ cams_g, int n_views, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const float* __restrict__ bg, const float* __restrict__ T_final,
    const uint32_t* __restrict__ n_contrib, const float* __restrict__ dL_drgb, const float* __restrict__ dL_dalpha,
    float4* __restrict__ grad2d) {
    extern __shared__ gsfit_camera cams[];
    __shared__ float2 s_xy[kTilePixels];
    __shared__ float4 s_co[kTilePixels];
    __shared__ float4 s_rgb[kTilePixels];
    __shared__ uint32_t s_rec[kTilePixels];
    __shared__ uint32_t s_max;
    load_cameras(cams, cams_g, n_views);
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    const int t = blockIdx.x;
    const TileCtx c = tile_ctx(cams, n_views, t);
    const uint2 range = ranges[t];
    const size_t rec0 = (size_t)c.view * n;
    const float fx = (float)c.px, fy = (float)c.py;
    const int lane = threadIdx.x & 31;

    float T = 1.0f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dA = 0.f;
    uint32_t last = 0;
    if (c.inside) {
        T = T_final[c.pix];
        last = n_contrib[c.pix];
        dC0 = dL_drgb[c.rgb_base];
        dC1 = dL_drgb[c.rgb_base + c.plane];
        dC2 = dL_drgb[c.rgb_base + 2 * c.plane];
        dA = dL_dalpha[c.pix];
        atomicMax(&s_max, last);
    }
    const float TN = T;
    const float* bgv = bg + 3 * c.view;
    const float tb0 = TN * bgv[0], tb1 = TN * bgv[1], tb2 = TN * bgv[2];
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;  // colour composited behind the current Gaussian
    __syncthreads();
    const uint32_t end = range.x + min(s_max, range.y - range.x);

    for (uint32_t b1 = end; b1 > range.x;) {
        const uint32_t b0 = (b1 - range.x > (uint32_t)kTilePixels) ? b1 - kTilePixels : range.x;
        __syncthreads();
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < b1) {
            const uint32_t g = vals[idx];
            if (g < (uint32_t)n) {
                const size_t r = rec0 + g;
                const float4 p = xyd[r];
                s_xy[threadIdx.x] = make_float2(p.x, p.y);
                s_co[threadIdx.x] = conic[r];
                s_rgb[threadIdx.x] = rgb[r];
            } else {  // only after a failed sort: never blended, never written
                s_xy[threadIdx.x] = make_float2(0.f, 0.f);
                s_co[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_rgb[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            s_rec[threadIdx.x] = g;
        }
        __syncthreads();
        for (int j = (int)(b1 - b0) - 1; j >= 0; --j) {
            const uint32_t pos = b0 + (uint32_t)j - range.x;
            float gu = 0.f, gv = 0.f, ga = 0.f, gb = 0.f, gc = 0.f, go = 0.f, gr = 0.f, gg = 0.f, gbl = 0.f;
            bool hit = false;
            if (pos < last) {
                const float2 xy = s_xy[j];
                const float4 co = s_co[j];
                const float dx = fx - xy.x, dy = fy - xy.y;
                const float power = splat_power(co, dx, dy);
                if (power <= 0.0f) {
                    const float G = __expf(power);
                    const float a = co.w * G;
                    const float alpha = fminf(kAlphaClamp, a);
                    if (alpha >= kAlphaSkip) {
                        hit = true;
                        const float one_m = 1.0f - alpha;
                        const float inv = 1.0f / one_m;
                        T = T * inv;  // transmittance in front of this Gaussian
                        const float4 col = s_rgb[j];
                        const float wT = alpha * T;
                        gr = dC0 * wT;
                        gg = dC1 * wT;
                        gbl = dC2 * wT;
                        const float dalpha = dA * TN * inv + dC0 * (T * col.x - (S0 + tb0) * inv) +
                                             dC1 * (T * col.y - (S1 + tb1) * inv) +
                                             dC2 * (T * col.z - (S2 + tb2) * inv);
                        S0 += col.x * wT;
                        S1 += col.y * wT;
                        S2 += col.z * wT;
                        if (a <= kAlphaClamp) {
                            const float dpow = dalpha * alpha;
                            go = dalpha * G;
                            gu = dpow * (co.x * dx + co.y * dy);
                            gv = dpow * (co.z * dy + co.y * dx);
                            ga = -0.5f * dpow * dx * dx;
                            gb = -dpow * dx * dy;
                            gc = -0.5f * dpow * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, hit)) {
                gu = warp_sum(gu); gv = warp_sum(gv); go = warp_sum(go);
                ga = warp_sum(ga); gb = warp_sum(gb); gc = warp_sum(gc);
                gr = warp_sum(gr); gg = warp_sum(gg); gbl = warp_sum(gbl);
                if (lane == 0) {
                    float4* dst = grad2d + 3 * (rec0 + s_rec[j]);
                    atomicAdd(dst + 0, make_float4(gu, gv, go, 0.f));
                    atomicAdd(dst + 1, make_float4(ga, gb, gc, 0.f));
                    atomicAdd(dst + 2, make_float4(gr, gg, gbl, 0.f));
                }
            }
        }
        b1 = b0;
    }
}

}  // namespace

bool valid_proj(const gsfit_proj* p);
bool valid_gaussians(const gsfit_gaussians* g);
int project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V, float* grad2d,
                float* grads, cudaStream_t s);

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_render_fwd(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                                int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges, const float* bg,
                                float* rgb, float* alpha, float* T_final, uint32_t* n_contrib,
                                cudaStream_t stream) {
    if (!valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || n < 1 || total_tiles < 1 ||
        !vals || !ranges || !bg || !rgb || !alpha || !T_final || !n_contrib)
        return GSFIT_ERR_INVALID_ARG;
    render_fwd_kernel<<<total_tiles, kTilePixels, sizeof(gsfit_camera) * n_views, stream>>>(
        reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), n, cams, n_views, vals, reinterpret_cast<const uint2*>(ranges),
        bg, rgb, alpha, T_final, n_contrib);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

extern "C" int gsfit_render_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                                int32_t n_views, int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                                const float* bg, const float* T_final, const uint32_t* n_contrib,
                                const float* dL_drgb, const float* dL_dalpha, float* grad2d, float* grads,
                                cudaStream_t stream) {
    if (!valid_gaussians(g) || !valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS ||
        total_tiles < 1 || !vals || !ranges || !bg || !T_final || !n_contrib || !dL_drgb || !dL_dalpha ||
        !grad2d || !grads || (reinterpret_cast<uintptr_t>(grad2d) % 16) != 0 ||
        (reinterpret_cast<uintptr_t>(grads) % 16) != 0)
        return GSFIT_ERR_INVALID_ARG;
    render_bwd_kernel<<<total_tiles, kTilePixels, sizeof(gsfit_camera) * n_views, stream>>>(
        reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), g->n, cams, n_views, vals,
        reinterpret_cast<const uint2*>(ranges), bg, T_final, n_contrib, dL_drgb, dL_dalpha,
        reinterpret_cast<float4*>(grad2d));
    GSFIT_LAUNCH_CHECK();
    return project_bwd(g, proj, cams, n_views, grad2d, grads, stream);
}
