// Photometric loss of a view batch and its gradient (3DGS loss on colour with
// an added L1 term on alpha for the alpha supervision of Section 4.2; targets
// are composited over the same randomised background as the render).
//
// Design: one work item is a 32 x 32 output tile of one colour channel of one
// view. The item loads render and target over the tile plus a 10-pixel halo
// into shared memory, forms the five windowed moments on the tile plus a
// 5-pixel halo with two separable 11-tap passes, evaluates the SSIM map and
// its partials there, and convolves the partials back onto the tile: the
// gradient of the windowed SSIM never leaves shared memory, so the kernel
// reads each input pixel once and writes each gradient once. Channel-0 items
// also handle the alpha term. Persistent CTAs stride over the items.
#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kOut = 32;             // output tile edge
constexpr int kR1 = kOut + 10;       // moments / partials region (halo 5): 42
constexpr int kR2 = kOut + 20;       // input region (halo 10): 52
constexpr int kStrip = 4;            // outputs per thread along a pass (register blocking)
constexpr int kR2p = 56;             // input rows / columns padded so strips never leave the array
constexpr int kR1p = 44;             // moment rows / columns padded to whole strips
constexpr int kLossThreads = 256;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct LossSmem {
    float x[kR2][kR2p];         // render, input region (zero outside the image and in the padding)
    float y[kR2][kR2p];         // target composited over the background
    float h[5][kR2p][kR1p];     // horizontal pass of x, y, x^2, y^2, xy; later the SSIM partials
    float m[5][kR1p][kR1];      // moments; later the horizontal pass of the partials
};

// Normalised 11-tap Gaussian, sigma = 1.5.
__device__ __forceinline__ void window(float w[11]) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 11; ++i) {
        const float d = (float)(i - 5);
        w[i] = expf(-d * d / (2.0f * 1.5f * 1.5f));
        s += w[i];
    }
#pragma unroll
    for (int i = 0; i < 11; ++i) w[i] /= s;
}

// One pass of the 11-tap window over a strip of kStrip consecutive outputs:
// the kStrip + 10 inputs are read once into registers.
template <int STRIDE>
__device__ __forceinline__ void strip11(const float* src, const float w[11], float out[kStrip]) {
    float in[kStrip + 10];
#pragma unroll
    for (int k = 0; k < kStrip + 10; ++k) in[k] = src[k * STRIDE];
#pragma unroll
    for (int o = 0; o < kStrip; ++o) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < 11; ++j) a += w[j] * in[o + j];
        out[o] = a;
    }
}

__global__ void __launch_bounds__(kLossThreads, 2) loss_kernel(
    const gsfit_camera* __restrict__ cams_g, int n_views, const float* __restrict__ rgb,
    const float* __restrict__ alpha, const float* __restrict__ t_rgb, const float* __restrict__ t_alpha,
    const float* __restrict__ bg, float lambda, float* __restrict__ g_rgb, float* __restrict__ g_alpha,
    float* __restrict__ acc /* 3 per view: sum|x-y|, sum SSIM, sum|A-A*| */) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LossSmem& S = *reinterpret_cast<LossSmem*>(smem_raw);
    __shared__ int s_item_off[GSFIT_MAX_VIEWS + 1];
    __shared__ float s_red[3][kLossThreads / 32];
    if (threadIdx.x == 0) {
        int o = 0;
        for (int v = 0; v < n_views; ++v) {
            s_item_off[v] = o;
            const int tx = (cams_g[v].width + kOut - 1) / kOut, ty = (cams_g[v].height + kOut - 1) / kOut;
            o += 3 * tx * ty;
        }
        s_item_off[n_views] = o;
    }
    // zero the padding once: rows / columns beyond the region stay zero
    for (int k = threadIdx.x; k < 5 * kR2p * kR1p; k += kLossThreads) (&S.h[0][0][0])[k] = 0.f;
    float w[11];
    window(w);
    __syncthreads();
    const int n_items = s_item_off[n_views];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int v = 0;
        while (s_item_off[v + 1] <= item) ++v;
        const gsfit_camera& cam = cams_g[v];
        const int W = cam.width, H = cam.height;
        const int txn = (W + kOut - 1) / kOut;
        const int local = item - s_item_off[v];
        const int ch = local % 3;
        const int tile = local / 3;
        const int oy = (tile / txn) * kOut, ox = (tile % txn) * kOut;
        const long long P = (long long)W * H;
        const float* X = rgb + 3ll * cam.pixel_offset + ch * P;
        const float* Yt = t_rgb + 3ll * cam.pixel_offset + ch * P;
        const float* At = t_alpha + cam.pixel_offset;
        const float bgc = bg[3 * v + ch];
        const float inv3PV = 1.0f / (3.0f * (float)P * (float)n_views);

        // 1. inputs over the 52 x 52 region (56 columns with zero padding);
        //    thread (column tid % 64, first row tid / 64) walks rows 4 apart
        {
            const int cidx = tid & 63, gx = ox - 10 + cidx;
            const bool col_ok = cidx < kR2 && gx >= 0 && gx < W;
            for (int r = tid >> 6; r < kR2; r += kLossThreads / 64) {
                const int gy = oy - 10 + r;
                float xv = 0.f, yv = 0.f;
                if (col_ok && gy >= 0 && gy < H) {
                    const long long q = (long long)gy * W + gx;
                    xv = X[q];
                    yv = Yt[q] + (1.0f - At[q]) * bgc;
                }
                if (cidx < kR2p) {
                    S.x[r][cidx] = xv;
                    S.y[r][cidx] = yv;
                }
            }
        }
        __syncthreads();
        // 2. horizontal pass of x, y, x^2, y^2, xy: 52 rows x 44 columns in strips of 4
        for (int k = tid; k < kR2 * (kR1p / kStrip); k += kLossThreads) {
            const int r = k / (kR1p / kStrip), c0 = (k - r * (kR1p / kStrip)) * kStrip;
            float xin[kStrip + 10], yin[kStrip + 10], xx[kStrip + 10], yy[kStrip + 10], xy[kStrip + 10];
#pragma unroll
            for (int j = 0; j < kStrip + 10; ++j) {
                xin[j] = S.x[r][c0 + j];
                yin[j] = S.y[r][c0 + j];
                xx[j] = xin[j] * xin[j];
                yy[j] = yin[j] * yin[j];
                xy[j] = xin[j] * yin[j];
            }
#pragma unroll
            for (int o = 0; o < kStrip; ++o) {
                float a = 0.f, b = 0.f, c = 0.f, d = 0.f, e = 0.f;
#pragma unroll
                for (int j = 0; j < 11; ++j) {
                    a += w[j] * xin[o + j];
                    b += w[j] * yin[o + j];
                    c += w[j] * xx[o + j];
                    d += w[j] * yy[o + j];
                    e += w[j] * xy[o + j];
                }
                S.h[0][r][c0 + o] = a; S.h[1][r][c0 + o] = b; S.h[2][r][c0 + o] = c;
                S.h[3][r][c0 + o] = d; S.h[4][r][c0 + o] = e;
            }
        }
        __syncthreads();
        // 3. vertical pass: moments on 44 x 42 (rows 42, 43 are padding) in strips of 4
        for (int k = tid; k < 5 * kR1 * (kR1p / kStrip); k += kLossThreads) {
            const int f = k / (kR1 * (kR1p / kStrip));
            const int rem = k - f * (kR1 * (kR1p / kStrip));
            const int cidx = rem % kR1, r0 = (rem / kR1) * kStrip;
            float out[kStrip];
            strip11<kR1p>(&S.h[f][r0][cidx], w, out);
#pragma unroll
            for (int o = 0; o < kStrip; ++o) S.m[f][r0 + o][cidx] = out[o];
        }
        __syncthreads();
        // 4. SSIM and its partials w.r.t. (mu_x, E[x^2], E[xy]) on the 42 x 42
        //    region; zero outside the image (those windows do not exist).
        float ssim_sum = 0.f;
        float (*part)[kR2p][kR1p] = S.h;  // reuse: part[0..2][r][c], r, c < 42
        for (int k = tid; k < kR1 * kR1; k += kLossThreads) {
            const int r = k / kR1, cidx = k - r * kR1;
            const int gy = oy - 5 + r, gx = ox - 5 + cidx;
            float dmu = 0.f, dxx = 0.f, dxy = 0.f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float mx = S.m[0][r][cidx], my = S.m[1][r][cidx];
                const float sx = S.m[2][r][cidx] - mx * mx, sy = S.m[3][r][cidx] - my * my;
                const float sxy = S.m[4][r][cidx] - mx * my;
                const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
                const float B1 = mx * mx + my * my + kC1, B2 = sx + sy + kC2;
                const float iB1 = 1.0f / B1, iB2 = 1.0f / B2;
                const float iB = iB1 * iB2;
                const float ss = A1 * A2 * iB;
                dmu = 2.f * my * (A2 - A1) * iB - 2.f * mx * ss * (iB1 - iB2);
                dxx = -ss * iB2;
                dxy = 2.f * A1 * iB;
                if (r >= 5 && r < 5 + kOut && cidx >= 5 && cidx < 5 + kOut) ssim_sum += ss;
            }
            part[0][r][cidx] = dmu;
            part[1][r][cidx] = dxx;
            part[2][r][cidx] = dxy;
        }
        __syncthreads();
        // 5. horizontal pass of the partials: 42 rows x 32 columns in strips of 4
        float (*hp)[kR1p][kR1] = S.m;  // reuse: hp[0..2][r][c], r < 42, c < 32
        for (int k = tid; k < 3 * kR1 * (kOut / kStrip); k += kLossThreads) {
            const int f = k / (kR1 * (kOut / kStrip));
            const int rem = k - f * (kR1 * (kOut / kStrip));
            const int r = rem / (kOut / kStrip), c0 = (rem % (kOut / kStrip)) * kStrip;
            float out[kStrip];
            strip11<1>(&part[f][r][c0], w, out);
#pragma unroll
            for (int o = 0; o < kStrip; ++o) hp[f][r][c0 + o] = out[o];
        }
        __syncthreads();
        // 6. vertical pass onto the tile (one 4-pixel column strip per thread) and
        //    the gradient
        float l1 = 0.f, la = 0.f;
        {
            const int cidx = tid % kOut, r0 = (tid / kOut) * kStrip;  // 32 columns x 8 strips = 256
            float cm[kStrip], cxx[kStrip], cxy[kStrip];
            strip11<kR1>(&hp[0][r0][cidx], w, cm);
            strip11<kR1>(&hp[1][r0][cidx], w, cxx);
            strip11<kR1>(&hp[2][r0][cidx], w, cxy);
#pragma unroll
            for (int o = 0; o < kStrip; ++o) {
                const int r = r0 + o;
                const int gy = oy + r, gx = ox + cidx;
                if (gy >= H || gx >= W) continue;
                const float xv = S.x[r + 10][cidx + 10], yv = S.y[r + 10][cidx + 10];
                const float dssim = cm[o] + 2.f * xv * cxx[o] + yv * cxy[o];
                const float diff = xv - yv;
                const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
                l1 += fabsf(diff);
                const long long q = (long long)gy * W + gx;
                g_rgb[3ll * cam.pixel_offset + ch * P + q] = ((1.0f - lambda) * sg - lambda * dssim) * inv3PV;
                if (ch == 0) {
                    const float da = alpha[cam.pixel_offset + q] - At[q];
                    la += fabsf(da);
                    g_alpha[cam.pixel_offset + q] =
                        (da > 0.f ? 1.f : (da < 0.f ? -1.f : 0.f)) / ((float)P * (float)n_views);
                }
            }
        }
        // block sums of the loss terms
        ssim_sum = warp_sum(ssim_sum);
        l1 = warp_sum(l1);
        la = warp_sum(la);
        if (lane == 0) {
            s_red[0][wid] = l1;
            s_red[1][wid] = ssim_sum;
            s_red[2][wid] = la;
        }
        __syncthreads();
        if (tid < 3) {
            float sacc = 0.f;
            for (int k = 0; k < kLossThreads / 32; ++k) sacc += s_red[tid][k];
            atomicAdd(&acc[3 * v + tid], sacc);
        }
        // (rows 52..55 of h, the only padding the passes read, are never written)
        __syncthreads();
    }
}

__global__ void loss_finalize_kernel(const gsfit_camera* __restrict__ cams, int n_views, float lambda,
                                     const float* __restrict__ acc, float* __restrict__ loss_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float L = 0.f;
    for (int v = 0; v < n_views; ++v) {
        const float P = (float)cams[v].width * (float)cams[v].height;
        const float l1 = acc[3 * v] / (3.f * P), ssim = acc[3 * v + 1] / (3.f * P), la = acc[3 * v + 2] / P;
        L += (1.f - lambda) * l1 + lambda * (1.f - ssim) + la;
    }
    *loss_out = L / (float)n_views;
}

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" size_t gsfit_loss_workspace_size(int32_t n_views) {
    if (n_views < 1 || n_views > GSFIT_MAX_VIEWS) return 0;
    return (size_t)(3 * n_views) * sizeof(float);
}

extern "C" int gsfit_loss(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
                          const float* target_rgb, const float* target_alpha, const float* bg, float lambda,
                          float* dL_drgb, float* dL_dalpha, float* loss_out, void* ws, size_t ws_bytes,
                          cudaStream_t stream) {
    if (!cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || !rgb || !alpha || !target_rgb || !target_alpha ||
        !bg || !dL_drgb || !dL_dalpha || !ws || ws_bytes < gsfit_loss_workspace_size(n_views))
        return GSFIT_ERR_INVALID_ARG;
    static bool attr_done[64] = {false};
    int dev = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GSFIT_ERR_CUDA;
    const size_t smem = sizeof(LossSmem);
    if (!attr_done[dev]) {
        GSFIT_CUDA_CHECK(cudaFuncSetAttribute(loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done[dev] = true;
    }
    int sms = 0;
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* acc = static_cast<float*>(ws);
    GSFIT_CUDA_CHECK(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * n_views, stream));
    loss_kernel<<<2 * sms, kLossThreads, smem, stream>>>(cams, n_views, rgb, alpha, target_rgb, target_alpha, bg,
                                                         lambda, dL_drgb, dL_dalpha, acc);
    GSFIT_LAUNCH_CHECK();
    if (loss_out) {
        loss_finalize_kernel<<<1, 32, 0, stream>>>(cams, n_views, lambda, acc, loss_out);
        GSFIT_LAUNCH_CHECK();
    }
    return GSFIT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant (no counterpart in the paper): the same kernels with
// the per-view accumulators in a fixed device array of this library, for
// callers that cannot allocate device memory (a real-time frame loop, a
// plug-in whose host application owns all device allocations).
// ---------------------------------------------------------------------------

namespace gsfit {
namespace {

constexpr int kNoAllocMaxViews = GSFIT_MAX_VIEWS;

// 3 accumulators per view: sum|x - y|, sum SSIM, sum|A - A*| (3 KB). Host code
// must not use this name as a pointer: it is a host-side stand-in; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float g_loss_noalloc_acc[3 * kNoAllocMaxViews];

// Device address of g_loss_noalloc_acc, looked up once per device with that
// device current.
int noalloc_acc_address(int dev, float** out) {
    static float* cached[64] = {nullptr};
    if (dev < 0 || dev >= 64) return GSFIT_ERR_CUDA;
    if (!cached[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_loss_noalloc_acc) != cudaSuccess || !p) return GSFIT_ERR_CUDA;
        cached[dev] = static_cast<float*>(p);
    }
    *out = cached[dev];
    return GSFIT_OK;
}

}  // namespace
}  // namespace gsfit

extern "C" int gsfit_loss_noalloc(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
                                  const float* target_rgb, const float* target_alpha, const float* bg,
                                  float lambda, float* dL_drgb, float* dL_dalpha, float* loss_out,
                                  cudaStream_t stream) {
    if (!cams || n_views < 1 || n_views > kNoAllocMaxViews || !rgb || !alpha || !target_rgb || !target_alpha ||
        !bg || !dL_drgb || !dL_dalpha)
        return GSFIT_ERR_INVALID_ARG;
    int dev = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    float* acc = nullptr;
    const int rc = noalloc_acc_address(dev, &acc);
    if (rc != GSFIT_OK) return rc;
    const size_t smem = sizeof(LossSmem);
    GSFIT_CUDA_CHECK(cudaFuncSetAttribute(loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 0;
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the array keeps the previous call's sums: clear this call's part first
    GSFIT_CUDA_CHECK(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * n_views, stream));
    loss_kernel<<<2 * sms, kLossThreads, smem, stream>>>(cams, n_views, rgb, alpha, target_rgb, target_alpha, bg,
                                                         lambda, dL_drgb, dL_dalpha, acc);
    GSFIT_LAUNCH_CHECK();
    if (loss_out) {
        loss_finalize_kernel<<<1, 32, 0, stream>>>(cams, n_views, lambda, acc, loss_out);
        GSFIT_LAUNCH_CHECK();
    }
    return GSFIT_OK;
}
