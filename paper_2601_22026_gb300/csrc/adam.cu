// Adam update of all Gaussian parameters (3DGS optimiser; Section 4.2 raises
// the scale / opacity / colour rates by about 50% for the abbreviated run and
// resets the optimiser state on every restart -- both are the caller's lr
// table and moment buffers).
//
// Design: the parameters, gradients and both moments share one float4-plane
// layout, so the update is a single streaming pass: per float4, read p, g,
// m, v (64 bytes) and write p, m, v (48 bytes); grid.y selects the plane and
// with it the four per-component learning rates. The step count lives on the
// device so a captured graph can be replayed without host updates. In the
// mixed-precision form the same pass writes the 16-bit copy of the SH planes
// (8 more bytes per float4 of those planes).
#include "common.cuh"

namespace gsfit {

namespace {

template <int FT>
__global__ void __launch_bounds__(256) adam_kernel(float4* __restrict__ p, const float4* __restrict__ g,
                                                   float4* __restrict__ m, float4* __restrict__ v, int n,
                                                   LrTable lrt, float b1, float b2, float eps,
                                                   const int32_t* __restrict__ step, uint2* __restrict__ feat) {
    const int plane = blockIdx.y;
    const float4 lr = lrt.lr[plane];
    const AdamCoef c = adam_coef(b1, b2, eps, *step);
    const size_t base = (size_t)plane * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t k = base + i;
        const float4 gg = g[k];
        float4 mm = m[k], vv = v[k], pp = p[k];
        adam_update(pp, mm, vv, gg, lr, c);
        m[k] = mm;
        v[k] = vv;
        p[k] = pp;
        if constexpr (FT != GSFIT_FEATURES_F32) {
            if (plane >= kFeaturePlane0) feat[(size_t)(plane - kFeaturePlane0) * n + i] = pack_features<FT>(pp);
        }
    }
}

template <int FT>
__global__ void __launch_bounds__(256) refresh_kernel(const float4* __restrict__ p, int n, int n_planes,
                                                      uint2* __restrict__ feat) {
    const size_t total = (size_t)(n_planes - kFeaturePlane0) * n;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
        feat[k] = pack_features<FT>(p[(size_t)kFeaturePlane0 * n + k]);
}

__global__ void step_increment_kernel(int32_t* step) { *step += 1; }

}  // namespace

int step_increment(int32_t* step, cudaStream_t s) {
    step_increment_kernel<<<1, 1, 0, s>>>(step);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, int32_t n_planes,
                               const float* lr, float beta1, float beta2, float eps, int32_t* step, void* features,
                               int32_t feature_dtype, cudaStream_t stream) {
    if (!params || !grads || !m || !v || !lr || !step || n < 1 || n_planes < 1 || n_planes > kMaxPlanes)
        return GSFIT_ERR_INVALID_ARG;
    if (feature_dtype != GSFIT_FEATURES_F32 && feature_dtype != GSFIT_FEATURES_F16 &&
        feature_dtype != GSFIT_FEATURES_BF16)
        return GSFIT_ERR_INVALID_ARG;
    if (feature_dtype != GSFIT_FEATURES_F32 && (!features || (reinterpret_cast<uintptr_t>(features) % 8) != 0))
        return GSFIT_ERR_INVALID_ARG;
    for (const float* q : {(const float*)params, grads, (const float*)m, (const float*)v})
        if ((reinterpret_cast<uintptr_t>(q) % 16) != 0) return GSFIT_ERR_INVALID_ARG;
    LrTable t;
    for (int k = 0; k < kMaxPlanes; ++k)
        t.lr[k] = k < n_planes ? make_float4(lr[4 * k], lr[4 * k + 1], lr[4 * k + 2], lr[4 * k + 3])
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    int dev = 0, sms = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int want = (n + 255) / 256;
    const int bx = want < 4 * sms ? want : 4 * sms;
    dim3 grid((unsigned)bx, (unsigned)n_planes);
    float4* p4 = reinterpret_cast<float4*>(params);
    const float4* g4 = reinterpret_cast<const float4*>(grads);
    float4* m4 = reinterpret_cast<float4*>(m);
    float4* v4 = reinterpret_cast<float4*>(v);
    uint2* f = reinterpret_cast<uint2*>(features);
    if (feature_dtype == GSFIT_FEATURES_F16)
        adam_kernel<GSFIT_FEATURES_F16><<<grid, 256, 0, stream>>>(p4, g4, m4, v4, n, t, beta1, beta2, eps, step, f);
    else if (feature_dtype == GSFIT_FEATURES_BF16)
        adam_kernel<GSFIT_FEATURES_BF16><<<grid, 256, 0, stream>>>(p4, g4, m4, v4, n, t, beta1, beta2, eps, step, f);
    else
        adam_kernel<GSFIT_FEATURES_F32><<<grid, 256, 0, stream>>>(p4, g4, m4, v4, n, t, beta1, beta2, eps, step,
                                                                  nullptr);
    GSFIT_LAUNCH_CHECK();
    return step_increment(step, stream);
}

extern "C" int gsfit_features_refresh(const float* params, int32_t n, int32_t n_planes, void* features,
                                      int32_t feature_dtype, cudaStream_t stream) {
    if (!params || !features || n < 1 || n_planes <= kFeaturePlane0 || n_planes > kMaxPlanes ||
        (reinterpret_cast<uintptr_t>(params) % 16) != 0 || (reinterpret_cast<uintptr_t>(features) % 8) != 0 ||
        (feature_dtype != GSFIT_FEATURES_F16 && feature_dtype != GSFIT_FEATURES_BF16))
        return GSFIT_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long total = (long long)(n_planes - kFeaturePlane0) * n;
    const long long want = (total + 255) / 256;
    const int blocks = (int)(want < 8ll * sms ? want : 8ll * sms);
    const float4* p4 = reinterpret_cast<const float4*>(params);
    uint2* f = reinterpret_cast<uint2*>(features);
    if (feature_dtype == GSFIT_FEATURES_F16)
        refresh_kernel<GSFIT_FEATURES_F16><<<blocks, 256, 0, stream>>>(p4, n, n_planes, f);
    else if (feature_dtype == GSFIT_FEATURES_BF16)
        refresh_kernel<GSFIT_FEATURES_BF16><<<blocks, 256, 0, stream>>>(p4, n, n_planes, f);
    else
        return GSFIT_ERR_INVALID_ARG;
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
