// Adam update of all Gaussian parameters (3DGS optimiser; Section 4.2 raises
// the scale / opacity / colour rates by about 50% for the abbreviated run and
// resets the optimiser state on every restart -- both are the caller's lr
// table and moment buffers).
//
// Design: the parameters, gradients and both moments share one float4-plane
// layout, so the update is a single streaming pass: per float4, read p, g,
// m, v (64 bytes) and write p, m, v (48 bytes); grid.y selects the plane and
// with it the four per-component learning rates. The step count lives on the
// device so a captured graph can be replayed without host updates.
#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kMaxPlanes = 16;

struct LrTable {
    float4 lr[kMaxPlanes];
};

__global__ void __launch_bounds__(256) adam_kernel(float4* __restrict__ p, const float4* __restrict__ g,
                                                   float4* __restrict__ m, float4* __restrict__ v, int n,
                                                   LrTable lrt, float b1, float b2, float eps,
                                                   const int32_t* __restrict__ step) {
    const int plane = blockIdx.y;
    const float4 lr = lrt.lr[plane];
    const int t = *step + 1;
    const float bc1 = 1.0f - powf(b1, (float)t);
    const float bc2 = 1.0f - powf(b2, (float)t);
    const float rbc2 = rsqrtf(bc2);
    const float s1 = 1.0f / bc1;
    const size_t base = (size_t)plane * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t k = base + i;
        const float4 gg = g[k];
        float4 mm = m[k], vv = v[k], pp = p[k];
#define GSFIT_ADAM_LANE(c)                                                     \
    mm.c = b1 * mm.c + (1.0f - b1) * gg.c;                                     \
    vv.c = b2 * vv.c + (1.0f - b2) * gg.c * gg.c;                              \
    pp.c -= lr.c * (mm.c * s1) / (sqrtf(vv.c) * rbc2 + eps);
        GSFIT_ADAM_LANE(x)
        GSFIT_ADAM_LANE(y)
        GSFIT_ADAM_LANE(z)
        GSFIT_ADAM_LANE(w)
#undef GSFIT_ADAM_LANE
        m[k] = mm;
        v[k] = vv;
        p[k] = pp;
    }
}

__global__ void step_increment_kernel(int32_t* step) { *step += 1; }

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, int32_t n_planes,
                               const float* lr, float beta1, float beta2, float eps, int32_t* step,
                               cudaStream_t stream) {
    if (!params || !grads || !m || !v || !lr || !step || n < 1 || n_planes < 1 || n_planes > kMaxPlanes)
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
    adam_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<float4*>(params), reinterpret_cast<const float4*>(grads),
                                          reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n, t, beta1,
                                          beta2, eps, step);
    GSFIT_LAUNCH_CHECK();
    step_increment_kernel<<<1, 1, 0, stream>>>(step);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
