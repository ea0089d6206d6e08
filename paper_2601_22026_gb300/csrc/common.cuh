// Internal helpers shared by the gsfit kernels (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gsfit.h"

#define GSFIT_CUDA_CHECK(expr)                          \
    do {                                                \
        cudaError_t err_ = (expr);                      \
        if (err_ != cudaSuccess) return GSFIT_ERR_CUDA; \
    } while (0)

#define GSFIT_LAUNCH_CHECK() GSFIT_CUDA_CHECK(cudaGetLastError())

namespace gsfit {

// Host-side set-up that must run once per device and CUDA context (a kernel
// attribute, a device symbol's address): a context reset (cudaDeviceReset, a
// released and recreated primary context) reloads the library's module, and
// the set-up has to run again. Identifies the context by its process-unique
// id (cuCtxGetId), not its handle, which a new context may reuse. Thread-safe.
struct ContextOnce {
    std::mutex m;
    unsigned long long ctx_id[64] = {};  // 0: not yet run on this device
};

// Two driver-API calls, resolved through the runtime's entry-point query so
// that the library needs no link against the driver (it loads on machines
// without one; the calls only run where a device exists).
struct DriverCtxApi {
    CUresult (*get_current)(CUcontext*) = nullptr;
    CUresult (*get_id)(CUcontext, unsigned long long*) = nullptr;
    bool ok = false;
};
inline const DriverCtxApi& driver_ctx_api() {
    static DriverCtxApi api;
    static std::once_flag flag;
    std::call_once(flag, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess && qb == cudaDriverEntryPointSuccess && a && b) {
            api.get_current = reinterpret_cast<CUresult (*)(CUcontext*)>(a);
            api.get_id = reinterpret_cast<CUresult (*)(CUcontext, unsigned long long*)>(b);
            api.ok = true;
        }
    });
    return api;
}

// The id of the calling thread's current context on device `dev` (created
// and made current by cudaSetDevice if there is none yet).
inline int current_context_id(int dev, unsigned long long* id) {
    const DriverCtxApi& api = driver_ctx_api();
    if (!api.ok) return GSFIT_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (api.get_current(&ctx) != CUDA_SUCCESS) return GSFIT_ERR_CUDA;
    if (!ctx) {
        if (cudaSetDevice(dev) != cudaSuccess || api.get_current(&ctx) != CUDA_SUCCESS || !ctx) return GSFIT_ERR_CUDA;
    }
    return api.get_id(ctx, id) == CUDA_SUCCESS && *id != 0 ? GSFIT_OK : GSFIT_ERR_CUDA;
}

// Runs fn() (returning a GSFIT status) unless it already succeeded on the
// current device in the current context.
template <typename Fn>
int run_once_per_context(ContextOnce& once, Fn fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GSFIT_ERR_CUDA;
    unsigned long long id = 0;
    const int rc = current_context_id(dev, &id);
    if (rc != GSFIT_OK) return rc;
    std::lock_guard<std::mutex> lock(once.m);
    if (once.ctx_id[dev] == id) return GSFIT_OK;
    const int r = fn();
    if (r == GSFIT_OK) once.ctx_id[dev] = id;
    return r;
}

// Opts `kernel` in to `bytes` of dynamic shared memory, once per device and context.
template <typename K>
int opt_in_smem(ContextOnce& once, K kernel, size_t bytes) {
    return run_once_per_context(once, [&] {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess
                   ? GSFIT_OK
                   : GSFIT_ERR_CUDA;
    });
}

constexpr int kTile = GSFIT_TILE;
constexpr int kTilePixels = kTile * kTile;
constexpr float kAlphaClamp = 0.99f;
constexpr float kAlphaSkip = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
constexpr float kDilation = 0.3f;
constexpr float kFrustumGuard = 1.3f;

inline int num_planes(int deg) {
    const int K = (deg + 1) * (deg + 1);
    return 3 + (3 * K + 3) / 4;
}

// Index of the view that owns global tile `t` (binary search over the
// per-view tile offsets held in shared memory; views are laid out in order).
__device__ __forceinline__ int view_of_tile(const gsfit_camera* cams, int n_views, int t) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_offset <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Copies the camera table into shared memory (whole block participates).
__device__ __forceinline__ void load_cameras(gsfit_camera* dst, const gsfit_camera* src, int n_views) {
    const int words = n_views * (int)(sizeof(gsfit_camera) / sizeof(int4));
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int k = threadIdx.x; k < words; k += blockDim.x) d[k] = s[k];
}

// Work buckets of the tile orders: quarter octaves of a count.
constexpr int kOrderBuckets = 128;

// Quarter octave of a count m: 4 floor(log2(m + 1)) plus the two bits below
// the leading one of m + 1, capped at 127 (the tile orders' work buckets).
__device__ __forceinline__ int quarter_octave(uint32_t m) {
    if (m >= 0x40000000u) return 127;
    const uint32_t x = m + 1u;
    const int l = 31 - __clz(x);  // floor(log2 x)
    const int f = l >= 2 ? (int)((x >> (l - 2)) & 3u) : (int)((x << (2 - l)) & 3u);
    return 4 * l + f;
}

// Tile edge of a camera's batch layout: 8 or 16 (16 for any other value).
__device__ __forceinline__ int tile_of(const gsfit_camera& c) { return c.tile == 8 ? 8 : 16; }
__device__ __forceinline__ int tiles_x_of(const gsfit_camera& c) {
    const int B = tile_of(c);
    return (c.width + B - 1) / B;
}
__device__ __forceinline__ int tiles_y_of(const gsfit_camera& c) {
    const int B = tile_of(c);
    return (c.height + B - 1) / B;
}

// Tile rectangle [x0, x1) x [y0, y1) of a splat with centre (u, w) and
// integer radius r (3DGS): x0 = floor((u - r) / B), x1 = floor(((u + r) + (B -
// 1)) / B), clamped to the view; every operation correctly rounded, so the
// projection and the key emission agree bit for bit.
struct Rect {
    int x0, y0, x1, y1;
};

// B is 8 or 16: x / B and x * (1 / B) are the same real number, so the
// correctly rounded product equals the correctly rounded quotient.
__device__ __forceinline__ Rect tile_rect(float u, float w, float radius, int tiles_x, int tiles_y, int B) {
    const float iB = B == 8 ? 0.125f : 0.0625f, Bm1 = (float)(B - 1);
    Rect t;
    t.x0 = min(tiles_x, max(0, (int)floorf(__fmul_rn(__fsub_rn(u, radius), iB))));
    t.x1 = min(tiles_x, max(0, (int)floorf(__fmul_rn(__fadd_rn(__fadd_rn(u, radius), Bm1), iB))));
    t.y0 = min(tiles_y, max(0, (int)floorf(__fmul_rn(__fsub_rn(w, radius), iB))));
    t.y1 = min(tiles_y, max(0, (int)floorf(__fmul_rn(__fadd_rn(__fadd_rn(w, radius), Bm1), iB))));
    return t;
}

// Exponent of a splat at pixel offset (dx, dy) = pixel - centre, from the
// conic as (a', b', b', c') and the offsets as pairs dxx = (dx, dx),
// dyy = (dy, dy): lin = (a' dx + b' dy, b' dx + c' dy) by packed two-lane
// operations (also the adjoint's d(-power)/d(dx, dy)), then
// power = -1/2 (dx lin.x + dy lin.y) = -1/2 (a' dx^2 + c' dy^2) - b' dx dy.
// Every rounding is explicit, and the forward pass and the adjoint both call
// this, so they take identical skip decisions.
__device__ __forceinline__ float splat_power(float4 cq, float2 dxx, float2 dyy, float2& lin) {
    lin = __ffma2_rn(make_float2(cq.x, cq.y), dxx, __fmul2_rn(make_float2(cq.z, cq.w), dyy));
    return -0.5f * __fmaf_rn(dxx.x, lin.x, __fmul_rn(dyy.x, lin.y));
}

// The same exponent from the conic as stored, (a', b', c', opacity), and the
// offsets as scalars: the same operations in the same order (a packed lane
// rounds like its scalar form, and fx - u = fx + (-u)), hence bit-identical.
__device__ __forceinline__ float splat_power(float4 co, float dx, float dy) {
    const float lx = __fmaf_rn(co.x, dx, __fmul_rn(co.y, dy)), ly = __fmaf_rn(co.y, dx, __fmul_rn(co.z, dy));
    return -0.5f * __fmaf_rn(dx, lx, __fmul_rn(dy, ly));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 16-bit feature copies: one float4 plane entry as four halves / bfloat16s in
// 8 bytes (round to nearest even; widening back is exact).
template <int FT>
__device__ __forceinline__ uint2 pack_features(float4 p) {
    static_assert(FT == GSFIT_FEATURES_F16 || FT == GSFIT_FEATURES_BF16, "16-bit feature types only");
    uint2 q;
    if constexpr (FT == GSFIT_FEATURES_F16) {
        const __half2 a = __floats2half2_rn(p.x, p.y), b = __floats2half2_rn(p.z, p.w);
        q.x = *reinterpret_cast<const uint32_t*>(&a);
        q.y = *reinterpret_cast<const uint32_t*>(&b);
    } else {
        const __nv_bfloat162 a = __floats2bfloat162_rn(p.x, p.y), b = __floats2bfloat162_rn(p.z, p.w);
        q.x = *reinterpret_cast<const uint32_t*>(&a);
        q.y = *reinterpret_cast<const uint32_t*>(&b);
    }
    return q;
}

template <int FT>
__device__ __forceinline__ float4 unpack_features(uint2 q) {
    static_assert(FT == GSFIT_FEATURES_F16 || FT == GSFIT_FEATURES_BF16, "16-bit feature types only");
    float2 a, b;
    if constexpr (FT == GSFIT_FEATURES_F16) {
        a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    } else {
        a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    }
    return make_float4(a.x, a.y, b.x, b.y);
}

// First parameter plane of the 16-bit feature copy: the SH coefficient planes
// 3.. (means, opacity, rotation and scales are always read in float32).
constexpr int kFeaturePlane0 = 3;

// Plane p of Gaussian i: planes 0-2 always from the float32 parameters, the
// SH planes 3.. from the 16-bit copy F when FT selects one.
template <int FT>
__device__ __forceinline__ float4 load_plane(const float4* __restrict__ P, const uint2* __restrict__ F, int n, int p,
                                             int i) {
    if constexpr (FT == GSFIT_FEATURES_F32) {
        return P[(size_t)p * n + i];
    } else {
        if (p < kFeaturePlane0) return P[(size_t)p * n + i];
        return unpack_features<FT>(F[(size_t)(p - kFeaturePlane0) * n + i]);
    }
}

// Adam (Kingma & Ba) with bias correction, shared by the plain update and the
// update fused into the projection adjoint. At step t = done + 1 (done:
// completed steps):
//   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
//   p -= lr (m / (1 - b1^t)) / (sqrt(v) / sqrt(1 - b2^t) + eps).
// Each operation is an explicit round-to-nearest intrinsic, which the
// compiler never contracts, so both kernels compute the same floats from the
// same gradient.
constexpr int kMaxPlanes = 16;

struct LrTable {
    float4 lr[kMaxPlanes];  // the rate of each component of each plane
};

struct AdamCoef {
    float b1, b2, eps;
    float omb1, omb2;  // 1 - b1, 1 - b2
    float s1;          // 1 / (1 - b1^t)
    float rbc2;        // 1 / sqrt(1 - b2^t)
};

__device__ __forceinline__ AdamCoef adam_coef(float b1, float b2, float eps, int32_t done) {
    const int t = done + 1;
    const float bc1 = __fsub_rn(1.0f, powf(b1, (float)t));
    const float bc2 = __fsub_rn(1.0f, powf(b2, (float)t));
    AdamCoef c;
    c.b1 = b1;
    c.b2 = b2;
    c.eps = eps;
    c.omb1 = __fsub_rn(1.0f, b1);
    c.omb2 = __fsub_rn(1.0f, b2);
    c.rbc2 = rsqrtf(bc2);
    c.s1 = __fdiv_rn(1.0f, bc1);
    return c;
}

__device__ __forceinline__ void adam_lane(float& p, float& m, float& v, float g, float lr, const AdamCoef& c) {
    m = __fmaf_rn(c.b1, m, __fmul_rn(c.omb1, g));
    v = __fmaf_rn(c.b2, v, __fmul_rn(__fmul_rn(c.omb2, g), g));
    const float den = __fmaf_rn(sqrtf(v), c.rbc2, c.eps);
    p = __fsub_rn(p, __fdiv_rn(__fmul_rn(lr, __fmul_rn(m, c.s1)), den));
}

__device__ __forceinline__ void adam_update(float4& p, float4& m, float4& v, float4 g, float4 lr,
                                            const AdamCoef& c) {
    adam_lane(p.x, m.x, v.x, g.x, lr.x, c);
    adam_lane(p.y, m.y, v.y, g.y, lr.y, c);
    adam_lane(p.z, m.z, v.z, g.z, lr.z, c);
    adam_lane(p.w, m.w, v.w, g.w, lr.w, c);
}

}  // namespace gsfit
