// First-hit point-cloud seeding (Section 4.1): rays cast toward the CT volume
// from viewpoints around it keep their first significant hit, the first point
// where the transfer function's opacity of the trilinearly interpolated volume
// reaches alpha_min. One thread per ray: slab test against the volume's box,
// fixed-step march from the entry point, 12 bisection steps on the bracketing
// interval. The march is bounded by the box's extent / step samples.
#include <cmath>

#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kMaxKnots = 8;

struct Volume {
    const int16_t* hu;
    int nx, ny, nz;
    float ox, oy, oz, vox;
};

struct TfTable {
    int n;
    float hu[kMaxKnots], r[kMaxKnots], g[kMaxKnots], b[kMaxKnots], a[kMaxKnots];
};

__device__ __forceinline__ float voxel_at(const Volume& V, int x, int y, int z) {
    x = min(max(x, 0), V.nx - 1);
    y = min(max(y, 0), V.ny - 1);
    z = min(max(z, 0), V.nz - 1);
    return (float)__ldg(V.hu + ((size_t)z * V.ny + y) * V.nx + x);
}

// Trilinear HU at world point p (voxel centres at origin + (i + 0.5) voxel).
__device__ float sample_hu(const Volume& V, float px, float py, float pz) {
    const float cx = (px - V.ox) / V.vox - 0.5f, cy = (py - V.oy) / V.vox - 0.5f, cz = (pz - V.oz) / V.vox - 0.5f;
    const float fx = floorf(cx), fy = floorf(cy), fz = floorf(cz);
    const int x0 = (int)fx, y0 = (int)fy, z0 = (int)fz;
    const float tx = cx - fx, ty = cy - fy, tz = cz - fz;
    float c[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
            c[dz][dy] = voxel_at(V, x0, y0 + dy, z0 + dz) * (1.0f - tx) + voxel_at(V, x0 + 1, y0 + dy, z0 + dz) * tx;
    const float c0 = c[0][0] * (1.0f - ty) + c[0][1] * ty;
    const float c1 = c[1][0] * (1.0f - ty) + c[1][1] * ty;
    return c0 * (1.0f - tz) + c1 * tz;
}

// Piecewise-linear transfer function, clamped outside the knots.
__device__ float4 tf_eval(const TfTable& T, float hu) {
    if (hu <= T.hu[0]) return make_float4(T.r[0], T.g[0], T.b[0], T.a[0]);
    for (int k = 1; k < T.n; ++k) {
        if (hu <= T.hu[k]) {
            const float w = (hu - T.hu[k - 1]) / (T.hu[k] - T.hu[k - 1]);
            return make_float4(T.r[k - 1] + w * (T.r[k] - T.r[k - 1]), T.g[k - 1] + w * (T.g[k] - T.g[k - 1]),
                               T.b[k - 1] + w * (T.b[k] - T.b[k - 1]), T.a[k - 1] + w * (T.a[k] - T.a[k - 1]));
        }
    }
    const int l = T.n - 1;
    return make_float4(T.r[l], T.g[l], T.b[l], T.a[l]);
}

__global__ void __launch_bounds__(256) first_hit_kernel(Volume V, TfTable T, const gsfit_camera* __restrict__ cams,
                                                        int n_views, int rays_x, int rays_y, float step,
                                                        float alpha_min, float4* __restrict__ points,
                                                        float4* __restrict__ colour) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_view = (long long)rays_x * rays_y;
    if (r >= per_view * n_views) return;
    const int v = (int)(r / per_view);
    const int rem = (int)(r - (long long)v * per_view);
    const int j = rem / rays_x, i = rem - j * rays_x;
    const gsfit_camera& cam = cams[v];
    const float* R = cam.viewmat;
    const float u = ((float)i + 0.5f) * (float)cam.width / (float)rays_x - 0.5f;
    const float w = ((float)j + 0.5f) * (float)cam.height / (float)rays_y - 0.5f;
    // camera-space direction, to world space with R^T
    const float dcx = (u - cam.cx) / cam.fx, dcy = (w - cam.cy) / cam.fy, dcz = 1.0f;
    float dx = R[0] * dcx + R[4] * dcy + R[8] * dcz;
    float dy = R[1] * dcx + R[5] * dcy + R[9] * dcz;
    float dz = R[2] * dcx + R[6] * dcy + R[10] * dcz;
    const float inv_len = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv_len;
    dy *= inv_len;
    dz *= inv_len;
    const float ox = cam.campos[0], oy = cam.campos[1], oz = cam.campos[2];
    // slab test against the volume's box
    const float lo[3] = {V.ox, V.oy, V.oz};
    const float hi[3] = {V.ox + V.nx * V.vox, V.oy + V.ny * V.vox, V.oz + V.nz * V.vox};
    const float o[3] = {ox, oy, oz}, d[3] = {dx, dy, dz};
    float t0 = 0.0f, t1 = 3.4e38f;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < lo[a] || o[a] > hi[a]) miss = true;
        } else {
            float ta = (lo[a] - o[a]) / d[a], tb = (hi[a] - o[a]) / d[a];
            if (ta > tb) {
                const float x = ta;
                ta = tb;
                tb = x;
            }
            t0 = fmaxf(t0, ta);
            t1 = fminf(t1, tb);
        }
    }
    float4 pt = make_float4(0.f, 0.f, 0.f, 0.f), col = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!miss && t0 <= t1) {
        const int n_samples = (int)floorf((t1 - t0) / step) + 1;  // bounded march
        float t_prev = t0;
        for (int k = 0; k < n_samples; ++k) {
            const float t = t0 + (float)k * step;
            if (tf_eval(T, sample_hu(V, ox + t * dx, oy + t * dy, oz + t * dz)).w >= alpha_min) {
                float a = t_prev, b = t;  // opacity below alpha_min at a (or a == b), at or above at b
                for (int it = 0; it < 12; ++it) {
                    const float m = 0.5f * (a + b);
                    if (tf_eval(T, sample_hu(V, ox + m * dx, oy + m * dy, oz + m * dz)).w >= alpha_min)
                        b = m;
                    else
                        a = m;
                }
                const float hx = ox + b * dx, hy = oy + b * dy, hz = oz + b * dz;
                pt = make_float4(hx, hy, hz, 1.0f);
                col = tf_eval(T, sample_hu(V, hx, hy, hz));
                break;
            }
            t_prev = t;
        }
    }
    points[r] = pt;
    colour[r] = col;
}

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_first_hit(const int16_t* hu, int32_t nx, int32_t ny, int32_t nz, const float* origin,
                               float voxel, const float* tf_knots, int32_t n_knots, const gsfit_camera* cams,
                               int32_t n_views, int32_t rays_x, int32_t rays_y, float step, float alpha_min,
                               float* points, float* colour, cudaStream_t stream) {
    if (!hu || !origin || !tf_knots || !cams || !points || !colour || nx < 1 || ny < 1 || nz < 1 ||
        !(voxel > 0.0f) || n_knots < 1 || n_knots > kMaxKnots || n_views < 1 || n_views > GSFIT_MAX_VIEWS ||
        rays_x < 1 || rays_y < 1 || !(step > 0.0f) || (reinterpret_cast<uintptr_t>(points) % 16) ||
        (reinterpret_cast<uintptr_t>(colour) % 16))
        return GSFIT_ERR_INVALID_ARG;
    for (int k = 1; k < n_knots; ++k)
        if (!(tf_knots[5 * k] > tf_knots[5 * (k - 1)])) return GSFIT_ERR_INVALID_ARG;
    Volume V{hu, nx, ny, nz, origin[0], origin[1], origin[2], voxel};
    TfTable T;
    T.n = n_knots;
    for (int k = 0; k < kMaxKnots; ++k) {
        const int q = k < n_knots ? k : n_knots - 1;
        T.hu[k] = tf_knots[5 * q];
        T.r[k] = tf_knots[5 * q + 1];
        T.g[k] = tf_knots[5 * q + 2];
        T.b[k] = tf_knots[5 * q + 3];
        T.a[k] = tf_knots[5 * q + 4];
    }
    const long long n_rays = (long long)n_views * rays_x * rays_y;
    first_hit_kernel<<<(unsigned)((n_rays + 255) / 256), 256, 0, stream>>>(
        V, T, cams, n_views, rays_x, rays_y, step, alpha_min, reinterpret_cast<float4*>(points),
        reinterpret_cast<float4*>(colour));
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
