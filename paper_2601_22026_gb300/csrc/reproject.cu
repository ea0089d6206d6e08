// Depth-guided reprojection of a foveal image to a newer head pose (Section
// 4.3, Eqs. 2-4). The viewer of the paper deforms a mesh by the path tracer's
// first-hit depth in a shader; here the same per-pixel transform runs as a
// kernel and the image is carried to the new view point by point into device
// buffers:
//   1. clear_kernel: the output z-buffer (one uint64 per output pixel).
//   2. splat_kernel, one thread per source pixel: Eqs. 2-4 (far-plane point
//      through the inverse old projection-view matrix, the ray scaled to the
//      pixel's linear depth, the new projection-view matrix), the clip-space
//      position written out, and an atomicMin of (w bits << 32 | source index)
//      on the output pixel it lands on: the nearest source wins, ties to the
//      lower index, independent of thread order.
//   3. resolve_kernel, one thread per output pixel: the winner's colour, or
//      0 and covered = 0 where no source landed (disocclusions).
// All arithmetic is float32; the matrices are kernel parameters.
#include "common.cuh"

namespace gsfit {

namespace {

struct Mat4 {
    float m[16];  // row-major, acting on column vectors
};

constexpr unsigned long long kEmpty = ~0ull;

__global__ void __launch_bounds__(256) clear_kernel(unsigned long long* __restrict__ zbuf, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        zbuf[k] = kEmpty;
}

__global__ void __launch_bounds__(256) splat_kernel(const float* __restrict__ depth, int W, int H, Mat4 inv_old,
                                                    float3 pos_old, Mat4 pv_new, int out_w, int out_h,
                                                    float4* __restrict__ clip,
                                                    unsigned long long* __restrict__ zbuf) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)W * H) return;
    const int y = (int)(k / W), x = (int)(k - (long long)y * W);
    const float d = depth[k];
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (d > 0.0f && isfinite(d)) {
        // Eq. 2: the pixel's point on the far plane of the old view
        const float nx = 2.0f * ((float)x + 0.5f) / (float)W - 1.0f;
        const float ny = 2.0f * ((float)y + 0.5f) / (float)H - 1.0f;
        const float* A = inv_old.m;
        const float hx = A[0] * nx + A[1] * ny + A[2] + A[3];
        const float hy = A[4] * nx + A[5] * ny + A[6] + A[7];
        const float hz = A[8] * nx + A[9] * ny + A[10] + A[11];
        const float hw = A[12] * nx + A[13] * ny + A[14] + A[15];
        const float fx = hx / hw - pos_old.x, fy = hy / hw - pos_old.y, fz = hz / hw - pos_old.z;
        // Eq. 3: along that ray, at the pixel's linear depth
        const float s = d * rsqrtf(fx * fx + fy * fy + fz * fz);
        const float wx = pos_old.x + fx * s, wy = pos_old.y + fy * s, wz = pos_old.z + fz * s;
        // Eq. 4: into the new view's clip space
        const float* B = pv_new.m;
        c.x = B[0] * wx + B[1] * wy + B[2] * wz + B[3];
        c.y = B[4] * wx + B[5] * wy + B[6] * wz + B[7];
        c.z = B[8] * wx + B[9] * wy + B[10] * wz + B[11];
        c.w = B[12] * wx + B[13] * wy + B[14] * wz + B[15];
        if (c.w > 0.0f) {
            const float px = (c.x / c.w + 1.0f) * 0.5f * (float)out_w - 0.5f;
            const float py = (c.y / c.w + 1.0f) * 0.5f * (float)out_h - 0.5f;
            const float rx = floorf(px + 0.5f), ry = floorf(py + 0.5f);
            if (rx >= 0.0f && ry >= 0.0f && rx < (float)out_w && ry < (float)out_h) {
                const long long t = (long long)ry * out_w + (long long)rx;
                const unsigned long long key = ((unsigned long long)__float_as_uint(c.w) << 32) | (unsigned long long)k;
                atomicMin(zbuf + t, key);
            }
        }
    }
    if (clip) clip[k] = c;
}

__global__ void __launch_bounds__(256) resolve_kernel(const float* __restrict__ rgb, long long src_plane,
                                                      const unsigned long long* __restrict__ zbuf, long long n_out,
                                                      float* __restrict__ out_rgb, uint8_t* __restrict__ covered) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_out) return;
    const unsigned long long key = zbuf[t];
    if (key == kEmpty) {
        out_rgb[t] = out_rgb[t + n_out] = out_rgb[t + 2 * n_out] = 0.0f;
        covered[t] = 0;
        return;
    }
    const long long s = (long long)(key & 0xffffffffull);
    out_rgb[t] = rgb[s];
    out_rgb[t + n_out] = rgb[s + src_plane];
    out_rgb[t + 2 * n_out] = rgb[s + 2 * src_plane];
    covered[t] = 1;
}

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" int gsfit_reproject(const float* rgb, const float* depth, int32_t width, int32_t height,
                               const float* inv_pv_old, const float* pos_old, const float* pv_new, int32_t out_w,
                               int32_t out_h, float* clip, unsigned long long* zbuf, float* out_rgb,
                               uint8_t* covered, cudaStream_t stream) {
    if (!rgb || !depth || !inv_pv_old || !pos_old || !pv_new || !zbuf || !out_rgb || !covered || width < 1 ||
        height < 1 || out_w < 1 || out_h < 1 || (long long)width * height >= (1ll << 32) ||
        (clip && (reinterpret_cast<uintptr_t>(clip) % 16) != 0) || (reinterpret_cast<uintptr_t>(zbuf) % 8) != 0)
        return GSFIT_ERR_INVALID_ARG;
    Mat4 a, b;
    for (int i = 0; i < 16; ++i) {
        a.m[i] = inv_pv_old[i];
        b.m[i] = pv_new[i];
    }
    const long long n_src = (long long)width * height, n_out = (long long)out_w * out_h;
    const int clear_blocks = (int)std::min<long long>((n_out + 255) / 256, 4096);
    clear_kernel<<<clear_blocks, 256, 0, stream>>>(zbuf, n_out);
    GSFIT_LAUNCH_CHECK();
    splat_kernel<<<(unsigned)((n_src + 255) / 256), 256, 0, stream>>>(
        depth, width, height, a, make_float3(pos_old[0], pos_old[1], pos_old[2]), b, out_w, out_h,
        reinterpret_cast<float4*>(clip), zbuf);
    GSFIT_LAUNCH_CHECK();
    resolve_kernel<<<(unsigned)((n_out + 255) / 256), 256, 0, stream>>>(rgb, n_src, zbuf, n_out, out_rgb, covered);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}
