// EWA projection with spherical-harmonic colour, and its adjoint.
//
// The peripheral model is a 3DGS model (Section 4.2); its projection is the
// EWA splat of 3DGS (not written out in the paper): Sigma = R(q) S^2 R(q)^T,
// Sigma' = J W Sigma W^T J^T + 0.3 I, conic = Sigma'^-1, radius =
// ceil(3 sqrt(lambda_max)), colour = SH(view direction) + 0.5 clamped at 0.
//
// Design: one thread per Gaussian loops over all views of the batch. The
// Gaussian's float4 planes are read once (coalesced: a warp reads 512
// contiguous bytes per plane) and kept in registers; the camera table sits in
// shared memory. Culled records write only their 16-byte centre record (radius
// 0) and a zero tile count, so narrow foveal crops cost little.
#include "common.cuh"

namespace gsfit {

// Adds one to the device step count after an Adam update (adam.cu).
int step_increment(int32_t* step, cudaStream_t s);

namespace {

// Real SH constants N_lm * (polynomial factor), from
// N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2 for m != 0) and the
// Condon-Shortley phase; the basis is ordered m = -l..l per band.
constexpr float kY00 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kY2xy = 1.0925484305920792f;   // m = -2 (xy), -1 (yz), 1 (xz)
constexpr float kY20 = 0.31539156525252005f;   // m = 0: (3 z^2 - 1)
constexpr float kY22 = 0.54627421529603959f;   // m = 2: (x^2 - y^2)
constexpr float kY33 = 0.59004358992664352f;   // m = -3, 3
constexpr float kY32a = 2.8906114426405547f;   // m = -2: xyz
constexpr float kY31 = 0.45704579946446577f;   // m = -1, 1: (5 z^2 - 1)
constexpr float kY30 = 0.37317633259011540f;   // m = 0: z (5 z^2 - 3)
constexpr float kY32b = 1.4453057213202773f;   // m = 2: z (x^2 - y^2)

template <int DEG>
struct SH {
    static constexpr int K = (DEG + 1) * (DEG + 1);
};

// Y_k(d) for the unit direction d.
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kY00;
    if (DEG >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (DEG >= 2) {
        Y[4] = kY2xy * x * y;
        Y[5] = -kY2xy * y * z;
        Y[6] = kY20 * (3.0f * z * z - 1.0f);
        Y[7] = -kY2xy * x * z;
        Y[8] = kY22 * (x * x - y * y);
    }
    if (DEG >= 3) {
        const float z5 = 5.0f * z * z;
        Y[9] = -kY33 * y * (3.0f * x * x - y * y);
        Y[10] = kY32a * x * y * z;
        Y[11] = -kY31 * y * (z5 - 1.0f);
        Y[12] = kY30 * z * (z5 - 3.0f);
        Y[13] = -kY31 * x * (z5 - 1.0f);
        Y[14] = kY32b * z * (x * x - y * y);
        Y[15] = -kY33 * x * (x * x - 3.0f * y * y);
    }
}

// sum_k w_k dY_k/d(x, y, z) for the polynomial forms above.
template <int DEG>
__device__ __forceinline__ float3 sh_basis_vjp(float x, float y, float z, const float* w) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (DEG >= 1) {
        gy -= kY1 * w[1];
        gz += kY1 * w[2];
        gx -= kY1 * w[3];
    }
    if (DEG >= 2) {
        gx += kY2xy * y * w[4];
        gy += kY2xy * x * w[4];
        gy -= kY2xy * z * w[5];
        gz -= kY2xy * y * w[5];
        gz += 6.0f * kY20 * z * w[6];
        gx -= kY2xy * z * w[7];
        gz -= kY2xy * x * w[7];
        gx += 2.0f * kY22 * x * w[8];
        gy -= 2.0f * kY22 * y * w[8];
    }
    if (DEG >= 3) {
        const float z5m1 = 5.0f * z * z - 1.0f;
        gx -= 6.0f * kY33 * x * y * w[9];
        gy -= 3.0f * kY33 * (x * x - y * y) * w[9];
        gx += kY32a * y * z * w[10];
        gy += kY32a * x * z * w[10];
        gz += kY32a * x * y * w[10];
        gy -= kY31 * z5m1 * w[11];
        gz -= 10.0f * kY31 * y * z * w[11];
        gz += kY30 * (15.0f * z * z - 3.0f) * w[12];
        gx -= kY31 * z5m1 * w[13];
        gz -= 10.0f * kY31 * x * z * w[13];
        gx += 2.0f * kY32b * x * z * w[14];
        gy -= 2.0f * kY32b * y * z * w[14];
        gz += kY32b * (x * x - y * y) * w[14];
        gx -= 3.0f * kY33 * (x * x - y * y) * w[15];
        gy += 6.0f * kY33 * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

// Camera-space coordinate row k in the fixed order ((R_k0 x + R_k1 y) + R_k2 z)
// + t_k with every operation correctly rounded (no contraction): depth cull,
// depth key and tile rectangle are decided on these bits.
__device__ __forceinline__ float cam_row(const gsfit_camera& c, int k, float x, float y, float z) {
    float s = __fadd_rn(__fmul_rn(c.viewmat[4 * k + 0], x), __fmul_rn(c.viewmat[4 * k + 1], y));
    s = __fadd_rn(s, __fmul_rn(c.viewmat[4 * k + 2], z));
    return __fadd_rn(s, c.viewmat[4 * k + 3]);
}

// Rotation matrix of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Compensated a*c - b*b (Kahan's two-product difference): the determinant of
// the dilated 2D covariance keeps full float32 accuracy even for long thin
// splats whose a*c and b*b nearly cancel.
__device__ __forceinline__ float det2(float a, float b, float c) {
    const float bb = b * b;
    const float e = fmaf(-b, b, bb);
    const float f = fmaf(a, c, -bb);
    return f + e;
}

struct Gauss {
    float mx, my, mz, logit;
    float qw, qx, qy, qz, qn;
    float s[3];
    float Sig[6];  // xx xy xz yy yz zz
    float R[9];
};

template <int FT>
__device__ __forceinline__ void load_gauss(const float4* __restrict__ P, const uint2* __restrict__ F, int n, int i,
                                           Gauss& g) {
    const float4 p0 = P[i];
    const float4 p1 = load_plane<FT>(P, F, n, 1, i);
    const float4 p2 = load_plane<FT>(P, F, n, 2, i);
    g.mx = p0.x; g.my = p0.y; g.mz = p0.z; g.logit = p0.w;
    g.qn = sqrtf(p1.x * p1.x + p1.y * p1.y + p1.z * p1.z + p1.w * p1.w);
    const float inv = 1.0f / g.qn;
    g.qw = p1.x * inv; g.qx = p1.y * inv; g.qy = p1.z * inv; g.qz = p1.w * inv;
    g.s[0] = expf(p2.x); g.s[1] = expf(p2.y); g.s[2] = expf(p2.z);
    quat_rot(g.qw, g.qx, g.qy, g.qz, g.R);
    const float* R = g.R;
    const float s0 = g.s[0] * g.s[0], s1 = g.s[1] * g.s[1], s2 = g.s[2] * g.s[2];
    // Sigma_ij = sum_k R_ik s_k^2 R_jk
    g.Sig[0] = R[0] * R[0] * s0 + R[1] * R[1] * s1 + R[2] * R[2] * s2;
    g.Sig[1] = R[0] * R[3] * s0 + R[1] * R[4] * s1 + R[2] * R[5] * s2;
    g.Sig[2] = R[0] * R[6] * s0 + R[1] * R[7] * s1 + R[2] * R[8] * s2;
    g.Sig[3] = R[3] * R[3] * s0 + R[4] * R[4] * s1 + R[5] * R[5] * s2;
    g.Sig[4] = R[3] * R[6] * s0 + R[4] * R[7] * s1 + R[5] * R[8] * s2;
    g.Sig[5] = R[6] * R[6] * s0 + R[7] * R[7] * s1 + R[8] * R[8] * s2;
}

template <int DEG, int FT>
__device__ __forceinline__ void load_sh(const float4* __restrict__ P, const uint2* __restrict__ F, int n, int i,
                                        float* sh) {
    constexpr int K3 = 3 * SH<DEG>::K;
    constexpr int NP = (K3 + 3) / 4;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float4 q = load_plane<FT>(P, F, n, 3 + p, i);
        if (4 * p + 0 < K3) sh[4 * p + 0] = q.x;
        if (4 * p + 1 < K3) sh[4 * p + 1] = q.y;
        if (4 * p + 2 < K3) sh[4 * p + 2] = q.z;
        if (4 * p + 3 < K3) sh[4 * p + 3] = q.w;
    }
}

// Per-view geometric quantities shared by the forward and adjoint passes.
struct ViewGeom {
    float tx, ty, tz;
    float rx, ry;          // t_x/t_z, t_y/t_z after the frustum guard
    bool gx, gy;           // guard active
    float M0[3], M1[3];    // rows of J W
    float a, b, c, det;    // dilated 2D covariance
};

__device__ __forceinline__ void view_geom(const gsfit_camera& cam, const Gauss& g, ViewGeom& o) {
    o.tx = cam_row(cam, 0, g.mx, g.my, g.mz);
    o.ty = cam_row(cam, 1, g.mx, g.my, g.mz);
    o.tz = cam_row(cam, 2, g.mx, g.my, g.mz);
    const float limx = kFrustumGuard * (0.5f * (float)cam.width / cam.fx);
    const float limy = kFrustumGuard * (0.5f * (float)cam.height / cam.fy);
    const float rx = o.tx / o.tz, ry = o.ty / o.tz;
    o.gx = (rx < -limx) || (rx > limx);
    o.gy = (ry < -limy) || (ry > limy);
    o.rx = fminf(limx, fmaxf(-limx, rx));
    o.ry = fminf(limy, fmaxf(-limy, ry));
    const float iz = 1.0f / o.tz;
    const float J00 = cam.fx * iz, J02 = -cam.fx * o.rx * iz;
    const float J11 = cam.fy * iz, J12 = -cam.fy * o.ry * iz;
    const float* W = cam.viewmat;  // rows 0..2 at W[0..2], W[4..6], W[8..10]
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.M0[j] = J00 * W[j] + J02 * W[8 + j];
        o.M1[j] = J11 * W[4 + j] + J12 * W[8 + j];
    }
    const float* S = g.Sig;
    const float sm0x = S[0] * o.M0[0] + S[1] * o.M0[1] + S[2] * o.M0[2];
    const float sm0y = S[1] * o.M0[0] + S[3] * o.M0[1] + S[4] * o.M0[2];
    const float sm0z = S[2] * o.M0[0] + S[4] * o.M0[1] + S[5] * o.M0[2];
    const float sm1x = S[0] * o.M1[0] + S[1] * o.M1[1] + S[2] * o.M1[2];
    const float sm1y = S[1] * o.M1[0] + S[3] * o.M1[1] + S[4] * o.M1[2];
    const float sm1z = S[2] * o.M1[0] + S[4] * o.M1[1] + S[5] * o.M1[2];
    o.a = o.M0[0] * sm0x + o.M0[1] * sm0y + o.M0[2] * sm0z + kDilation;
    o.b = o.M0[0] * sm1x + o.M0[1] * sm1y + o.M0[2] * sm1z;
    o.c = o.M1[0] * sm1x + o.M1[1] * sm1y + o.M1[2] * sm1z + kDilation;
    o.det = det2(o.a, o.b, o.c);
}

template <int DEG, int FT>
__global__ void __launch_bounds__(256, 3) project_kernel(const float4* __restrict__ P, const uint2* __restrict__ F, int n,
                                                      const gsfit_camera* __restrict__ cams_g, int n_views,
                                                      float4* __restrict__ xyd, float4* __restrict__ conic,
                                                      float4* __restrict__ rgb, uint32_t* __restrict__ tiles) {
    extern __shared__ gsfit_camera cams[];
    load_cameras(cams, cams_g, n_views);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int K = SH<DEG>::K;
    Gauss g;
    load_gauss<FT>(P, F, n, i, g);
    float sh[3 * K];
    load_sh<DEG, FT>(P, F, n, i, sh);
    const float opacity = 1.0f / (1.0f + expf(-g.logit));

#pragma unroll 2
    for (int v = 0; v < n_views; ++v) {
        const gsfit_camera& cam = cams[v];
        const size_t r = (size_t)v * n + i;
        ViewGeom vg;
        view_geom(cam, g, vg);
        if (!(vg.tz > cam.near_plane) || !(vg.det > 0.0f)) {
            xyd[r] = make_float4(0.f, 0.f, vg.tz, 0.f);
            tiles[r] = 0u;
            continue;
        }
        const float inv_det = 1.0f / fmaxf(vg.det, 1e-12f);
        const float mid = 0.5f * (vg.a + vg.c);
        const float lambda = mid + sqrtf(fmaxf(0.1f, mid * mid - vg.det));
        const float radius = ceilf(3.0f * sqrtf(lambda));
        // centre, correctly rounded in a fixed order: (fx * t_x) / t_z + cx
        const float u = __fadd_rn(__fdiv_rn(__fmul_rn(cam.fx, vg.tx), vg.tz), cam.cx);
        const float w = __fadd_rn(__fdiv_rn(__fmul_rn(cam.fy, vg.ty), vg.tz), cam.cy);
        const Rect rc = tile_rect(u, w, radius, tiles_x_of(cam), tiles_y_of(cam), tile_of(cam));
        const uint32_t nt = (uint32_t)((rc.x1 - rc.x0) * (rc.y1 - rc.y0));
        if (nt == 0u) {
            xyd[r] = make_float4(u, w, vg.tz, 0.f);
            tiles[r] = 0u;
            continue;
        }
        // view-dependent colour
        float dx = g.mx - cam.campos[0], dy = g.my - cam.campos[1], dz = g.mz - cam.campos[2];
        const float idist = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= idist; dy *= idist; dz *= idist;
        float Y[K];
        sh_basis<DEG>(dx, dy, dz, Y);
        float col[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += Y[k] * sh[3 * k + ch];
            col[ch] = acc + 0.5f;
        }
        if (!(opacity >= 0.0f) || !isfinite(col[0] + col[1] + col[2])) {  // non-finite parameters: culled
            xyd[r] = make_float4(u, w, vg.tz, 0.f);
            tiles[r] = 0u;
            continue;
        }
        const float mask = (col[0] < 0.f ? 1.f : 0.f) + (col[1] < 0.f ? 2.f : 0.f) + (col[2] < 0.f ? 4.f : 0.f);
        xyd[r] = make_float4(u, w, vg.tz, radius);
        conic[r] = make_float4(vg.c * inv_det, -vg.b * inv_det, vg.a * inv_det, opacity);
        rgb[r] = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), mask);
        tiles[r] = nt;
    }
}

// The adjoint of one binned (view, Gaussian) record: from the accumulated 2D
// gradients (ga: du, dv, dopacity; gb: da', db', dc'; gc: dr, dg, db) through
// the conic, the EWA covariance, the Jacobian and the camera transform, plus
// the view-direction term of the SH colour. Returns dL/dmean (this view's
// part), dL/dSigma (xx xy xz yy yz zz) and the colour gradient with the clamp
// mask (cm.w) applied.
template <int DEG, int FT>
__device__ __forceinline__ void record_bwd(const gsfit_camera& cam, const Gauss& g, float4 ga, float4 gb, float4 gc,
                                           float4 cq, float4 cm, const float4* __restrict__ P,
                                           const uint2* __restrict__ F, int n, int i, float (&dmean)[3],
                                           float (&dSig)[6], float (&gcol)[3]) {
    ViewGeom vg;
    view_geom(cam, g, vg);
    const float iz = 1.0f / vg.tz, iz2 = iz * iz;
    float dtx = ga.x * cam.fx * iz;
    float dty = ga.y * cam.fy * iz;
    float dtz = -(ga.x * cam.fx * vg.tx + ga.y * cam.fy * vg.ty) * iz2;

    // conic Q = S^-1: dL/dS = -Q G Q with G = [[da', db'/2], [db'/2, dc']]
    const float q00 = cq.x, q01 = cq.y, q11 = cq.z;
    const float g00 = gb.x, g01 = 0.5f * gb.y, g11 = gb.z;
    const float t00 = q00 * g00 + q01 * g01, t01 = q00 * g01 + q01 * g11;
    const float t10 = q01 * g00 + q11 * g01, t11 = q01 * g01 + q11 * g11;
    const float dS00 = -(t00 * q00 + t01 * q01);
    const float dS01 = -(t00 * q01 + t01 * q11);
    const float dS11 = -(t10 * q01 + t11 * q11);

    // S = M Sigma M^T: dSigma = M^T dS M; dM = 2 dS M Sigma
    const float* M0 = vg.M0;
    const float* M1 = vg.M1;
    float u0[3], u1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        u0[j] = dS00 * M0[j] + dS01 * M1[j];
        u1[j] = dS01 * M0[j] + dS11 * M1[j];
    }
    dSig[0] = M0[0] * u0[0] + M1[0] * u1[0];
    dSig[1] = M0[0] * u0[1] + M1[0] * u1[1];
    dSig[2] = M0[0] * u0[2] + M1[0] * u1[2];
    dSig[3] = M0[1] * u0[1] + M1[1] * u1[1];
    dSig[4] = M0[1] * u0[2] + M1[1] * u1[2];
    dSig[5] = M0[2] * u0[2] + M1[2] * u1[2];
    const float* S = g.Sig;
    float dM0[3], dM1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float sk0 = (k == 0) ? S[0] : (k == 1) ? S[1] : S[2];
        const float sk1 = (k == 0) ? S[1] : (k == 1) ? S[3] : S[4];
        const float sk2 = (k == 0) ? S[2] : (k == 1) ? S[4] : S[5];
        dM0[k] = 2.f * (u0[0] * sk0 + u0[1] * sk1 + u0[2] * sk2);
        dM1[k] = 2.f * (u1[0] * sk0 + u1[1] * sk1 + u1[2] * sk2);
    }
    // M = J W: dJ = dM W^T (only J00, J02, J11, J12 are non-zero)
    const float* W = cam.viewmat;
    const float dJ00 = dM0[0] * W[0] + dM0[1] * W[1] + dM0[2] * W[2];
    const float dJ02 = dM0[0] * W[8] + dM0[1] * W[9] + dM0[2] * W[10];
    const float dJ11 = dM1[0] * W[4] + dM1[1] * W[5] + dM1[2] * W[6];
    const float dJ12 = dM1[0] * W[8] + dM1[1] * W[9] + dM1[2] * W[10];
    dtz += -dJ00 * cam.fx * iz2 - dJ11 * cam.fy * iz2 + dJ02 * cam.fx * vg.rx * iz2 + dJ12 * cam.fy * vg.ry * iz2;
    const float drx = -dJ02 * cam.fx * iz, dry = -dJ12 * cam.fy * iz;
    if (!vg.gx) {
        dtx += drx * iz;
        dtz -= drx * vg.tx * iz2;
    }
    if (!vg.gy) {
        dty += dry * iz;
        dtz -= dry * vg.ty * iz2;
    }
    // t = W mu + t_w
#pragma unroll
    for (int j = 0; j < 3; ++j) dmean[j] = W[j] * dtx + W[4 + j] * dty + W[8 + j] * dtz;
    // colour: clamped channels pass no gradient
    const int mask = (int)cm.w;
    gcol[0] = (mask & 1) ? 0.f : gc.x;
    gcol[1] = (mask & 2) ? 0.f : gc.y;
    gcol[2] = (mask & 4) ? 0.f : gc.z;
    if (DEG > 0) {
        // colour = sum_k c_k Y_k(d), d = (mu - campos) / |mu - campos|
        constexpr int K = SH<DEG>::K;
        float dx = g.mx - cam.campos[0], dy = g.my - cam.campos[1], dz = g.mz - cam.campos[2];
        const float idist = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= idist; dy *= idist; dz *= idist;
        float sh[3 * K];
        load_sh<DEG, FT>(P, F, n, i, sh);
        float wk[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            wk[k] = sh[3 * k + 0] * gcol[0] + sh[3 * k + 1] * gcol[1] + sh[3 * k + 2] * gcol[2];
        const float3 dd = sh_basis_vjp<DEG>(dx, dy, dz, wk);
        const float proj = dx * dd.x + dy * dd.y + dz * dd.z;
        dmean[0] += (dd.x - dx * proj) * idist;
        dmean[1] += (dd.y - dy * proj) * idist;
        dmean[2] += (dd.z - dz * proj) * idist;
    }
}

// Adjoint of project_kernel: one thread per Gaussian walks the views where the
// Gaussian was binned. Per view it reads the record's accumulated 2D
// gradients (zeroing them for the next iteration) and chains them back
// (record_bwd) while the next binned view's record loads are in flight; the
// sums over views then go through the opacity sigmoid, the SH coefficients
// (accumulators in shared memory) and dL/dSigma to scale and rotation once.
constexpr int kProjBwdThreads = 256;

// Accumulator k of this thread's SH gradient; [k][thread] layout, so a warp's
// accesses hit 32 different banks.
__device__ __forceinline__ float& dsh_acc(float* s_dsh, int k) { return s_dsh[k * kProjBwdThreads + threadIdx.x]; }

// The loads of one binned record: 2D gradients and the record's conic and colour mask.
struct RecIn {
    float4 ga, gb, gc, cq, cm;
};
__device__ __forceinline__ RecIn load_rec(const float4* __restrict__ grad2d, const float4* __restrict__ conic,
                                          const float4* __restrict__ rgbm, size_t r) {
    RecIn x;
    x.ga = grad2d[4 * r + 0];
    x.gb = grad2d[4 * r + 1];
    x.gc = grad2d[4 * r + 2];
    x.cq = __ldg(conic + r);
    x.cm = __ldg(rgbm + r);
    return x;
}

__device__ __forceinline__ bool finite4(float4 q) {
    return isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w);
}

// The gradient of Gaussian i summed over the views that binned it: planes
// 0-2 (means and opacity logit, quaternion, log-scales) in gq, the SH planes
// in this thread's shared-memory accumulators, which the caller zeroed.
// Zeroes the records' 2D gradients it reads. Returns false, with gq zero,
// for a Gaussian that no view binned: it contributes to no pixel, so its
// gradient is zero (also where its parameters are not finite and the chain
// would give 0 x NaN). P and F carry no __restrict__ here: the fused Adam
// kernel updates them in place after this returns. (project_bwd_kernel keeps
// its own copy of this chain: calling this function from it measured 5%
// slower.)
template <int DEG, int FT>
__device__ __forceinline__ bool gaussian_grad(const float4* P, const uint2* F, int n, int i,
                                              const gsfit_camera* cams, int n_views,
                                              const float4* __restrict__ xyd, const float4* __restrict__ conic,
                                              const float4* __restrict__ rgbm, float4* __restrict__ grad2d,
                                              float* s_dsh, float4 (&gq)[3]) {
    constexpr int K = SH<DEG>::K;
    Gauss g;
    load_gauss<FT>(P, F, n, i, g);

    float dmean[3] = {0.f, 0.f, 0.f};
    float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx xy xz yy yz zz (symmetric, dL/dSigma_ij)
    float dop = 0.f;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    bool binned = false;  // some view binned this Gaussian

    for (int v0 = 0; v0 < n_views; v0 += 32) {
        // visibility of up to 32 views first: independent loads, one latency
        uint32_t vis = 0;
        const int vn = min(32, n_views - v0);
#pragma unroll 8
        for (int k = 0; k < vn; ++k)
            if (__ldg(&xyd[(size_t)(v0 + k) * n + i].w) != 0.0f) vis |= 1u << k;
        if (!vis) continue;
        binned = true;
        int v = v0 + __ffs(vis) - 1;
        vis &= vis - 1;
        RecIn cur = load_rec(grad2d, conic, rgbm, (size_t)v * n + i);
        for (;;) {
            // the next binned view's loads go out before this view's chain
            const int vnext = vis ? v0 + __ffs(vis) - 1 : -1;
            vis &= vis - 1;
            RecIn nxt;
            if (vnext >= 0) nxt = load_rec(grad2d, conic, rgbm, (size_t)vnext * n + i);
            const size_t r = (size_t)v * n + i;
            grad2d[4 * r + 0] = zero;  // the adjoint's atomics fill these three
            grad2d[4 * r + 1] = zero;
            grad2d[4 * r + 2] = zero;
            const gsfit_camera& cam = cams[v];
            float dm[3], dS[6], gcol[3];
            record_bwd<DEG, FT>(cam, g, cur.ga, cur.gb, cur.gc, cur.cq, cur.cm, P, F, n, i, dm, dS, gcol);
            dmean[0] += dm[0]; dmean[1] += dm[1]; dmean[2] += dm[2];
            dop += cur.ga.z;
#pragma unroll
            for (int k = 0; k < 6; ++k) dSig[k] += dS[k];
            float dx = g.mx - cam.campos[0], dy = g.my - cam.campos[1], dz = g.mz - cam.campos[2];
            const float idist = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= idist; dy *= idist; dz *= idist;
            float Y[K];
            sh_basis<DEG>(dx, dy, dz, Y);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dsh_acc(s_dsh, 3 * k + 0) += Y[k] * gcol[0];
                dsh_acc(s_dsh, 3 * k + 1) += Y[k] * gcol[1];
                dsh_acc(s_dsh, 3 * k + 2) += Y[k] * gcol[2];
            }
            if (vnext < 0) break;
            v = vnext;
            cur = nxt;
        }
    }
    if (!binned) {
        gq[0] = gq[1] = gq[2] = zero;
        return false;
    }
    const float opacity = 1.0f / (1.0f + expf(-g.logit));
    const float dlogit = dop * opacity * (1.f - opacity);

    // Sigma = Ms Ms^T, Ms = R diag(s): dMs = 2 dSigma Ms
    const float* R = g.R;
    float dls[3], dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // column k of Ms is s_k R[:, k]
        const float c0 = R[0 + k] * g.s[k], c1 = R[3 + k] * g.s[k], c2 = R[6 + k] * g.s[k];
        const float m0 = 2.f * (dSig[0] * c0 + dSig[1] * c1 + dSig[2] * c2);
        const float m1 = 2.f * (dSig[1] * c0 + dSig[3] * c1 + dSig[4] * c2);
        const float m2 = 2.f * (dSig[2] * c0 + dSig[4] * c1 + dSig[5] * c2);
        dls[k] = (m0 * R[0 + k] + m1 * R[3 + k] + m2 * R[6 + k]) * g.s[k];
        dR[0 + k] = m0 * g.s[k];
        dR[3 + k] = m1 * g.s[k];
        dR[6 + k] = m2 * g.s[k];
    }
    const float w = g.qw, x = g.qx, y = g.qy, z = g.qz;
    float dq[4];
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                   x * dR[6] + y * dR[7]);
    const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    const float iq = 1.0f / g.qn;

    const float4 g0 = make_float4(dmean[0], dmean[1], dmean[2], dlogit);
    const float4 g1 = make_float4((dq[0] - w * qd) * iq, (dq[1] - x * qd) * iq, (dq[2] - y * qd) * iq,
                                  (dq[3] - z * qd) * iq);
    const float4 g2 = make_float4(dls[0], dls[1], dls[2], 0.f);
    gq[0] = make_float4(dmean[0], dmean[1], dmean[2], dlogit);
    gq[1] = make_float4((dq[0] - w * qd) * iq, (dq[1] - x * qd) * iq, (dq[2] - y * qd) * iq, (dq[3] - z * qd) * iq);
    gq[2] = make_float4(dls[0], dls[1], dls[2], 0.f);
    return true;
}

// This thread's SH gradient plane q (3 K accumulators, zero past them).
template <int DEG>
__device__ __forceinline__ float4 sh_grad_plane(float* s_dsh, int q) {
    constexpr int K3 = 3 * SH<DEG>::K;
    float4 r;
    r.x = (4 * q + 0 < K3) ? dsh_acc(s_dsh, 4 * q + 0) : 0.f;
    r.y = (4 * q + 1 < K3) ? dsh_acc(s_dsh, 4 * q + 1) : 0.f;
    r.z = (4 * q + 2 < K3) ? dsh_acc(s_dsh, 4 * q + 2) : 0.f;
    r.w = (4 * q + 3 < K3) ? dsh_acc(s_dsh, 4 * q + 3) : 0.f;
    return r;
}

template <int DEG, int FT>
__global__ void __launch_bounds__(kProjBwdThreads, 2) project_bwd_kernel(
    const float4* __restrict__ P, const uint2* __restrict__ F, int n, const gsfit_camera* __restrict__ cams_g,
    int n_views, const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgbm,
    float4* __restrict__ grad2d, float4* __restrict__ G, int32_t* __restrict__ status) {
    // dynamic shared memory: the camera table, then 3K SH-gradient accumulators
    // per thread (kept out of registers)
    extern __shared__ __align__(16) unsigned char smem_pb[];
    gsfit_camera* cams = reinterpret_cast<gsfit_camera*>(smem_pb);
    float* s_dsh = reinterpret_cast<float*>(smem_pb + sizeof(gsfit_camera) * n_views);
    constexpr int K = SH<DEG>::K;
    load_cameras(cams, cams_g, n_views);
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) dsh_acc(s_dsh, k) = 0.f;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Gauss g;
    load_gauss<FT>(P, F, n, i, g);

    float dmean[3] = {0.f, 0.f, 0.f};
    float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx xy xz yy yz zz (symmetric, dL/dSigma_ij)
    float dop = 0.f;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    bool binned = false;  // some view binned this Gaussian

    for (int v0 = 0; v0 < n_views; v0 += 32) {
        // visibility of up to 32 views first: independent loads, one latency
        uint32_t vis = 0;
        const int vn = min(32, n_views - v0);
#pragma unroll 8
        for (int k = 0; k < vn; ++k)
            if (__ldg(&xyd[(size_t)(v0 + k) * n + i].w) != 0.0f) vis |= 1u << k;
        if (!vis) continue;
        binned = true;
        int v = v0 + __ffs(vis) - 1;
        vis &= vis - 1;
        RecIn cur = load_rec(grad2d, conic, rgbm, (size_t)v * n + i);
        for (;;) {
            // the next binned view's loads go out before this view's chain
            const int vnext = vis ? v0 + __ffs(vis) - 1 : -1;
            vis &= vis - 1;
            RecIn nxt;
            if (vnext >= 0) nxt = load_rec(grad2d, conic, rgbm, (size_t)vnext * n + i);
            const size_t r = (size_t)v * n + i;
            grad2d[4 * r + 0] = zero;  // the adjoint's atomics fill these three
            grad2d[4 * r + 1] = zero;
            grad2d[4 * r + 2] = zero;
            const gsfit_camera& cam = cams[v];
            float dm[3], dS[6], gcol[3];
            record_bwd<DEG, FT>(cam, g, cur.ga, cur.gb, cur.gc, cur.cq, cur.cm, P, F, n, i, dm, dS, gcol);
            dmean[0] += dm[0]; dmean[1] += dm[1]; dmean[2] += dm[2];
            dop += cur.ga.z;
#pragma unroll
            for (int k = 0; k < 6; ++k) dSig[k] += dS[k];
            float dx = g.mx - cam.campos[0], dy = g.my - cam.campos[1], dz = g.mz - cam.campos[2];
            const float idist = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= idist; dy *= idist; dz *= idist;
            float Y[K];
            sh_basis<DEG>(dx, dy, dz, Y);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dsh_acc(s_dsh, 3 * k + 0) += Y[k] * gcol[0];
                dsh_acc(s_dsh, 3 * k + 1) += Y[k] * gcol[1];
                dsh_acc(s_dsh, 3 * k + 2) += Y[k] * gcol[2];
            }
            if (vnext < 0) break;
            v = vnext;
            cur = nxt;
        }
    }
    if (!binned) {
        // a Gaussian no view binned contributes to no pixel: its gradient is
        // zero (written as such, also where its parameters are not finite and
        // the chain below would give 0 x NaN)
        constexpr int NPL = 3 + (3 * K + 3) / 4;
#pragma unroll
        for (int p = 0; p < NPL; ++p) G[(size_t)p * n + i] = zero;
        return;
    }
    const float opacity = 1.0f / (1.0f + expf(-g.logit));
    const float dlogit = dop * opacity * (1.f - opacity);

    // Sigma = Ms Ms^T, Ms = R diag(s): dMs = 2 dSigma Ms
    const float* R = g.R;
    float dls[3], dR[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // column k of Ms is s_k R[:, k]
        const float c0 = R[0 + k] * g.s[k], c1 = R[3 + k] * g.s[k], c2 = R[6 + k] * g.s[k];
        const float m0 = 2.f * (dSig[0] * c0 + dSig[1] * c1 + dSig[2] * c2);
        const float m1 = 2.f * (dSig[1] * c0 + dSig[3] * c1 + dSig[4] * c2);
        const float m2 = 2.f * (dSig[2] * c0 + dSig[4] * c1 + dSig[5] * c2);
        dls[k] = (m0 * R[0 + k] + m1 * R[3 + k] + m2 * R[6 + k]) * g.s[k];
        dR[0 + k] = m0 * g.s[k];
        dR[3 + k] = m1 * g.s[k];
        dR[6 + k] = m2 * g.s[k];
    }
    const float w = g.qw, x = g.qx, y = g.qy, z = g.qz;
    float dq[4];
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                   x * dR[6] + y * dR[7]);
    const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    const float iq = 1.0f / g.qn;

    const float4 g0 = make_float4(dmean[0], dmean[1], dmean[2], dlogit);
    const float4 g1 = make_float4((dq[0] - w * qd) * iq, (dq[1] - x * qd) * iq, (dq[2] - y * qd) * iq,
                                  (dq[3] - z * qd) * iq);
    const float4 g2 = make_float4(dls[0], dls[1], dls[2], 0.f);
    G[i] = g0;
    G[(size_t)n + i] = g1;
    G[2 * (size_t)n + i] = g2;
    bool finite = finite4(g0) && finite4(g1) && finite4(g2);
    constexpr int K3 = 3 * K;
    constexpr int NP = (K3 + 3) / 4;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float4 q;
        q.x = (4 * p + 0 < K3) ? dsh_acc(s_dsh, 4 * p + 0) : 0.f;
        q.y = (4 * p + 1 < K3) ? dsh_acc(s_dsh, 4 * p + 1) : 0.f;
        q.z = (4 * p + 2 < K3) ? dsh_acc(s_dsh, 4 * p + 2) : 0.f;
        q.w = (4 * p + 3 < K3) ? dsh_acc(s_dsh, 4 * p + 3) : 0.f;
        G[(size_t)(3 + p) * n + i] = q;
        finite = finite && finite4(q);
    }
    // a non-finite gradient (from a non-finite image, cotangent or 2D
    // gradient upstream) is reported, not hidden: the first such Gaussian sets
    // the status word unless an earlier error already has
    if (!finite && status) atomicCAS(status, GSFIT_OK, GSFIT_ERR_NONFINITE);
}

// Adam over the C planes p0 .. p0 + C - 1 of Gaussian i: every load of the
// chunk first, then the updates and stores (G, when given, receives the
// gradient; F the 16-bit copy of the SH planes).
template <int C, int FT, int NG>
__device__ __forceinline__ void adam_chunk(float4* P, uint2* F, float4* __restrict__ m, float4* __restrict__ v,
                                           float4* __restrict__ G, int n, int i, int p0, const float4 (&g)[NG],
                                           const float4* s_lr, const AdamCoef& c) {
    static_assert(C <= NG, "chunk larger than its gradients");
    float4 pp[C], mm[C], vv[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const size_t k = (size_t)(p0 + j) * n + i;
        pp[j] = P[k];
        mm[j] = m[k];
        vv[j] = v[k];
    }
#pragma unroll
    for (int j = 0; j < C; ++j) {
        const size_t k = (size_t)(p0 + j) * n + i;
        if (G) G[k] = g[j];
        adam_update(pp[j], mm[j], vv[j], g[j], s_lr[p0 + j], c);
        P[k] = pp[j];
        m[k] = mm[j];
        v[k] = vv[j];
        if constexpr (FT != GSFIT_FEATURES_F32) {
            if (p0 + j >= kFeaturePlane0) F[(size_t)(p0 + j - kFeaturePlane0) * n + i] = pack_features<FT>(pp[j]);
        }
    }
}

// project_bwd_kernel and the Adam update in one pass: each thread takes its
// Gaussian's gradient from gaussian_grad straight into adam_update (the same
// arithmetic as adam_kernel) plane by plane, so the gradient never goes
// through memory unless G is given. P and F (the 16-bit copy of the SH
// planes) are read by the chain and then rewritten by the same thread only.
template <int DEG, int FT>
__global__ void __launch_bounds__(kProjBwdThreads, 2) project_bwd_adam_kernel(
    float4* P, uint2* F, int n, const gsfit_camera* __restrict__ cams_g, int n_views,
    const float4* __restrict__ xyd, const float4* __restrict__ conic, const float4* __restrict__ rgbm,
    float4* __restrict__ grad2d, float4* __restrict__ G, float4* __restrict__ m, float4* __restrict__ v,
    LrTable lrt, float b1, float b2, float eps, const int32_t* __restrict__ step, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_pb[];
    __shared__ float4 s_lr[kMaxPlanes];
    gsfit_camera* cams = reinterpret_cast<gsfit_camera*>(smem_pb);
    float* s_dsh = reinterpret_cast<float*>(smem_pb + sizeof(gsfit_camera) * n_views);
    constexpr int K = SH<DEG>::K;
    constexpr int NP = (3 * K + 3) / 4;
    load_cameras(cams, cams_g, n_views);
    if (threadIdx.x < kMaxPlanes) s_lr[threadIdx.x] = lrt.lr[threadIdx.x];
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) dsh_acc(s_dsh, k) = 0.f;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 gq[3];
    const bool binned = gaussian_grad<DEG, FT>(P, F, n, i, cams, n_views, xyd, conic, rgbm, grad2d, s_dsh, gq);
    const AdamCoef c = adam_coef(b1, b2, eps, *step);
    bool finite = finite4(gq[0]) && finite4(gq[1]) && finite4(gq[2]);
    // planes 0-2, then the SH planes three at a time: each chunk loads all its
    // parameters and moments before its first store, so a thread has a
    // chunk's loads in flight at once (a later plane's loads cannot move above
    // an earlier plane's stores to P, which the compiler cannot tell apart)
    adam_chunk<3, FT>(P, F, m, v, G, n, i, 0, gq, s_lr, c);
#pragma unroll
    for (int q0 = 0; q0 < NP; q0 += 3) {
        float4 gg[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gg[j] = q0 + j < NP ? sh_grad_plane<DEG>(s_dsh, q0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            finite = finite && finite4(gg[j]);
        }
        if (NP - q0 >= 3) adam_chunk<3, FT>(P, F, m, v, G, n, i, 3 + q0, gg, s_lr, c);
        else if (NP - q0 == 2) adam_chunk<2, FT>(P, F, m, v, G, n, i, 3 + q0, gg, s_lr, c);
        else adam_chunk<1, FT>(P, F, m, v, G, n, i, 3 + q0, gg, s_lr, c);
    }
    if (binned && !finite && status) atomicCAS(status, GSFIT_OK, GSFIT_ERR_NONFINITE);
}

template <int DEG, int FT>
int launch_project(const gsfit_gaussians* g, const gsfit_camera* cams, int V, gsfit_proj* out, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (g->n + threads - 1) / threads;
    const size_t smem = sizeof(gsfit_camera) * V;
    project_kernel<DEG, FT><<<blocks, threads, smem, s>>>(
        reinterpret_cast<const float4*>(g->params), reinterpret_cast<const uint2*>(g->features), g->n, cams, V,
        reinterpret_cast<float4*>(out->xyd), reinterpret_cast<float4*>(out->conic),
        reinterpret_cast<float4*>(out->rgb), out->tiles);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

template <int DEG, int FT>
int launch_project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V,
                       float* grad2d, float* grads, int32_t* status, cudaStream_t s) {
    const int threads = kProjBwdThreads;
    const int blocks = (g->n + threads - 1) / threads;
    const float4* P = reinterpret_cast<const float4*>(g->params);
    const uint2* F = reinterpret_cast<const uint2*>(g->features);
    const size_t smem = sizeof(gsfit_camera) * V + sizeof(float) * 3 * SH<DEG>::K * threads;
    static ContextOnce once;
    const size_t max_smem = sizeof(gsfit_camera) * GSFIT_MAX_VIEWS + sizeof(float) * 3 * SH<DEG>::K * threads;
    const int rc = opt_in_smem(once, project_bwd_kernel<DEG, FT>, max_smem);
    if (rc != GSFIT_OK) return rc;
    project_bwd_kernel<DEG, FT><<<blocks, threads, smem, s>>>(
        P, F, g->n, cams, V, reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), reinterpret_cast<float4*>(grad2d),
        reinterpret_cast<float4*>(grads), status);
    GSFIT_LAUNCH_CHECK();
    return GSFIT_OK;
}

// Dispatch over the feature storage type.
template <int DEG>
int project_ft(const gsfit_gaussians* g, const gsfit_camera* cams, int V, gsfit_proj* out, cudaStream_t s) {
    switch (g->feature_dtype) {
        case GSFIT_FEATURES_F16: return launch_project<DEG, GSFIT_FEATURES_F16>(g, cams, V, out, s);
        case GSFIT_FEATURES_BF16: return launch_project<DEG, GSFIT_FEATURES_BF16>(g, cams, V, out, s);
        default: return launch_project<DEG, GSFIT_FEATURES_F32>(g, cams, V, out, s);
    }
}

template <int DEG>
int project_bwd_ft(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V, float* grad2d,
                   float* grads, int32_t* status, cudaStream_t s) {
    switch (g->feature_dtype) {
        case GSFIT_FEATURES_F16:
            return launch_project_bwd<DEG, GSFIT_FEATURES_F16>(g, proj, cams, V, grad2d, grads, status, s);
        case GSFIT_FEATURES_BF16:
            return launch_project_bwd<DEG, GSFIT_FEATURES_BF16>(g, proj, cams, V, grad2d, grads, status, s);
        default: return launch_project_bwd<DEG, GSFIT_FEATURES_F32>(g, proj, cams, V, grad2d, grads, status, s);
    }
}

// The Adam arguments of the fused adjoint, as gsfit_adam_step takes them.
struct AdamArgs {
    float* m;
    float* v;
    LrTable lrt;
    float b1, b2, eps;
    int32_t* step;
};

template <int DEG, int FT>
int launch_project_bwd_adam(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V,
                            float* grad2d, float* grads, const AdamArgs& a, int32_t* status, cudaStream_t s) {
    const int threads = kProjBwdThreads;
    const int blocks = (g->n + threads - 1) / threads;
    // the parameters and their 16-bit copy are updated in place
    float4* P = reinterpret_cast<float4*>(const_cast<float*>(g->params));
    uint2* F = reinterpret_cast<uint2*>(const_cast<void*>(g->features));
    const size_t smem = sizeof(gsfit_camera) * V + sizeof(float) * 3 * SH<DEG>::K * threads;
    static ContextOnce once;
    const size_t max_smem = sizeof(gsfit_camera) * GSFIT_MAX_VIEWS + sizeof(float) * 3 * SH<DEG>::K * threads;
    const int rc = opt_in_smem(once, project_bwd_adam_kernel<DEG, FT>, max_smem);
    if (rc != GSFIT_OK) return rc;
    project_bwd_adam_kernel<DEG, FT><<<blocks, threads, smem, s>>>(
        P, F, g->n, cams, V, reinterpret_cast<const float4*>(proj->xyd), reinterpret_cast<const float4*>(proj->conic),
        reinterpret_cast<const float4*>(proj->rgb), reinterpret_cast<float4*>(grad2d),
        reinterpret_cast<float4*>(grads), reinterpret_cast<float4*>(a.m), reinterpret_cast<float4*>(a.v), a.lrt,
        a.b1, a.b2, a.eps, a.step, status);
    GSFIT_LAUNCH_CHECK();
    return step_increment(a.step, s);
}

template <int DEG>
int project_bwd_adam_ft(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V,
                        float* grad2d, float* grads, const AdamArgs& a, int32_t* status, cudaStream_t s) {
    switch (g->feature_dtype) {
        case GSFIT_FEATURES_F16:
            return launch_project_bwd_adam<DEG, GSFIT_FEATURES_F16>(g, proj, cams, V, grad2d, grads, a, status, s);
        case GSFIT_FEATURES_BF16:
            return launch_project_bwd_adam<DEG, GSFIT_FEATURES_BF16>(g, proj, cams, V, grad2d, grads, a, status, s);
        default:
            return launch_project_bwd_adam<DEG, GSFIT_FEATURES_F32>(g, proj, cams, V, grad2d, grads, a, status, s);
    }
}

}  // namespace

bool valid_gaussians(const gsfit_gaussians* g) {
    if (!(g && g->params && g->n > 0 && g->sh_degree >= 0 && g->sh_degree <= 3 &&
          (reinterpret_cast<uintptr_t>(g->params) % 16) == 0))
        return false;
    if (g->feature_dtype == GSFIT_FEATURES_F32) return true;
    return (g->feature_dtype == GSFIT_FEATURES_F16 || g->feature_dtype == GSFIT_FEATURES_BF16) && g->features &&
           (reinterpret_cast<uintptr_t>(g->features) % 8) == 0;
}

bool valid_proj(const gsfit_proj* p) {
    return p && p->xyd && p->conic && p->rgb && p->tiles && (reinterpret_cast<uintptr_t>(p->xyd) % 16) == 0 &&
           (reinterpret_cast<uintptr_t>(p->conic) % 16) == 0 && (reinterpret_cast<uintptr_t>(p->rgb) % 16) == 0;
}

int project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int V, float* grad2d,
                float* grads, int32_t* status, cudaStream_t s) {
    switch (g->sh_degree) {
        case 0: return project_bwd_ft<0>(g, proj, cams, V, grad2d, grads, status, s);
        case 1: return project_bwd_ft<1>(g, proj, cams, V, grad2d, grads, status, s);
        case 2: return project_bwd_ft<2>(g, proj, cams, V, grad2d, grads, status, s);
        default: return project_bwd_ft<3>(g, proj, cams, V, grad2d, grads, status, s);
    }
}

}  // namespace gsfit

extern "C" int gsfit_num_planes(int sh_degree) {
    if (sh_degree < 0 || sh_degree > 3) return GSFIT_ERR_INVALID_ARG;
    return gsfit::num_planes(sh_degree);
}

extern "C" int gsfit_project(const gsfit_gaussians* g, const gsfit_camera* cams, int32_t n_views, gsfit_proj* out,
                             cudaStream_t stream) {
    if (!gsfit::valid_gaussians(g) || !cams || !gsfit::valid_proj(out) || n_views < 1 ||
        n_views > GSFIT_MAX_VIEWS)
        return GSFIT_ERR_INVALID_ARG;
    switch (g->sh_degree) {
        case 0: return gsfit::project_ft<0>(g, cams, n_views, out, stream);
        case 1: return gsfit::project_ft<1>(g, cams, n_views, out, stream);
        case 2: return gsfit::project_ft<2>(g, cams, n_views, out, stream);
        default: return gsfit::project_ft<3>(g, cams, n_views, out, stream);
    }
}

extern "C" int gsfit_project_bwd_adam(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                                      int32_t n_views, float* grad2d, float* grads, float* m, float* v,
                                      const float* lr, float beta1, float beta2, float eps, int32_t* step,
                                      int32_t* status, cudaStream_t stream) {
    if (!gsfit::valid_gaussians(g) || !gsfit::valid_proj(proj) || !cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || !grad2d ||
        !m || !v || !lr || !step)
        return GSFIT_ERR_INVALID_ARG;
    for (const float* q : {(const float*)grad2d, (const float*)grads, (const float*)m, (const float*)v})
        if ((reinterpret_cast<uintptr_t>(q) % 16) != 0) return GSFIT_ERR_INVALID_ARG;
    const int n_planes = gsfit_num_planes(g->sh_degree);
    gsfit::AdamArgs a;
    a.m = m;
    a.v = v;
    for (int k = 0; k < gsfit::kMaxPlanes; ++k)
        a.lrt.lr[k] = k < n_planes ? make_float4(lr[4 * k], lr[4 * k + 1], lr[4 * k + 2], lr[4 * k + 3])
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    a.b1 = beta1;
    a.b2 = beta2;
    a.eps = eps;
    a.step = step;
    switch (g->sh_degree) {
        case 0: return gsfit::project_bwd_adam_ft<0>(g, proj, cams, n_views, grad2d, grads, a, status, stream);
        case 1: return gsfit::project_bwd_adam_ft<1>(g, proj, cams, n_views, grad2d, grads, a, status, stream);
        case 2: return gsfit::project_bwd_adam_ft<2>(g, proj, cams, n_views, grad2d, grads, a, status, stream);
        default: return gsfit::project_bwd_adam_ft<3>(g, proj, cams, n_views, grad2d, grads, a, status, stream);
    }
}
