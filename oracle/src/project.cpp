// Projection of one 3D Gaussian into one view, and its adjoint.
//
// Section 4.2 (the peripheral model is a 3DGS model); the splat model is the
// EWA splatting of 3DGS, which the paper inherits without writing it out:
//   activations  s = exp(log_scale), q normalised, o = sigmoid(logit)
//   covariance   Sigma = R(q) diag(s^2) R(q)^T
//   camera       t = R_view mu + t_view, +z forward, culled if t_z <= near
//   EWA          Sigma' = J R_view Sigma R_view^T J^T + 0.3 I, with the 3DGS
//                frustum guard on t_x/t_z, t_y/t_z (+-1.3 tan(fov/2))
//   conic        inverse of Sigma'; radius = ceil(3 sqrt(lambda_max))
//   centre       u = fx t_x / t_z + cx, v = fy t_y / t_z + cy
//   colour       SH(dir) . k + 0.5 clamped at 0, dir = normalise(mu - campos)
#include <cmath>
#include <cstring>

#include "oracle.h"

namespace oracle {

std::vector<Camera> unpack_cameras(int V, const double* c, int tile) {
    std::vector<Camera> cams(V);
    int toff = 0;
    long long poff = 0;
    for (int v = 0; v < V; ++v) {
        const double* r = c + (size_t)v * CAM_DOUBLES;
        Camera& k = cams[v];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                k.R[i][j] = r[4 * i + j];
                k.Rf[i][j] = (float)r[4 * i + j];
            }
            k.t[i] = r[4 * i + 3];
            k.tf[i] = (float)r[4 * i + 3];
            k.campos[i] = r[12 + i];
        }
        k.fx = r[15]; k.fy = r[16]; k.cx = r[17]; k.cy = r[18]; k.near_plane = r[19];
        k.fxf = (float)k.fx; k.fyf = (float)k.fy; k.cxf = (float)k.cx; k.cyf = (float)k.cy;
        k.nearf = (float)k.near_plane;
        k.W = (int)r[20];
        k.H = (int)r[21];
        k.tiles_x = (k.W + tile - 1) / tile;
        k.tiles_y = (k.H + tile - 1) / tile;
        k.tile_offset = toff;
        k.pixel_offset = poff;
        toff += k.tiles_x * k.tiles_y;
        poff += (long long)k.W * k.H;
    }
    return cams;
}

int total_tiles(const std::vector<Camera>& cams) {
    int t = 0;
    for (const Camera& c : cams) t += c.tiles_x * c.tiles_y;
    return t;
}

namespace {

// Camera-space coordinate row k in float32, in the fixed order
// ((R_k0 x + R_k1 y) + R_k2 z) + t_k, every operation rounded to float32.
// This value decides the depth key, the depth cull and the tile rectangle.
float cam_coord_f32(const Camera& c, int k, const float m[3]) {
    float a = c.Rf[k][0] * m[0];
    float b = c.Rf[k][1] * m[1];
    float s = a + b;
    float d = c.Rf[k][2] * m[2];
    s = s + d;
    return s + c.tf[k];
}

void quat_to_rot(const double qn[4], double R[3][3]) {
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

// Everything the forward pass computes for one (view, Gaussian), kept so the
// adjoint can reuse it.
struct Fwd {
    bool in_front;
    float depth32, u32, v32;
    double mean[3], s[3], qnorm, qn[4], Rq[3][3], Sigma[3][3];
    double t[3], rho[2];
    bool guard_clamped[2];
    double J[2][3], M[2][3];
    double a, b, c, det, conic[3];
    double u, v;
    double opacity;
    int K, deg;
    double dir[3], dist, Y[16], rgb_raw[3];
};

void forward(const double* g, int K, const Camera& cam, Fwd& f) {
    f.K = K;
    f.deg = (int)std::lround(std::sqrt((double)K)) - 1;
    for (int i = 0; i < 3; ++i) f.mean[i] = g[i];
    const float mf[3] = {(float)g[0], (float)g[1], (float)g[2]};
    f.depth32 = cam_coord_f32(cam, 2, mf);
    f.in_front = f.depth32 > cam.nearf;
    const float tx32 = cam_coord_f32(cam, 0, mf);
    const float ty32 = cam_coord_f32(cam, 1, mf);
    // Centre in float32: (fx * t_x) / t_z + cx, correctly rounded each step.
    f.u32 = (cam.fxf * tx32) / f.depth32 + cam.cxf;
    f.v32 = (cam.fyf * ty32) / f.depth32 + cam.cyf;

    for (int i = 0; i < 3; ++i) f.s[i] = std::exp(g[3 + i]);
    f.qnorm = std::sqrt(g[6] * g[6] + g[7] * g[7] + g[8] * g[8] + g[9] * g[9]);
    for (int i = 0; i < 4; ++i) f.qn[i] = g[6 + i] / f.qnorm;
    quat_to_rot(f.qn, f.Rq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += f.Rq[i][k] * f.s[k] * f.s[k] * f.Rq[j][k];
            f.Sigma[i][j] = acc;
        }

    for (int i = 0; i < 3; ++i) {
        double acc = cam.t[i];
        for (int j = 0; j < 3; ++j) acc += cam.R[i][j] * f.mean[j];
        f.t[i] = acc;
    }
    const double tz = f.t[2];
    const double lim[2] = {FRUSTUM_GUARD * 0.5 * cam.W / cam.fx, FRUSTUM_GUARD * 0.5 * cam.H / cam.fy};
    for (int k = 0; k < 2; ++k) {
        const double r = f.t[k] / tz;
        f.guard_clamped[k] = (r < -lim[k]) || (r > lim[k]);
        f.rho[k] = r < -lim[k] ? -lim[k] : (r > lim[k] ? lim[k] : r);
    }
    f.J[0][0] = cam.fx / tz; f.J[0][1] = 0.0;          f.J[0][2] = -cam.fx * f.rho[0] / tz;
    f.J[1][0] = 0.0;         f.J[1][1] = cam.fy / tz;  f.J[1][2] = -cam.fy * f.rho[1] / tz;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += f.J[i][k] * cam.R[k][j];
            f.M[i][j] = acc;
        }
    double S2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += f.M[i][k] * f.Sigma[k][l] * f.M[j][l];
            S2[i][j] = acc;
        }
    f.a = S2[0][0] + COV_DILATION;
    f.b = S2[0][1];
    f.c = S2[1][1] + COV_DILATION;
    f.det = f.a * f.c - f.b * f.b;
    f.conic[0] = f.c / f.det;
    f.conic[1] = -f.b / f.det;
    f.conic[2] = f.a / f.det;
    f.u = cam.fx * f.t[0] / tz + cam.cx;
    f.v = cam.fy * f.t[1] / tz + cam.cy;
    f.opacity = 1.0 / (1.0 + std::exp(-g[10]));

    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = f.mean[i] - cam.campos[i];
    f.dist = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) f.dir[i] = d[i] / f.dist;
    real_sh(f.deg, f.dir, f.Y, nullptr);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += f.Y[k] * g[11 + 3 * k + ch];
        f.rgb_raw[ch] = acc + 0.5;
    }
}

}  // namespace

void project_one(const double* g, int K, const Camera& cam, int tile, int flags, double* out) {
    std::memset(out, 0, sizeof(double) * P_STRIDE);
    Fwd f;
    forward(g, K, cam, f);
    out[P_DEPTH32] = f.depth32;
    out[P_U32] = f.u32;
    out[P_V32] = f.v32;
    if (!f.in_front || !(f.det > 0.0)) return;
    const double mid = 0.5 * (f.a + f.c);
    const double lambda = mid + std::sqrt(std::fmax(0.1, mid * mid - f.det));
    const double x = 3.0 * std::sqrt(lambda);
    const int radius = (int)std::ceil(x);
    const double frac_lo = x - std::floor(x), frac_hi = std::ceil(x) - x;
    out[P_NEAR_BOUNDARY] = (std::fmin(frac_lo, frac_hi) < 1e-5 * x) ? 1.0 : 0.0;

    // Tile rectangle [x0, x1) x [y0, y1) from the float32 centre, in float32:
    // x0 = floor((u - r) / B), x1 = floor(((u + r) + (B - 1)) / B), clamped.
    const float rf = (float)radius, Bf = (float)tile, Bm1 = (float)(tile - 1);
    auto clampi = [](int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); };
    const int x0 = clampi((int)std::floor((f.u32 - rf) / Bf), 0, cam.tiles_x);
    const int x1 = clampi((int)std::floor(((f.u32 + rf) + Bm1) / Bf), 0, cam.tiles_x);
    const int y0 = clampi((int)std::floor((f.v32 - rf) / Bf), 0, cam.tiles_y);
    const int y1 = clampi((int)std::floor(((f.v32 + rf) + Bm1) / Bf), 0, cam.tiles_y);
    const int tiles = (x1 - x0) * (y1 - y0);

    out[P_U] = f.u;
    out[P_V] = f.v;
    out[P_RADIUS] = radius;
    for (int k = 0; k < 3; ++k) out[P_CONIC_A + k] = f.conic[k];
    out[P_COV_A] = f.a;
    out[P_COV_B] = f.b;
    out[P_COV_C] = f.c;
    out[P_OPACITY] = f.opacity;
    for (int ch = 0; ch < 3; ++ch) {
        const bool clamped = f.rgb_raw[ch] < 0.0;
        out[P_R + ch] = clamped ? 0.0 : f.rgb_raw[ch];
        out[P_CLAMP_R + ch] = clamped ? 1.0 : 0.0;
    }
    out[P_RECT_X0] = x0; out[P_RECT_Y0] = y0; out[P_RECT_X1] = x1; out[P_RECT_Y1] = y1;
    out[P_TILES] = tiles;
    out[P_VISIBLE] = (flags & FLAG_SMOOTH) ? 1.0 : (tiles > 0 ? 1.0 : 0.0);
}

// Adjoint of project_one. g2 holds dL/d(u, v, conic a', b', c', opacity,
// r, g, b) for this (view, Gaussian); gout accumulates dL/d(parameters) in the
// Gaussian record layout. Every derivative is that of the function above,
// including the zero derivative of an active frustum guard or colour clamp.
void project_bwd_one(const double* g, int K, const Camera& cam, const double g2[9], double* gout) {
    Fwd f;
    forward(g, K, cam, f);
    const double tz = f.t[2];
    double dt[3] = {0.0, 0.0, 0.0};
    double dmean[3] = {0.0, 0.0, 0.0};

    // centre: u = fx t_x / t_z + cx, v = fy t_y / t_z + cy
    dt[0] += g2[0] * cam.fx / tz;
    dt[1] += g2[1] * cam.fy / tz;
    dt[2] += -g2[0] * cam.fx * f.t[0] / (tz * tz) - g2[1] * cam.fy * f.t[1] / (tz * tz);

    // conic = inverse(S), S = [[a, b], [b, c]]; dL/dS = -Q G Q, with G the
    // symmetric matrix of dL/dQ (the off-diagonal conic entry b' counts twice).
    const double Q[2][2] = {{f.conic[0], f.conic[1]}, {f.conic[1], f.conic[2]}};
    const double G[2][2] = {{g2[2], 0.5 * g2[3]}, {0.5 * g2[3], g2[4]}};
    double QG[2][2], dS[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) QG[i][j] = Q[i][0] * G[0][j] + Q[i][1] * G[1][j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) dS[i][j] = -(QG[i][0] * Q[0][j] + QG[i][1] * Q[1][j]);

    // S = M Sigma M^T + 0.3 I: dL/dSigma = M^T dS M, dL/dM = 2 dS M Sigma.
    double dSigma[3][3], dM[2][3];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            double acc = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) acc += f.M[i][k] * dS[i][j] * f.M[j][l];
            dSigma[k][l] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 3; ++l) acc += dS[i][j] * f.M[j][l] * f.Sigma[l][k];
            dM[i][k] = 2.0 * acc;
        }
    // M = J R_view: dL/dJ = dM R_view^T
    double dJ[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += dM[i][j] * cam.R[k][j];
            dJ[i][k] = acc;
        }
    // J00 = fx/tz, J11 = fy/tz, J02 = -fx rho_x / tz, J12 = -fy rho_y / tz,
    // rho = t_xy / t_z unless the frustum guard clamps it.
    const double fxy[2] = {cam.fx, cam.fy};
    for (int k = 0; k < 2; ++k) {
        const double dJdiag = dJ[k][k];
        const double dJ2 = dJ[k][2];
        dt[2] += dJdiag * (-fxy[k] / (tz * tz)) + dJ2 * (fxy[k] * f.rho[k] / (tz * tz));
        const double drho = dJ2 * (-fxy[k] / tz);
        if (!f.guard_clamped[k]) {
            dt[k] += drho / tz;
            dt[2] += drho * (-f.t[k] / (tz * tz));
        }
    }
    // t = R_view mu + t_view
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) dmean[j] += cam.R[i][j] * dt[i];

    // Sigma = Ms Ms^T with Ms = R(q) diag(s)
    double dMs[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += dSigma[i][j] * f.Rq[j][k] * f.s[k];
            dMs[i][k] = 2.0 * acc;
        }
    double dR[3][3];
    for (int k = 0; k < 3; ++k) {
        double ds = 0.0;
        for (int i = 0; i < 3; ++i) {
            ds += dMs[i][k] * f.Rq[i][k];
            dR[i][k] = dMs[i][k] * f.s[k];
        }
        gout[3 + k] += ds * f.s[k];  // d/dlog_scale
    }
    // R(q^) for the unit quaternion (w, x, y, z)
    const double w = f.qn[0], x = f.qn[1], y = f.qn[2], z = f.qn[3];
    double dq[4];
    dq[0] = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    dq[1] = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                 w * dR[2][1] - 2 * x * dR[2][2]);
    dq[2] = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                 z * dR[2][1] - 2 * y * dR[2][2]);
    dq[3] = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] + y * dR[1][2] +
                 x * dR[2][0] + y * dR[2][1]);
    // q^ = q / |q|
    const double qdot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    for (int i = 0; i < 4; ++i) gout[6 + i] += (dq[i] - f.qn[i] * qdot) / f.qnorm;

    // opacity = sigmoid(logit)
    gout[10] += g2[5] * f.opacity * (1.0 - f.opacity);

    // colour = max(0, SH(dir) . k + 0.5)
    double Y[16], dY[48];
    real_sh(f.deg, f.dir, Y, dY);
    double gc[3];
    for (int ch = 0; ch < 3; ++ch) gc[ch] = f.rgb_raw[ch] < 0.0 ? 0.0 : g2[6 + ch];
    double ddir[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < K; ++k) {
        double wk = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            gout[11 + 3 * k + ch] += Y[k] * gc[ch];
            wk += g[11 + 3 * k + ch] * gc[ch];
        }
        for (int i = 0; i < 3; ++i) ddir[i] += dY[3 * k + i] * wk;
    }
    // dir = d / |d|, d = mu - campos
    const double dd = f.dir[0] * ddir[0] + f.dir[1] * ddir[1] + f.dir[2] * ddir[2];
    for (int i = 0; i < 3; ++i) dmean[i] += (ddir[i] - f.dir[i] * dd) / f.dist;

    for (int i = 0; i < 3; ++i) gout[i] += dmean[i];
}

}  // namespace oracle
