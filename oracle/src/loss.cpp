// Photometric loss and its gradient with respect to the rendered image.
//
// Section 4.2 trains with alpha supervision against renders composited over
// randomised backgrounds; the loss itself is not stated, so the 3DGS loss is
// used on colour, plus an L1 term on alpha:
//   L_v = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)) + mean|A - A*|
//   L   = (1/V) sum_v L_v,  lambda = 0.2
// where y = target_rgb + (1 - target_alpha) bg is the (premultiplied) target
// composited over the same background as the render. SSIM uses an 11x11
// Gaussian window (sigma 1.5, normalised), zero padding at the image border,
// C1 = 0.01^2, C2 = 0.03^2, averaged over channels and pixels. The L1
// subgradient at zero is 0.
#include <cmath>
#include <vector>

#include "oracle.h"

namespace oracle {

namespace {

constexpr int WIN = 11, HALF = 5;
constexpr double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;

void window(double w[WIN][WIN]) {
    double g[WIN], s = 0.0;
    for (int i = 0; i < WIN; ++i) {
        g[i] = std::exp(-double((i - HALF) * (i - HALF)) / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < WIN; ++i)
        for (int j = 0; j < WIN; ++j) w[i][j] = g[i] * g[j] / (s * s);
}

inline double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

}  // namespace

// rgb / target_rgb: per view 3 planes of H x W at 3 * pixel_offset;
// alpha / target_alpha: per view one plane at pixel_offset.
double loss_fwd_bwd(int V, const int* W, const int* H, const double* rgb, const double* alpha,
                    const double* target_rgb, const double* target_alpha, const double* bg, double lambda,
                    double* dL_drgb, double* dL_dalpha, double* ssim_out /* nullable, per view */) {
    double w[WIN][WIN];
    window(w);
    double total = 0.0;
    long long poff = 0;
    for (int v = 0; v < V; ++v) {
        const int w_ = W[v], h_ = H[v];
        const long long P = (long long)w_ * h_;
        const double inv3P = 1.0 / (3.0 * P);
        double l1 = 0.0, ssim_sum = 0.0, la = 0.0;
        for (long long p = 0; p < P; ++p) {
            const double d = alpha[poff + p] - target_alpha[poff + p];
            la += std::fabs(d);
            dL_dalpha[poff + p] = sgn(d) / (double)P / V;
        }
        for (int ch = 0; ch < 3; ++ch) {
            const double* x = rgb + 3 * poff + ch * P;
            std::vector<double> y(P);
            for (long long p = 0; p < P; ++p)
                y[p] = target_rgb[3 * poff + ch * P + p] + (1.0 - target_alpha[poff + p]) * bg[3 * v + ch];
            // windowed moments, zero outside the image
            std::vector<double> mx(P), my(P), exx(P), eyy(P), exy(P);
            for (int py = 0; py < h_; ++py)
                for (int px = 0; px < w_; ++px) {
                    double a = 0, b = 0, c = 0, d = 0, e = 0;
                    for (int i = 0; i < WIN; ++i)
                        for (int j = 0; j < WIN; ++j) {
                            const int qy = py + i - HALF, qx = px + j - HALF;
                            if (qy < 0 || qy >= h_ || qx < 0 || qx >= w_) continue;
                            const double xv = x[(long long)qy * w_ + qx], yv = y[(long long)qy * w_ + qx];
                            a += w[i][j] * xv;
                            b += w[i][j] * yv;
                            c += w[i][j] * xv * xv;
                            d += w[i][j] * yv * yv;
                            e += w[i][j] * xv * yv;
                        }
                    const long long q = (long long)py * w_ + px;
                    mx[q] = a; my[q] = b; exx[q] = c; eyy[q] = d; exy[q] = e;
                }
            // SSIM map and its partials w.r.t. mu_x, E[x^2], E[xy] at each pixel
            std::vector<double> dmu(P), dxx(P), dxy(P);
            for (long long q = 0; q < P; ++q) {
                const double sx = exx[q] - mx[q] * mx[q], sy = eyy[q] - my[q] * my[q];
                const double sxy = exy[q] - mx[q] * my[q];
                const double A1 = 2 * mx[q] * my[q] + C1, A2 = 2 * sxy + C2;
                const double B1 = mx[q] * mx[q] + my[q] * my[q] + C1, B2 = sx + sy + C2;
                const double S = A1 * A2 / (B1 * B2);
                ssim_sum += S;
                dmu[q] = (2 * my[q] * A2 - 2 * my[q] * A1) / (B1 * B2) - S * (2 * mx[q] / B1 - 2 * mx[q] / B2);
                dxx[q] = -S / B2;
                dxy[q] = 2 * A1 / (B1 * B2);
            }
            // dL/dx_p = sum over pixels q whose window covers p
            for (int py = 0; py < h_; ++py)
                for (int px = 0; px < w_; ++px) {
                    const long long p = (long long)py * w_ + px;
                    double gm = 0, gxx = 0, gxy = 0;
                    for (int i = 0; i < WIN; ++i)
                        for (int j = 0; j < WIN; ++j) {
                            const int qy = py - (i - HALF), qx = px - (j - HALF);
                            if (qy < 0 || qy >= h_ || qx < 0 || qx >= w_) continue;
                            const long long q = (long long)qy * w_ + qx;
                            gm += w[i][j] * dmu[q];
                            gxx += w[i][j] * dxx[q];
                            gxy += w[i][j] * dxy[q];
                        }
                    const double dssim = gm + 2.0 * x[p] * gxx + y[p] * gxy;
                    l1 += std::fabs(x[p] - y[p]);
                    dL_drgb[3 * poff + ch * P + p] =
                        ((1.0 - lambda) * sgn(x[p] - y[p]) * inv3P - lambda * dssim * inv3P) / V;
                }
        }
        const double ssim_mean = ssim_sum * inv3P;
        if (ssim_out) ssim_out[v] = ssim_mean;
        total += ((1.0 - lambda) * l1 * inv3P + lambda * (1.0 - ssim_mean) + la / (double)P) / V;
        poff += P;
    }
    return total;
}

// Adam with bias correction (Kingma & Ba 2015), as used by 3DGS; the paper
// raises the scale / opacity / colour learning rates by about 50% for the
// abbreviated run and discards the optimiser state on restart (Section 4.2).
// step is 1-based.
void adam(long long n, double* p, const double* g, double* m, double* v, const double* lr, double b1, double b2,
          double eps, int step) {
    const double bc1 = 1.0 - std::pow(b1, step), bc2 = 1.0 - std::pow(b2, step);
    for (long long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mhat = m[i] / bc1, vhat = v[i] / bc2;
        p[i] -= lr[i] * mhat / (std::sqrt(vhat) + eps);
    }
}

}  // namespace oracle
