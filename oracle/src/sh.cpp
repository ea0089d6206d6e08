// Real spherical harmonics for the view-dependent colour of a Gaussian.
//
// The paper's model carries "RGBA color" from the transfer function
// (Section 4.1) and is fitted as a 3DGS model (Section 4.2), whose colour is
// a real spherical-harmonic expansion of the viewing direction of degree 0..3
// plus 0.5, clamped at zero. The basis is written out here from its
// definition rather than from hand-expanded polynomials:
//
//   Y_l^m(d) = N_lm * A_m(x, y) * D_lm(z)
//   N_lm     = sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!), times sqrt(2) if m != 0
//   A_m      = Re((x + i y)^m) for m > 0, Im((x + i y)^|m|) for m < 0, 1 for m = 0
//   D_lm(z)  = (-1)^|m| d^|m| P_l(z) / dz^|m|    (Condon-Shortley phase)
//
// with P_l the Legendre polynomials. On the unit sphere (x+iy)^|m| carries the
// (1 - z^2)^{|m|/2} factor of the associated Legendre function, so this is the
// usual real basis. Coefficients are ordered band by band, m = -l..l.
#include <cmath>
#include <vector>

#include "oracle.h"

namespace oracle {

namespace {

// Legendre polynomial P_l as coefficients c[0..l] (c[k] multiplies z^k),
// from Bonnet's recursion (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}.
std::vector<double> legendre(int l) {
    std::vector<double> p0{1.0}, p1{0.0, 1.0};
    if (l == 0) return p0;
    for (int n = 1; n < l; ++n) {
        std::vector<double> p2(n + 2, 0.0);
        for (int k = 0; k <= n; ++k) p2[k + 1] += (2.0 * n + 1.0) * p1[k];
        for (int k = 0; k < n; ++k) p2[k] -= n * p0[k];
        for (double& c : p2) c /= (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

std::vector<double> derivative(const std::vector<double>& c) {
    if (c.size() <= 1) return {0.0};
    std::vector<double> d(c.size() - 1);
    for (size_t k = 1; k < c.size(); ++k) d[k - 1] = k * c[k];
    return d;
}

double horner(const std::vector<double>& c, double z) {
    double r = 0.0;
    for (size_t k = c.size(); k-- > 0;) r = r * z + c[k];
    return r;
}

double factorial(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

// (x + i y)^n as (re, im); n >= 0.
void cpow(double x, double y, int n, double& re, double& im) {
    re = 1.0;
    im = 0.0;
    for (int k = 0; k < n; ++k) {
        double r = re * x - im * y;
        double i = re * y + im * x;
        re = r;
        im = i;
    }
}

}  // namespace

void real_sh(int deg, const double d[3], double* Y, double* dY) {
    const double x = d[0], y = d[1], z = d[2];
    int k = 0;
    for (int l = 0; l <= deg; ++l) {
        std::vector<double> P = legendre(l);
        for (int m = -l; m <= l; ++m, ++k) {
            const int am = m < 0 ? -m : m;
            double N = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            if (m != 0) N *= std::sqrt(2.0);
            std::vector<double> Dp = P;
            for (int r = 0; r < am; ++r) Dp = derivative(Dp);
            const double sgn = (am % 2) ? -1.0 : 1.0;
            const double D = sgn * horner(Dp, z);
            const double dD = sgn * horner(derivative(Dp), z);
            double re, im, re1 = 0.0, im1 = 0.0;
            cpow(x, y, am, re, im);
            if (am > 0) cpow(x, y, am - 1, re1, im1);
            double A, dAx, dAy;
            if (m > 0) {          // Re((x+iy)^m)
                A = re;
                dAx = am * re1;
                dAy = -am * im1;
            } else if (m < 0) {   // Im((x+iy)^|m|)
                A = im;
                dAx = am * im1;
                dAy = am * re1;
            } else {
                A = 1.0;
                dAx = 0.0;
                dAy = 0.0;
            }
            Y[k] = N * A * D;
            if (dY) {
                dY[3 * k + 0] = N * dAx * D;
                dY[3 * k + 1] = N * dAy * D;
                dY[3 * k + 2] = N * A * dD;
            }
        }
    }
}

}  // namespace oracle
