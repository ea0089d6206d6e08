// FP64 CPU oracle of the periphery fit step (test infrastructure only).
//
// This is the plain, slow, reference implementation that the GPU path is
// checked against. It is used by the tests, by the CPU baseline leg of the
// benchmark and by the smoke check only; the product path never calls it.
// It shares no code with the CUDA kernels.
//
// Section 4.2 fits the peripheral model with a 3D Gaussian Splatting
// optimisation (built on Mini-Splatting2 / Taming 3DGS) with alpha training
// and randomised backgrounds; the paper does not write the splatting math
// out, so every stage below follows the standard 3DGS conventions (Kerbl et
// al. 2023: EWA splatting after Zwicker et al. 2001, real spherical-harmonic
// colour, tile-binned front-to-back compositing, L1 + D-SSIM loss, Adam).
// Floating point is FP64 throughout except where a float32 value decides an
// integer (the depth key, the depth cull and the tile rectangle); those are
// computed in float32 with a fixed order of correctly rounded operations so
// that the decision is reproducible bit for bit.
#pragma once
#include <cstdint>
#include <vector>

namespace oracle {

// Relative margin of the compositing's near-threshold flags (raster.cpp).
extern double g_threshold_margin;


// One pinhole camera. viewmat rows are the camera's right, down and forward
// axes; p_cam = R p_world + t. campos is the camera centre in world space.
struct Camera {
    double R[3][3], t[3], campos[3];
    float Rf[3][3], tf[3];          // the same values as stored in float32
    double fx, fy, cx, cy, near_plane;
    float fxf, fyf, cxf, cyf, nearf;
    int W, H;
    int tiles_x, tiles_y, tile_offset;  // for a given tile size
    long long pixel_offset;
};

// Number of doubles per camera record in the C interface:
// viewmat[12], campos[3], fx, fy, cx, cy, near, W, H.
constexpr int CAM_DOUBLES = 24;

// Gaussian record in the C interface (doubles, one Gaussian after another):
// mean[3], log_scale[3], quat[4] (w, x, y, z), opacity_logit, sh[K][3].
inline int gauss_stride(int K) { return 11 + 3 * K; }

// Per-(view, Gaussian) projected record (doubles) in the C interface.
enum ProjField {
    P_VISIBLE = 0,  // 1 if the Gaussian is binned into at least one tile
    P_DEPTH32,      // float32 camera-space depth (exact value)
    P_U, P_V,       // FP64 pixel-space centre
    P_U32, P_V32,   // float32 pixel-space centre: decides the tile rectangle and
                    // is the centre used in compositing
    P_RADIUS,       // integer pixel radius ceil(3 sqrt(lambda_max))
    P_CONIC_A, P_CONIC_B, P_CONIC_C,  // inverse 2D covariance (a', b', c')
    P_COV_A, P_COV_B, P_COV_C,        // dilated 2D covariance
    P_OPACITY,
    P_R, P_G, P_B,                     // clamped colour
    P_CLAMP_R, P_CLAMP_G, P_CLAMP_B,   // 1 where the colour clamp is active
    P_RECT_X0, P_RECT_Y0, P_RECT_X1, P_RECT_Y1,  // tiles [x0, x1) x [y0, y1)
    P_TILES,
    P_NEAR_BOUNDARY,  // 1 if float32 rounding could move the radius across an integer
    P_STRIDE
};

constexpr int FLAG_SMOOTH = 1;  // no culls / skips / early stop (finite-difference mode)

constexpr double ALPHA_CLAMP = 0.99;
constexpr double ALPHA_SKIP = 1.0 / 255.0;
constexpr double T_STOP = 1e-4;
constexpr double COV_DILATION = 0.3;
constexpr double FRUSTUM_GUARD = 1.3;

std::vector<Camera> unpack_cameras(int V, const double* cams, int tile);
int total_tiles(const std::vector<Camera>& cams);

// Real spherical harmonics (Condon-Shortley phase, m = -l..l per band):
// Y[k] for k < (deg+1)^2 at unit direction d, and optionally dY/dd (3 per k)
// treating the polynomial form as a function of independent x, y, z.
void real_sh(int deg, const double d[3], double* Y, double* dY /* nullable, 3 per k */);

void project_one(const double* g, int K, const Camera& cam, int tile, int flags, double* out);

}  // namespace oracle
