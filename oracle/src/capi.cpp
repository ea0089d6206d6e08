// C interface of the oracle (loaded with ctypes by oracle/__init__.py).
// All arrays are caller-owned host memory.
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

namespace oracle {
long long bin_tiles(int n, const std::vector<Camera>& cams, const double* proj, std::vector<uint64_t>& keys,
                    std::vector<uint32_t>& vals, std::vector<uint32_t>& ranges);
void render_fwd(int n, const std::vector<Camera>& cams, int tile, const double* proj, const uint32_t* vals,
                const uint32_t* ranges, const double* bg, int flags, double* rgb, double* alpha, double* T_final,
                int32_t* n_contrib, uint8_t* ambiguous, int32_t* n_blended, double* importance);
void render_bwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, const double* proj,
                const uint32_t* vals, const uint32_t* ranges, const double* bg, int flags, const double* dL_drgb,
                const double* dL_dalpha, double* grad2d, double* grads, uint8_t* gauss_ambiguous);
double loss_fwd_bwd(int V, const int* W, const int* H, const double* rgb, const double* alpha,
                    const double* target_rgb, const double* target_alpha, const double* bg, double lambda,
                    double* dL_drgb, double* dL_dalpha, double* ssim_out);
void adam(long long n, double* p, const double* g, double* m, double* v, const double* lr, double b1, double b2,
          double eps, int step);
void tiles_fwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, int n_items,
               const int32_t* items, const double* bg, double* rgb, double* alpha, double* T_final, int32_t* nc,
               uint8_t* amb, int32_t* list_len, uint32_t* lists, int max_list, int32_t* nb);
void gauss_bwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, const double* bg,
               const double* dL_drgb, const double* dL_dalpha, int n_req, const int32_t* req, double* grads_out,
               uint8_t* amb_out);
void project_bwd_one(const double* g, int K, const Camera& cam, const double g2[9], double* gout);
}  // namespace oracle

using namespace oracle;

extern "C" {

int oracle_proj_stride(void) { return P_STRIDE; }

// Relative margin of the near-threshold flags of the compositing (see raster.cpp).
void oracle_set_threshold_margin(double m) { oracle::g_threshold_margin = m; }
double oracle_threshold_margin(void) { return oracle::g_threshold_margin; }
int oracle_cam_doubles(void) { return CAM_DOUBLES; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_total_tiles(int V, const double* cams, int tile) { return total_tiles(unpack_cameras(V, cams, tile)); }

// proj: V * n * P_STRIDE doubles
void oracle_project(int n, int K, const double* gauss, int V, const double* cams, int tile, int flags,
                    double* proj) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    const int stride = gauss_stride(K);
#pragma omp parallel for schedule(static)
    for (long long w = 0; w < (long long)V * n; ++w) {
        const int v = (int)(w / n), i = (int)(w % n);
        project_one(gauss + (size_t)i * stride, K, c[v], tile, flags, proj + (size_t)w * P_STRIDE);
    }
}

// Returns the number of (Gaussian, tile) pairs; copies at most `capacity` of
// them. ranges: 2 * total_tiles entries.
long long oracle_bin(int n, int V, const double* cams, int tile, const double* proj, uint64_t* keys,
                     uint32_t* vals, long long capacity, uint32_t* ranges) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    std::vector<uint64_t> k;
    std::vector<uint32_t> v, r;
    const long long count = bin_tiles(n, c, proj, k, v, r);
    const long long m = count < capacity ? count : capacity;
    if (m > 0) {
        std::memcpy(keys, k.data(), sizeof(uint64_t) * m);
        std::memcpy(vals, v.data(), sizeof(uint32_t) * m);
    }
    std::memcpy(ranges, r.data(), sizeof(uint32_t) * r.size());
    return count;
}

void oracle_render_fwd(int n, int V, const double* cams, int tile, const double* proj, const uint32_t* vals,
                       const uint32_t* ranges, const double* bg, int flags, double* rgb, double* alpha,
                       double* T_final, int32_t* n_contrib, uint8_t* ambiguous, int32_t* n_blended,
                       double* importance) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    render_fwd(n, c, tile, proj, vals, ranges, bg, flags, rgb, alpha, T_final, n_contrib, ambiguous, n_blended,
               importance);
}

void oracle_render_bwd(int n, int K, const double* gauss, int V, const double* cams, int tile, const double* proj,
                       const uint32_t* vals, const uint32_t* ranges, const double* bg, int flags,
                       const double* dL_drgb, const double* dL_dalpha, double* grad2d, double* grads,
                       uint8_t* gauss_ambiguous) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    render_bwd(n, K, gauss, c, tile, proj, vals, ranges, bg, flags, dL_drgb, dL_dalpha, grad2d, grads,
               gauss_ambiguous);
}

// The projection adjoint alone (the second half of oracle_render_bwd): for
// every visible (view, Gaussian) record, dL/d(parameters) of the 2D gradients
// in grad2d (V * n * 9, the layout render_bwd writes), summed over views into
// grads (zeroed first). Used to time the per-view share of an iteration.
void oracle_project_bwd(int n, int K, const double* gauss, int V, const double* cams, int tile, const double* proj,
                        const double* grad2d, double* grads) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    const int stride = gauss_stride(K);
    std::memset(grads, 0, sizeof(double) * (size_t)n * stride);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int v = 0; v < V; ++v) {
            const double* p = proj + ((size_t)v * n + i) * P_STRIDE;
            if (p[P_VISIBLE] == 0.0) continue;
            project_bwd_one(gauss + (size_t)i * stride, K, c[v], grad2d + ((size_t)v * n + i) * 9,
                            grads + (size_t)i * stride);
        }
}

double oracle_loss(int V, const int* W, const int* H, const double* rgb, const double* alpha,
                   const double* target_rgb, const double* target_alpha, const double* bg, double lambda,
                   double* dL_drgb, double* dL_dalpha, double* ssim_out) {
    return loss_fwd_bwd(V, W, H, rgb, alpha, target_rgb, target_alpha, bg, lambda, dL_drgb, dL_dalpha, ssim_out);
}

void oracle_adam(long long n, double* p, const double* g, double* m, double* v, const double* lr, double b1,
                 double b2, double eps, int step) {
    adam(n, p, g, m, v, lr, b1, b2, eps, step);
}

void oracle_real_sh(int deg, const double* dir, double* Y, double* dY) { real_sh(deg, dir, Y, dY); }

void oracle_tiles_fwd(int n, int K, const double* gauss, int V, const double* cams, int tile, int n_items,
                      const int32_t* items, const double* bg, double* rgb, double* alpha, double* T_final,
                      int32_t* nc, uint8_t* amb, int32_t* list_len, uint32_t* lists, int max_list, int32_t* nb) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    tiles_fwd(n, K, gauss, c, tile, n_items, items, bg, rgb, alpha, T_final, nc, amb, list_len, lists, max_list, nb);
}

void oracle_gauss_bwd(int n, int K, const double* gauss, int V, const double* cams, int tile, const double* bg,
                      const double* dL_drgb, const double* dL_dalpha, int n_req, const int32_t* req,
                      double* grads_out, uint8_t* amb_out) {
    const std::vector<Camera> c = unpack_cameras(V, cams, tile);
    gauss_bwd(n, K, gauss, c, tile, bg, dL_drgb, dL_dalpha, n_req, req, grads_out, amb_out);
}

}  // extern "C"
