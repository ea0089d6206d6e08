// Tile binning, front-to-back compositing and its adjoint.
//
// Section 4.2: the periphery is rendered and trained as a 3DGS model with
// alpha training and randomised backgrounds. Per pixel, the Gaussians whose
// tile rectangle covers the pixel's tile are taken in order of increasing
// float32 depth (ties by Gaussian index) and composited front to back:
//   power = -1/2 (a' dx^2 + c' dy^2) - b' dx dy,  skipped if power > 0
//   alpha = min(0.99, o exp(power)),              skipped if alpha < 1/255
//   stop before a Gaussian that would take T below 1e-4
//   C = sum c_i alpha_i T_i + T_N bg,   A = 1 - T_N
// n_contrib is one past the list position of the last blended Gaussian.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "oracle.h"

namespace oracle {

// Keys ((global tile id) << 32 | float32 depth bits) and values (Gaussian
// index) of every (Gaussian, covered tile) pair, emitted view by view,
// Gaussian by Gaussian, tiles row-major, then stably sorted by key; and the
// [start, end) range of every tile. Returns the number of pairs.
long long bin_tiles(int n, const std::vector<Camera>& cams, const double* proj, std::vector<uint64_t>& keys,
                    std::vector<uint32_t>& vals, std::vector<uint32_t>& ranges) {
    keys.clear();
    vals.clear();
    const int V = (int)cams.size();
    for (int v = 0; v < V; ++v) {
        const Camera& cam = cams[v];
        for (int i = 0; i < n; ++i) {
            const double* p = proj + ((size_t)v * n + i) * P_STRIDE;
            if (p[P_VISIBLE] == 0.0 || p[P_TILES] == 0.0) continue;
            float d = (float)p[P_DEPTH32];
            uint32_t bits;
            std::memcpy(&bits, &d, 4);
            for (int ty = (int)p[P_RECT_Y0]; ty < (int)p[P_RECT_Y1]; ++ty)
                for (int tx = (int)p[P_RECT_X0]; tx < (int)p[P_RECT_X1]; ++tx) {
                    const uint64_t tile = (uint64_t)(cam.tile_offset + ty * cam.tiles_x + tx);
                    keys.push_back((tile << 32) | bits);
                    vals.push_back((uint32_t)i);
                }
        }
    }
    std::vector<size_t> order(keys.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return keys[a] < keys[b]; });
    std::vector<uint64_t> k2(keys.size());
    std::vector<uint32_t> v2(vals.size());
    for (size_t j = 0; j < order.size(); ++j) {
        k2[j] = keys[order[j]];
        v2[j] = vals[order[j]];
    }
    keys.swap(k2);
    vals.swap(v2);
    const int T = total_tiles(cams);
    ranges.assign(2 * (size_t)T, 0u);
    for (size_t j = 0; j < keys.size(); ++j) {
        const uint32_t t = (uint32_t)(keys[j] >> 32);
        if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[2 * t] = (uint32_t)j;
        if (j + 1 == keys.size() || (uint32_t)(keys[j + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    return (long long)keys.size();
}

// Relative margin of the near-threshold flags (2e-4 by default; a test of a
// lower-precision form widens it with oracle_set_threshold_margin). It only
// flags pixels and Gaussians; it changes no computed value.
double g_threshold_margin = 2e-4;

namespace {

struct Blend {
    int pos, gauss;
    double alpha, T, G, dx, dy;
    bool clamped;
};

struct Pixel {
    double C[3], T;
    int n_contrib;
    bool ambiguous;
    std::vector<Blend> blends;
    std::vector<int> ambiguous_gauss;  // Gaussians whose own decision was near a threshold
};

// |x - thr| within a relative margin: float32 rounding on the GPU side could
// take the other branch of this comparison (g_threshold_margin).
inline bool near_threshold(double x, double thr) { return std::fabs(x - thr) <= g_threshold_margin * thr; }

void composite_pixel(int px, int py, const uint32_t* list, int count, const double* proj_v, int flags, Pixel& out) {
    const bool smooth = flags & FLAG_SMOOTH;
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    out.n_contrib = 0;
    out.ambiguous = false;
    out.blends.clear();
    out.ambiguous_gauss.clear();
    for (int j = 0; j < count; ++j) {
        const int gi = (int)list[j];
        const double* p = proj_v + (size_t)gi * P_STRIDE;
        // Normal mode takes the splat centre at its float32 value (computed
        // with correctly rounded float32 operations, it is identical in every
        // implementation and already decides the tile rectangle); smooth mode
        // keeps the FP64 centre so the image is differentiable in the mean.
        const double dx = px - (smooth ? p[P_U] : p[P_U32]);
        const double dy = py - (smooth ? p[P_V] : p[P_V32]);
        const double power = -0.5 * (p[P_CONIC_A] * dx * dx + p[P_CONIC_C] * dy * dy) - p[P_CONIC_B] * dx * dy;
        if (power > 0.0) continue;
        const double G = std::exp(power);
        const double a = p[P_OPACITY] * G;
        const bool clamped = a > ALPHA_CLAMP;
        const double alpha = clamped ? ALPHA_CLAMP : a;
        bool amb = near_threshold(a, ALPHA_CLAMP);
        if (!smooth) amb = amb || near_threshold(a, ALPHA_SKIP);
        if (amb) {
            out.ambiguous = true;
            out.ambiguous_gauss.push_back(gi);
        }
        if (!smooth && alpha < ALPHA_SKIP) continue;
        const double Tn = T * (1.0 - alpha);
        if (!smooth) {
            if (near_threshold(Tn, T_STOP)) {
                out.ambiguous = true;
                out.ambiguous_gauss.push_back(gi);
            }
            if (Tn < T_STOP) break;
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += p[P_R + ch] * alpha * T;
        out.blends.push_back(Blend{j, gi, alpha, T, G, dx, dy, clamped});
        T = Tn;
        out.n_contrib = j + 1;
    }
    for (int ch = 0; ch < 3; ++ch) out.C[ch] = C[ch];
    out.T = T;
}

// The pixel's list is its tile's sorted range (normal mode) or every visible
// Gaussian of the view in depth order (smooth mode).
std::vector<uint32_t> depth_sorted_visible(int n, const double* proj_v) {
    std::vector<uint32_t> idx;
    for (int i = 0; i < n; ++i)
        if (proj_v[(size_t)i * P_STRIDE + P_VISIBLE] != 0.0) idx.push_back((uint32_t)i);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
        float da = (float)proj_v[(size_t)a * P_STRIDE + P_DEPTH32];
        float db = (float)proj_v[(size_t)b * P_STRIDE + P_DEPTH32];
        return da < db;
    });
    return idx;
}

struct WorkItem {
    int v, tx, ty;
};

std::vector<WorkItem> work_items(const std::vector<Camera>& cams) {
    std::vector<WorkItem> w;
    for (int v = 0; v < (int)cams.size(); ++v)
        for (int ty = 0; ty < cams[v].tiles_y; ++ty)
            for (int tx = 0; tx < cams[v].tiles_x; ++tx) w.push_back(WorkItem{v, tx, ty});
    return w;
}

}  // namespace

// importance (optional, n entries, added to): per Gaussian the sum over the
// pixels of its blend weight alpha T, the weight its colour receives in C.
void render_fwd(int n, const std::vector<Camera>& cams, int tile, const double* proj, const uint32_t* vals,
                const uint32_t* ranges, const double* bg, int flags, double* rgb, double* alpha, double* T_final,
                int32_t* n_contrib, uint8_t* ambiguous, int32_t* n_blended, double* importance) {
    const int V = (int)cams.size();
    std::vector<std::vector<uint32_t>> sorted(V);
    if (flags & FLAG_SMOOTH)
        for (int v = 0; v < V; ++v) sorted[v] = depth_sorted_visible(n, proj + (size_t)v * n * P_STRIDE);
    const std::vector<WorkItem> items = work_items(cams);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long w = 0; w < (long long)items.size(); ++w) {
        const WorkItem it = items[w];
        const Camera& cam = cams[it.v];
        const double* proj_v = proj + (size_t)it.v * n * P_STRIDE;
        const uint32_t* list;
        int count;
        if (flags & FLAG_SMOOTH) {
            list = sorted[it.v].data();
            count = (int)sorted[it.v].size();
        } else {
            const int t = cam.tile_offset + it.ty * cam.tiles_x + it.tx;
            list = vals + ranges[2 * t];
            count = (int)(ranges[2 * t + 1] - ranges[2 * t]);
        }
        Pixel px;
        for (int py = it.ty * tile; py < std::min((it.ty + 1) * tile, cam.H); ++py)
            for (int pxx = it.tx * tile; pxx < std::min((it.tx + 1) * tile, cam.W); ++pxx) {
                composite_pixel(pxx, py, list, count, proj_v, flags, px);
                const long long pix = cam.pixel_offset + (long long)py * cam.W + pxx;
                const long long plane = (long long)cam.W * cam.H;
                for (int ch = 0; ch < 3; ++ch)
                    rgb[3 * cam.pixel_offset + ch * plane + (long long)py * cam.W + pxx] =
                        px.C[ch] + px.T * bg[3 * it.v + ch];
                alpha[pix] = 1.0 - px.T;
                T_final[pix] = px.T;
                n_contrib[pix] = px.n_contrib;
                ambiguous[pix] = px.ambiguous ? 1 : 0;
                if (n_blended) n_blended[pix] = (int32_t)px.blends.size();
                if (importance)
                    for (const Blend& e : px.blends) {
#pragma omp atomic
                        importance[e.gauss] += e.alpha * e.T;
                    }
            }
    }
}

void project_bwd_one(const double* g, int K, const Camera& cam, const double g2[9], double* gout);

// Adjoint of render_fwd followed by the projection adjoint. dL_drgb and
// dL_dalpha are the upstream gradients in the image layout; grad2d receives
// dL/d(u, v, a', b', c', opacity, r, g, b) per (view, Gaussian) and grads the
// sum over views of dL/d(parameters). gauss_ambiguous marks (view, Gaussian)
// pairs blended at a pixel with a near-threshold decision.
void render_bwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, const double* proj,
                const uint32_t* vals, const uint32_t* ranges, const double* bg, int flags, const double* dL_drgb,
                const double* dL_dalpha, double* grad2d, double* grads, uint8_t* gauss_ambiguous) {
    const int V = (int)cams.size();
    std::memset(grad2d, 0, sizeof(double) * 9 * (size_t)V * n);
    std::memset(gauss_ambiguous, 0, (size_t)V * n);
    std::vector<std::vector<uint32_t>> sorted(V);
    if (flags & FLAG_SMOOTH)
        for (int v = 0; v < V; ++v) sorted[v] = depth_sorted_visible(n, proj + (size_t)v * n * P_STRIDE);
    const std::vector<WorkItem> items = work_items(cams);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long w = 0; w < (long long)items.size(); ++w) {
        const WorkItem it = items[w];
        const Camera& cam = cams[it.v];
        const double* proj_v = proj + (size_t)it.v * n * P_STRIDE;
        double* g2v = grad2d + (size_t)it.v * n * 9;
        const uint32_t* list;
        int count;
        if (flags & FLAG_SMOOTH) {
            list = sorted[it.v].data();
            count = (int)sorted[it.v].size();
        } else {
            const int t = cam.tile_offset + it.ty * cam.tiles_x + it.tx;
            list = vals + ranges[2 * t];
            count = (int)(ranges[2 * t + 1] - ranges[2 * t]);
        }
        Pixel px;
        const long long plane = (long long)cam.W * cam.H;
        for (int py = it.ty * tile; py < std::min((it.ty + 1) * tile, cam.H); ++py)
            for (int pxx = it.tx * tile; pxx < std::min((it.tx + 1) * tile, cam.W); ++pxx) {
                composite_pixel(pxx, py, list, count, proj_v, flags, px);
                const long long pix = cam.pixel_offset + (long long)py * cam.W + pxx;
                double dC[3];
                for (int ch = 0; ch < 3; ++ch)
                    dC[ch] = dL_drgb[3 * cam.pixel_offset + ch * plane + (long long)py * cam.W + pxx];
                const double dA = dL_dalpha[pix];
                const double TN = px.T;
                double S[3] = {0.0, 0.0, 0.0};  // sum over later Gaussians of c alpha T
                for (int b = (int)px.blends.size() - 1; b >= 0; --b) {
                    const Blend& e = px.blends[b];
                    const double* p = proj_v + (size_t)e.gauss * P_STRIDE;
                    double dalpha = dA * TN / (1.0 - e.alpha);
                    double* out = g2v + (size_t)e.gauss * 9;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double c = p[P_R + ch];
                        dalpha += dC[ch] * (e.T * c - (S[ch] + TN * bg[3 * it.v + ch]) / (1.0 - e.alpha));
#pragma omp atomic
                        out[6 + ch] += dC[ch] * e.alpha * e.T;
                    }
                    for (int ch = 0; ch < 3; ++ch) S[ch] += p[P_R + ch] * e.alpha * e.T;
                    if (e.clamped) continue;  // alpha = 0.99 does not depend on o or power
                    const double dpower = dalpha * e.alpha;
                    const double gu = dpower * (p[P_CONIC_A] * e.dx + p[P_CONIC_B] * e.dy);
                    const double gv = dpower * (p[P_CONIC_C] * e.dy + p[P_CONIC_B] * e.dx);
                    const double ga = dpower * (-0.5 * e.dx * e.dx);
                    const double gb = dpower * (-e.dx * e.dy);
                    const double gc = dpower * (-0.5 * e.dy * e.dy);
                    const double go = dalpha * e.G;
#pragma omp atomic
                    out[0] += gu;
#pragma omp atomic
                    out[1] += gv;
#pragma omp atomic
                    out[2] += ga;
#pragma omp atomic
                    out[3] += gb;
#pragma omp atomic
                    out[4] += gc;
#pragma omp atomic
                    out[5] += go;
                }
                for (int gi : px.ambiguous_gauss) gauss_ambiguous[(size_t)it.v * n + gi] = 1;
            }
    }
    const int stride = gauss_stride(K);
    std::memset(grads, 0, sizeof(double) * (size_t)n * stride);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int v = 0; v < V; ++v) {
            const double* p = proj + ((size_t)v * n + i) * P_STRIDE;
            if (p[P_VISIBLE] == 0.0) continue;
            project_bwd_one(gauss + (size_t)i * stride, K, cams[v], grad2d + ((size_t)v * n + i) * 9,
                            grads + (size_t)i * stride);
        }
}

}  // namespace oracle

// ---------------------------------------------------------------------------
// Sampled evaluation for workloads too large to render whole (the same
// arithmetic as above, one view at a time, only where asked).
// ---------------------------------------------------------------------------

namespace oracle {

namespace {

// Projection and sorted tile lists of one view.
struct ViewBins {
    std::vector<double> proj;  // n * P_STRIDE
    std::vector<uint64_t> keys;
    std::vector<uint32_t> vals, ranges;
};

void bin_view(int n, int K, const double* gauss, const Camera& cam, int tile, ViewBins& vb) {
    vb.proj.assign((size_t)n * P_STRIDE, 0.0);
    const int stride = gauss_stride(K);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) project_one(gauss + (size_t)i * stride, K, cam, tile, 0, vb.proj.data() + (size_t)i * P_STRIDE);
    Camera c = cam;
    c.tile_offset = 0;
    c.pixel_offset = 0;
    std::vector<Camera> one{c};
    bin_tiles(n, one, vb.proj.data(), vb.keys, vb.vals, vb.ranges);
}

}  // namespace

// items: n_items (view, local tile) pairs. Per item, B x B pixels (row-major
// in the tile; pixels outside the view get n_contrib -1): colour (3 planes),
// alpha, T_final, n_contrib, ambiguity, and (if nb is not null) the number of
// blended and of clamped Gaussians (nb: 2 ints per pixel); and the tile's
// sorted Gaussian list (list_len[item] entries, at most max_list copied).
void tiles_fwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, int n_items,
               const int32_t* items, const double* bg, double* rgb, double* alpha, double* T_final, int32_t* nc,
               uint8_t* amb, int32_t* list_len, uint32_t* lists, int max_list, int32_t* nb) {
    const int B2 = tile * tile;
    for (int v = 0; v < (int)cams.size(); ++v) {
        bool any = false;
        for (int k = 0; k < n_items; ++k) any = any || items[2 * k] == v;
        if (!any) continue;
        ViewBins vb;
        bin_view(n, K, gauss, cams[v], tile, vb);
        const Camera& cam = cams[v];
        for (int k = 0; k < n_items; ++k) {
            if (items[2 * k] != v) continue;
            const int t = items[2 * k + 1];
            const int tx = t % cam.tiles_x, ty = t / cam.tiles_x;
            const uint32_t* list = vb.vals.data() + vb.ranges[2 * t];
            const int count = (int)(vb.ranges[2 * t + 1] - vb.ranges[2 * t]);
            list_len[k] = count;
            for (int j = 0; j < count && j < max_list; ++j) lists[(size_t)k * max_list + j] = list[j];
            Pixel px;
            for (int q = 0; q < B2; ++q) {
                const int pxx = tx * tile + q % tile, py = ty * tile + q / tile;
                const size_t o = (size_t)k * B2 + q;
                if (pxx >= cam.W || py >= cam.H) {
                    nc[o] = -1;
                    continue;
                }
                composite_pixel(pxx, py, list, count, vb.proj.data(), 0, px);
                for (int ch = 0; ch < 3; ++ch) rgb[3 * (size_t)k * B2 + ch * B2 + q] = px.C[ch] + px.T * bg[3 * v + ch];
                alpha[o] = 1.0 - px.T;
                T_final[o] = px.T;
                nc[o] = px.n_contrib;
                amb[o] = px.ambiguous ? 1 : 0;
                if (nb) {
                    int clamped = 0;
                    for (const Blend& e : px.blends) clamped += e.clamped ? 1 : 0;
                    nb[2 * o] = (int32_t)px.blends.size();
                    nb[2 * o + 1] = clamped;
                }
            }
        }
    }
}

// Complete parameter gradients of the requested Gaussians: every tile any of
// them covers is composited and back-propagated in full; dL_drgb / dL_dalpha
// are the packed full-batch upstream gradients. amb_out marks requested
// Gaussians whose own decision was near a threshold somewhere (or whose radius
// lies within rounding of an integer in some view).
void gauss_bwd(int n, int K, const double* gauss, const std::vector<Camera>& cams, int tile, const double* bg,
               const double* dL_drgb, const double* dL_dalpha, int n_req, const int32_t* req, double* grads_out,
               uint8_t* amb_out) {
    const int stride = gauss_stride(K);
    std::memset(grads_out, 0, sizeof(double) * (size_t)n_req * stride);
    std::memset(amb_out, 0, (size_t)n_req);
    std::vector<int> slot(n, -1);
    for (int r = 0; r < n_req; ++r) slot[req[r]] = r;
    for (int v = 0; v < (int)cams.size(); ++v) {
        const Camera& cam = cams[v];
        ViewBins vb;
        bin_view(n, K, gauss, cam, tile, vb);
        std::vector<char> want((size_t)cam.tiles_x * cam.tiles_y, 0);
        bool any = false;
        for (int r = 0; r < n_req; ++r) {
            const double* p = vb.proj.data() + (size_t)req[r] * P_STRIDE;
            if (p[P_VISIBLE] == 0.0) continue;
            if (p[P_NEAR_BOUNDARY] != 0.0) amb_out[r] = 1;
            for (int ty = (int)p[P_RECT_Y0]; ty < (int)p[P_RECT_Y1]; ++ty)
                for (int tx = (int)p[P_RECT_X0]; tx < (int)p[P_RECT_X1]; ++tx) want[(size_t)ty * cam.tiles_x + tx] = 1;
            any = true;
        }
        if (!any) continue;
        std::vector<double> g2((size_t)n_req * 9, 0.0);
        const long long plane = (long long)cam.W * cam.H;
        for (int t = 0; t < cam.tiles_x * cam.tiles_y; ++t) {
            if (!want[t]) continue;
            const int tx = t % cam.tiles_x, ty = t / cam.tiles_x;
            const uint32_t* list = vb.vals.data() + vb.ranges[2 * t];
            const int count = (int)(vb.ranges[2 * t + 1] - vb.ranges[2 * t]);
            Pixel px;
            for (int py = ty * tile; py < std::min((ty + 1) * tile, cam.H); ++py)
                for (int pxx = tx * tile; pxx < std::min((tx + 1) * tile, cam.W); ++pxx) {
                    composite_pixel(pxx, py, list, count, vb.proj.data(), 0, px);
                    for (int gi : px.ambiguous_gauss)
                        if (slot[gi] >= 0) amb_out[slot[gi]] = 1;
                    const long long pix = cam.pixel_offset + (long long)py * cam.W + pxx;
                    double dC[3];
                    for (int ch = 0; ch < 3; ++ch)
                        dC[ch] = dL_drgb[3 * cam.pixel_offset + ch * plane + (long long)py * cam.W + pxx];
                    const double dA = dL_dalpha[pix];
                    const double TN = px.T;
                    double S[3] = {0.0, 0.0, 0.0};
                    for (int b = (int)px.blends.size() - 1; b >= 0; --b) {
                        const Blend& e = px.blends[b];
                        const double* p = vb.proj.data() + (size_t)e.gauss * P_STRIDE;
                        const int sl = slot[e.gauss];
                        double dalpha = dA * TN / (1.0 - e.alpha);
                        for (int ch = 0; ch < 3; ++ch) {
                            const double c = p[P_R + ch];
                            dalpha += dC[ch] * (e.T * c - (S[ch] + TN * bg[3 * v + ch]) / (1.0 - e.alpha));
                            if (sl >= 0) g2[(size_t)sl * 9 + 6 + ch] += dC[ch] * e.alpha * e.T;
                        }
                        for (int ch = 0; ch < 3; ++ch) S[ch] += p[P_R + ch] * e.alpha * e.T;
                        if (sl < 0 || e.clamped) continue;
                        const double dpower = dalpha * e.alpha;
                        double* out = g2.data() + (size_t)sl * 9;
                        out[0] += dpower * (p[P_CONIC_A] * e.dx + p[P_CONIC_B] * e.dy);
                        out[1] += dpower * (p[P_CONIC_C] * e.dy + p[P_CONIC_B] * e.dx);
                        out[2] += dpower * (-0.5 * e.dx * e.dx);
                        out[3] += dpower * (-e.dx * e.dy);
                        out[4] += dpower * (-0.5 * e.dy * e.dy);
                        out[5] += dalpha * e.G;
                    }
                }
        }
        for (int r = 0; r < n_req; ++r) {
            const double* p = vb.proj.data() + (size_t)req[r] * P_STRIDE;
            if (p[P_VISIBLE] == 0.0) continue;
            project_bwd_one(gauss + (size_t)req[r] * stride, K, cam, g2.data() + (size_t)r * 9,
                            grads_out + (size_t)r * stride);
        }
    }
}

}  // namespace oracle
