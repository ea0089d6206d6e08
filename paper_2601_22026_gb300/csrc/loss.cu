// Photometric loss of a view batch and its gradient (3DGS loss on colour with
// an added L1 term on alpha for the alpha supervision of Section 4.2; targets
// are composited over the same randomised background as the render).
//
// Design: one work item is a 32 x 32 output tile of one colour channel of one
// view. The item loads render and target over the tile plus a 10-pixel halo
// into shared memory, forms the four windowed moments mu_x, mu_y, E[x^2 +
// y^2], E[xy] on the tile plus a 5-pixel halo with two separable 11-tap
// passes (SSIM uses the two variances only through their sum, so one moment
// of x^2 + y^2 serves both), evaluates the SSIM map and
// its partials there, and convolves the partials back onto the tile: the
// gradient of the windowed SSIM never leaves shared memory: the kernel reads
// each input region once from DRAM (the output pixels' own values a second
// time, from L2, for the gradient) and writes each gradient once. Channel-0 items
// also handle the alpha term. Persistent CTAs stride over the items.
// Where render and target are equal over an item's whole input region (the
// background around the splats), SSIM is 1 there and the colour gradient
// zero: such items skip the stencil. A pre-pass reads the images once and
// records per 16 x 16 block and channel whether they agree, so that most such
// items are settled without loading their regions.
#include "common.cuh"

namespace gsfit {

namespace {

constexpr int kOut = 32;             // output tile edge
constexpr int kR1 = kOut + 10;       // moments / partials region (halo 5): 42
constexpr int kR2 = kOut + 20;       // input region (halo 10): 52
constexpr int kLossThreads = 256;
constexpr int kLossCtasPerSm = 4;    // 64 registers, 56.6 KB of shared memory each
static_assert(kR1 % 3 == 0 && kR1 % 7 == 0, "strip lengths of the stencil passes divide the region");
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

// 56.6 KB: four CTAs per SM. The input region is reused for the SSIM partials
// and the horizontal-pass buffer for the horizontal pass of the partials.
// Maps that the packed two-lane FMAs take together are interleaved as float2,
// so one 8-byte shared-memory access moves an operand pair.
struct LossSmem {
    union {
        float2 xy[kR2][kR2];           // (render, target over the background), input region; zero outside the image
        struct {
            float2 p01[kR1][kR1];      // dSSIM/d(mu_x, E[x^2 + y^2]) on the 42 x 42 region
            float p2[kR1][kR1];        // dSSIM/dE[xy]
        } part;
    } a;
    union {
        struct {
            float2 h01[kR2][kR1];      // horizontal pass of (x, y)
            float2 h23[kR2][kR1];      // horizontal pass of (x^2 + y^2, xy)
        } h;
        struct {
            float2 hp01[kR1][kOut];    // horizontal pass of the first two partials
            float hp2[kR1][kOut];      // and of the third
            float at[kR2][kR2];        // next item's target alpha (prefetched during the last pass)
        } st;
    } b;
};

// The SSIM window: 11-tap Gaussian, sigma = 1.5, normalised
// (exp(-(i - 5)^2 / 4.5) / sum, evaluated in double, rounded to float).
__device__ constexpr float kWin[11] = {0x1.0d956cp-10f, 0x1.f1fe02p-8f, 0x1.26eb18p-5f, 0x1.bff0fep-4f,
                                       0x1.b43c40p-3f,  0x1.106560p-2f, 0x1.b43c40p-3f, 0x1.bff0fep-4f,
                                       0x1.26eb18p-5f,  0x1.f1fe02p-8f, 0x1.0d956cp-10f};

// N outputs of the 11-tap window from N + 10 consecutive inputs read once
// (stride STRIDE floats apart).
template <int N, int STRIDE>
__device__ __forceinline__ void strip11(const float* src, float out[N]) {
    float in[N + 10];
#pragma unroll
    for (int k = 0; k < N + 10; ++k) in[k] = src[k * STRIDE];
#pragma unroll
    for (int o = 0; o < N; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 11; ++j) acc += kWin[j] * in[o + j];
        out[o] = acc;
    }
}

// The same for two interleaved maps at once (STRIDE in float2): each tap is
// one packed two-lane FMA (fma.rn.f32x2, each lane rounded as a scalar FMA),
// so the results equal two strip11 calls.
template <int N, int STRIDE>
__device__ __forceinline__ void strip11x2(const float2* src, float2 out[N]) {
    float2 in[N + 10];
#pragma unroll
    for (int k = 0; k < N + 10; ++k) in[k] = src[k * STRIDE];
#pragma unroll
    for (int o = 0; o < N; ++o) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 11; ++j) acc = __ffma2_rn(make_float2(kWin[j], kWin[j]), in[o + j], acc);
        out[o] = acc;
    }
}

// The same for two maps at separate addresses (two rows of one map).
template <int N, int STRIDE>
__device__ __forceinline__ void strip11x2(const float* a, const float* b, float2 out[N]) {
    float2 in[N + 10];
#pragma unroll
    for (int k = 0; k < N + 10; ++k) in[k] = make_float2(a[k * STRIDE], b[k * STRIDE]);
#pragma unroll
    for (int o = 0; o < N; ++o) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 11; ++j) acc = __ffma2_rn(make_float2(kWin[j], kWin[j]), in[o + j], acc);
        out[o] = acc;
    }
}

// Edge of the blocks whose agreement the match pre-pass records (per channel).
constexpr int kBlk = 16;

__host__ __device__ inline int blocks_of(const gsfit_camera& c) {
    return ((c.width + kBlk - 1) / kBlk) * ((c.height + kBlk - 1) / kBlk);
}

// Loss workspace: the per-view accumulators, then (when the workspace holds
// them) one agreement byte per 16-pixel block and channel.
__host__ __device__ inline size_t flags_offset(int n_views) { return ((size_t)n_views * 3 * sizeof(float) + 255) & ~(size_t)255; }

// The view owning work item `item`, the index of that view's first item and
// of its first 16-pixel block.
__device__ __forceinline__ void locate_item(const gsfit_camera* __restrict__ cams, int item, int& v, int& first,
                                            int& boff) {
    v = 0;
    first = 0;
    boff = 0;
    for (;; ++v) {
        const int k = 3 * ((cams[v].width + kOut - 1) / kOut) * ((cams[v].height + kOut - 1) / kOut);
        if (item < first + k) break;
        first += k;
        boff += blocks_of(cams[v]);
    }
}

// Whether a view's rows can be read in 16-byte pieces: width and pixel offset
// multiples of 4 (so every channel plane and row starts 16-byte aligned, and
// a 4-pixel piece starting at a multiple of 4 lies wholly inside or outside
// the image), and the three input arrays 16-byte aligned.
__device__ __forceinline__ bool rows16(const gsfit_camera& cam, bool bases16) {
    return bases16 && (cam.width & 3) == 0 && (cam.pixel_offset & 3) == 0;
}

// The match pre-pass: for every 16 x 16 pixel block and colour channel,
// whether the render equals the target composited over the background
// (the same expression as the loss kernel's) at every pixel of the block. One
// warp per block (lane l: row l / 2, eight pixels from column 8 (l mod 2)),
// the loads coalesced in 64-byte row pieces, 16-byte loads where the view's
// rows allow them (all seven maps of a piece in flight together); the whole
// images are read once.
__global__ void __launch_bounds__(256) match_kernel(const gsfit_camera* __restrict__ cams_g, int n_views,
                                                    const float* __restrict__ rgb, const float* __restrict__ t_rgb,
                                                    const float* __restrict__ t_alpha, const float* __restrict__ bg,
                                                    uint8_t* __restrict__ flags, size_t flag_bytes) {
    int n_blocks = 0;
    for (int v = 0; v < n_views; ++v) n_blocks += blocks_of(cams_g[v]);
    if (3 * (size_t)n_blocks > flag_bytes) return;  // no room: the loss kernel then tests every item itself
    const bool bases16 = ((reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(t_rgb) |
                           reinterpret_cast<uintptr_t>(t_alpha)) & 15u) == 0;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x / 32);
    for (int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); b < n_blocks; b += warps) {
        int v = 0, base = 0;
        for (;; ++v) {  // the block's view (warp-uniform)
            const int nb = blocks_of(cams_g[v]);
            if (b < base + nb) break;
            base += nb;
        }
        const gsfit_camera& cam = cams_g[v];
        const int W = cam.width, H = cam.height, nbx = (W + kBlk - 1) / kBlk;
        const int local = b - base, by = local / nbx, bx = local - by * nbx;
        const int gy = by * kBlk + (lane >> 1), gx0 = bx * kBlk + (lane & 1) * 8;
        const long long P = (long long)W * H;
        const float* X = rgb + 3ll * cam.pixel_offset;
        const float* Yt = t_rgb + 3ll * cam.pixel_offset;
        const float* At = t_alpha + cam.pixel_offset;
        bool d0 = false, d1 = false, d2 = false;
        const float b0 = bg[3 * v + 0], b1 = bg[3 * v + 1], b2 = bg[3 * v + 2];
        auto same4 = [](float4 x, float4 t, float4 a, float b) {
            return x.x == t.x + (1.0f - a.x) * b && x.y == t.y + (1.0f - a.y) * b && x.z == t.z + (1.0f - a.z) * b &&
                   x.w == t.w + (1.0f - a.w) * b;
        };
        if (gy < H && rows16(cam, bases16)) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gx = gx0 + 4 * h;
                if (gx >= W) break;  // W is a multiple of 4: a piece lies wholly inside or outside
                const long long q = (long long)gy * W + gx;
                const float4 a = __ldg(reinterpret_cast<const float4*>(At + q));
                const float4 t0 = __ldg(reinterpret_cast<const float4*>(Yt + q));
                const float4 t1 = __ldg(reinterpret_cast<const float4*>(Yt + P + q));
                const float4 t2 = __ldg(reinterpret_cast<const float4*>(Yt + 2 * P + q));
                const float4 x0 = __ldg(reinterpret_cast<const float4*>(X + q));
                const float4 x1 = __ldg(reinterpret_cast<const float4*>(X + P + q));
                const float4 x2 = __ldg(reinterpret_cast<const float4*>(X + 2 * P + q));
                d0 = d0 || !same4(x0, t0, a, b0);
                d1 = d1 || !same4(x1, t1, a, b1);
                d2 = d2 || !same4(x2, t2, a, b2);
            }
        } else if (gy < H) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gx = gx0 + e;
                if (gx >= W) break;
                const long long q = (long long)gy * W + gx;
                const float a = __ldg(At + q);
                const float y0 = __ldg(Yt + q) + (1.0f - a) * b0;
                const float y1 = __ldg(Yt + P + q) + (1.0f - a) * b1;
                const float y2 = __ldg(Yt + 2 * P + q) + (1.0f - a) * b2;
                d0 = d0 || !(__ldg(X + q) == y0);
                d1 = d1 || !(__ldg(X + P + q) == y1);
                d2 = d2 || !(__ldg(X + 2 * P + q) == y2);
            }
        }
        const bool a0 = __any_sync(0xffffffffu, d0), a1 = __any_sync(0xffffffffu, d1),
                   a2 = __any_sync(0xffffffffu, d2);
        if (lane == 0) {
            flags[3 * (size_t)b + 0] = a0 ? 0 : 1;
            flags[3 * (size_t)b + 1] = a1 ? 0 : 1;
            flags[3 * (size_t)b + 2] = a2 ? 0 : 1;
        }
    }
}

// Whether the 16-pixel blocks that cover work item `it`'s 52 x 52 input
// region (4 x 4 of them: columns ox - 16 .. ox + 47) all agree in its channel,
// blocks outside the image counting as agreeing (block-uniform; one barrier).
// Then the item's exact agreement test would pass too, and it needs no loads.
__device__ __forceinline__ bool blocks_agree(const uint8_t* __restrict__ flags, const gsfit_camera* __restrict__ cams_g,
                                             int it, int v, int first, int boff) {
    const gsfit_camera& cam = cams_g[v];
    const int W = cam.width, H = cam.height;
    const int txn = (W + kOut - 1) / kOut, nbx = (W + kBlk - 1) / kBlk, nby = (H + kBlk - 1) / kBlk;
    const int local = it - first, ch = local % 3, tile = local / 3;
    const int oy = (tile / txn) * kOut, ox = (tile % txn) * kOut;
    bool differ = false;
    if (threadIdx.x < 16) {
        const int bx = ((ox - 10) >> 4) + (threadIdx.x & 3), by = ((oy - 10) >> 4) + (threadIdx.x >> 2);
        if (bx >= 0 && bx < nbx && by >= 0 && by < nby)
            differ = flags[3 * ((size_t)boff + (size_t)by * nbx + bx) + ch] == 0;
    }
    return __syncthreads_or(differ) == 0;
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool ok) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int n = ok ? 4 : 0;  // source size 0: zero fill, nothing read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}

// Starts the copies of an item's render, target and target alpha over its
// 52 x 52 input region (zero outside the image) into x, y and at.
__device__ __forceinline__ void prefetch_item(LossSmem& S, const gsfit_camera* __restrict__ cams_g, int item, int v,
                                              int first, const float* __restrict__ rgb,
                                              const float* __restrict__ t_rgb, const float* __restrict__ t_alpha) {
    const gsfit_camera& cam = cams_g[v];
    const int W = cam.width, H = cam.height;
    const int txn = (W + kOut - 1) / kOut;
    const int local = item - first;
    const int ch = local % 3, tile = local / 3;
    const int oy = (tile / txn) * kOut, ox = (tile % txn) * kOut;
    const long long P = (long long)W * H;
    const float* X = rgb + 3ll * cam.pixel_offset + ch * P;
    const float* Yt = t_rgb + 3ll * cam.pixel_offset + ch * P;
    const float* At = t_alpha + cam.pixel_offset;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool interior = ox >= 10 && oy >= 10 && ox + kOut + 10 <= W && oy + kOut + 10 <= H;
    // warp w copies rows w, w + 8, ...; lane l columns l and l + 32
    if (interior) {
        // the region lies inside the image: no bounds, row pointers advanced by 8 rows
        const long long row0 = (long long)(oy - 10 + wid) * W + (ox - 10);
        const long long step = (long long)(kLossThreads / 32) * W;
        const float* xr = X + row0;
        const float* yr = Yt + row0;
        const float* ar = At + row0;
        for (int r = wid; r < kR2; r += kLossThreads / 32, xr += step, yr += step, ar += step) {
#pragma unroll
            for (int c = lane; c < kR2; c += 32) {
                cp_async4(&S.a.xy[r][c].x, xr + c, true);
                cp_async4(&S.a.xy[r][c].y, yr + c, true);
                cp_async4(&S.b.st.at[r][c], ar + c, true);
            }
        }
    } else {
        for (int r = wid; r < kR2; r += kLossThreads / 32) {
            const int gy = oy - 10 + r;
            for (int c = lane; c < kR2; c += 32) {
                const int gx = ox - 10 + c;
                const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const long long q = ok ? (long long)gy * W + gx : 0;
                cp_async4(&S.a.xy[r][c].x, X + q, ok);
                cp_async4(&S.a.xy[r][c].y, Yt + q, ok);
                cp_async4(&S.b.st.at[r][c], At + q, ok);
            }
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Adds the block's sums of the three loss terms to a view's accumulators
// (sum |x - y|, sum SSIM, sum |A - A*|); ends with a barrier.
__device__ __forceinline__ void block_loss_sums(float (&s_red)[3][kLossThreads / 32], float* acc_v, float l1,
                                                float ssim_sum, float la) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    ssim_sum = warp_sum(ssim_sum);
    l1 = warp_sum(l1);
    la = warp_sum(la);
    if (lane == 0) {
        s_red[0][wid] = l1;
        s_red[1][wid] = ssim_sum;
        s_red[2][wid] = la;
    }
    __syncthreads();
    if (tid < 3) {
        float sacc = 0.f;
        for (int k = 0; k < kLossThreads / 32; ++k) sacc += s_red[tid][k];
        atomicAdd(&acc_v[tid], sacc);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kLossThreads, kLossCtasPerSm) loss_kernel(
    const gsfit_camera* __restrict__ cams_g, int n_views, const float* __restrict__ rgb,
    const float* __restrict__ alpha, const float* __restrict__ t_rgb, const float* __restrict__ t_alpha,
    const float* __restrict__ bg, float lambda, float* __restrict__ g_rgb, float* __restrict__ g_alpha,
    float* __restrict__ acc /* 3 per view: sum|x-y|, sum SSIM, sum|A-A*| */,
    const uint8_t* __restrict__ flags /* the match pre-pass's, or null */, size_t flag_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LossSmem& S = *reinterpret_cast<LossSmem*>(smem_raw);
    __shared__ float s_red[3][kLossThreads / 32];
    __shared__ int s_view, s_first, s_boff;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int n_items = 0, n_blocks = 0;
    for (int v = 0; v < n_views; ++v) {
        n_items += 3 * ((cams_g[v].width + kOut - 1) / kOut) * ((cams_g[v].height + kOut - 1) / kOut);
        n_blocks += blocks_of(cams_g[v]);
    }
    if (3 * (size_t)n_blocks > flag_bytes) flags = nullptr;  // as the pre-pass decided

    // The inputs of each item are copied asynchronously while the previous
    // item finishes (its last pass leaves the input region and most of the
    // horizontal-pass buffer free).
    if (tid == 0 && (int)blockIdx.x < n_items) locate_item(cams_g, blockIdx.x, s_view, s_first, s_boff);
    __syncthreads();
    const bool bases16 = ((reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(t_rgb) |
                           reinterpret_cast<uintptr_t>(t_alpha)) & 15u) == 0;
    // An item is started (its inputs copied, where they are copied) only if
    // the match flags do not already settle it.
    auto start_item = [&](int it) -> bool {  // block-uniform; the item's location in s_view, s_first, s_boff
        if (it >= n_items) return false;
        if (flags && blocks_agree(flags, cams_g, it, s_view, s_first, s_boff)) return true;
        if (!rows16(cams_g[s_view], bases16)) prefetch_item(S, cams_g, it, s_view, s_first, rgb, t_rgb, t_alpha);
        return false;
    };
    bool settled = start_item(blockIdx.x);  // the current item agrees by the match flags
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int v = s_view;
        const int first = s_first;
        const int next = item + gridDim.x;
        __syncthreads();  // every thread has read this item's view
        if (tid == 0 && next < n_items) locate_item(cams_g, next, s_view, s_first, s_boff);
        const gsfit_camera& cam = cams_g[v];
        const int W = cam.width, H = cam.height;
        const int txn = (W + kOut - 1) / kOut;
        const int local = item - first;
        const int ch = local % 3;
        const int tile = local / 3;
        const int oy = (tile / txn) * kOut, ox = (tile % txn) * kOut;
        const long long P = (long long)W * H;
        const float* At = t_alpha + cam.pixel_offset;
        const float bgc = bg[3 * v + ch];
        const float inv3PV = 1.0f / (3.0f * (float)P * (float)n_views);

        // 1. the inputs: target composited over the background (zero outside
        //    the image); and whether render and target agree over the whole
        //    region
        bool differ = false;
        if (settled) {
            // nothing to load
        } else if (rows16(cam, bases16)) {
            // 16-byte loads into registers, the composite and the comparison
            // there, then the region into shared memory as (x, y) pairs: the
            // window is read 2 columns wider on each side (columns ox - 12 ..
            // ox + 43, 14 pieces of 4 per row) so that every piece is aligned;
            // comparing the extra columns only makes the agreement test
            // stricter. No copy into shared memory is pending for such a view
            // (none is started for it).
            constexpr int kPC = 14, kPN = kR2 * kPC;
            static_assert(4 * kPC == kR2 + 4, "pieces cover the region and 2 columns each side");
            const float* X = rgb + 3ll * cam.pixel_offset + ch * P;
            const float* Yt = t_rgb + 3ll * cam.pixel_offset + ch * P;
            for (int k = tid; k < kPN; k += kLossThreads) {
                const int r = k / kPC, pq = k - r * kPC;
                const int gy = oy - 10 + r, gx = ox - 12 + 4 * pq;
                const bool ok = gy >= 0 && gy < H && gx >= 0 && gx < W;
                float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), yv = xv;
                if (ok) {
                    const long long o = (long long)gy * W + gx;
                    xv = __ldg(reinterpret_cast<const float4*>(X + o));
                    const float4 t = __ldg(reinterpret_cast<const float4*>(Yt + o));
                    const float4 a = __ldg(reinterpret_cast<const float4*>(At + o));
                    yv = make_float4(t.x + (1.0f - a.x) * bgc, t.y + (1.0f - a.y) * bgc, t.z + (1.0f - a.z) * bgc,
                                     t.w + (1.0f - a.w) * bgc);
                }
                differ = differ || !(xv.x == yv.x) || !(xv.y == yv.y) || !(xv.z == yv.z) || !(xv.w == yv.w);
                const int c = 4 * pq - 2;  // shared-memory column of the piece's first pixel
                if (c >= 0) *reinterpret_cast<float4*>(&S.a.xy[r][c]) = make_float4(xv.x, yv.x, xv.y, yv.y);
                if (c + 2 < kR2) *reinterpret_cast<float4*>(&S.a.xy[r][c + 2]) = make_float4(xv.z, yv.z, xv.w, yv.w);
            }
        } else {
            // the copies started while the previous item finished
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();  // block-uniform branch: the view decides it
            if (ox >= 10 && oy >= 10 && ox + kOut + 10 <= W && oy + kOut + 10 <= H) {  // the region lies inside
                float2* xyf = &S.a.xy[0][0];
                const float* af = &S.b.st.at[0][0];
                for (int k = tid; k < kR2 * kR2; k += kLossThreads) {
                    const float yv = xyf[k].y + (1.0f - af[k]) * bgc;
                    xyf[k].y = yv;
                    differ = differ || !(xyf[k].x == yv);
                }
            } else {
                for (int r = wid; r < kR2; r += kLossThreads / 32) {
                    const int gy = oy - 10 + r;
                    for (int c = lane; c < kR2; c += 32) {
                        const int gx = ox - 10 + c;
                        const bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
                        const float yv = ok ? S.a.xy[r][c].y + (1.0f - S.b.st.at[r][c]) * bgc : 0.0f;
                        S.a.xy[r][c].y = yv;
                        differ = differ || !(S.a.xy[r][c].x == yv);
                    }
                }
            }
        }
        // Render and target equal over the whole input region (the tile and
        // the 10-pixel reach of a gradient: windows of radius 5 around pixels
        // within 5): every window in play has x = y, so SSIM 1 there, and
        // zero gradient (SSIM(., y) is largest at y, and the L1 subgradient
        // at 0 is 0). The item then needs no stencil: the exact results are
        // written directly (the stencil would give them up to rounding). In a
        // periphery batch this is every item inside the background around
        // the splats, where both are the background colour bit for bit.
        if (__syncthreads_or(differ) == 0) {  // (also: the next item's location is visible)
            // the input region is no longer read: start the next item
            settled = start_item(next);
            // the item's sums: L1 0, SSIM 1 per pixel (added as a count) and, in channel 0, the alpha
            // term (a warp sum and one atomic per warp): no block reduction
            float la = 0.f;
            const int cidx = tid % kOut, r0 = (tid / kOut) * 4;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int gy = oy + r0 + o, gx = ox + cidx;
                if (gy >= H || gx >= W) continue;
                const long long q = (long long)gy * W + gx;
                g_rgb[3ll * cam.pixel_offset + ch * P + q] = 0.0f;
                if (ch == 0) {
                    const float da = alpha[cam.pixel_offset + q] - At[q];
                    la += fabsf(da);
                    g_alpha[cam.pixel_offset + q] =
                        (da > 0.f ? 1.f : (da < 0.f ? -1.f : 0.f)) / ((float)P * (float)n_views);
                }
            }
            if (ch == 0) {
                la = warp_sum(la);
                if (lane == 0 && la != 0.f) atomicAdd(&acc[3 * v + 2], la);
            }
            if (tid == 0) atomicAdd(&acc[3 * v + 1], (float)(min(kOut, W - ox) * min(kOut, H - oy)));
            continue;
        }
        // 2. horizontal pass of x, y, x^2 + y^2, xy: 52 rows x 42 columns in
        //    strips of 3 (728 strips: 95% of the threads busy over three
        //    rounds); and a copy of the output pixels
        constexpr int kHS = 3, kHN = kR1 / kHS;
        for (int k = tid; k < kR2 * kHN; k += kLossThreads) {
            const int r = k / kHN, c0 = (k - r * kHN) * kHS;
            // packed pairs: (x, y) and (x^2 + y^2, xy), one two-lane FMA per tap and pair
            float2 xy2[kHS + 10], qp[kHS + 10];
#pragma unroll
            for (int j = 0; j < kHS + 10; ++j) {
                xy2[j] = S.a.xy[r][c0 + j];
                qp[j] = make_float2(xy2[j].x * xy2[j].x + xy2[j].y * xy2[j].y, xy2[j].x * xy2[j].y);
            }
#pragma unroll
            for (int o = 0; o < kHS; ++o) {
                float2 ab = make_float2(0.f, 0.f), ce = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 11; ++j) {
                    const float2 wj = make_float2(kWin[j], kWin[j]);
                    ab = __ffma2_rn(wj, xy2[o + j], ab);
                    ce = __ffma2_rn(wj, qp[o + j], ce);
                }
                S.b.h.h01[r][c0 + o] = ab;
                S.b.h.h23[r][c0 + o] = ce;
            }
        }
        __syncthreads();
        // 3. vertical pass (strips of 7 rows: 252 strips, one round) straight
        //    into SSIM and its partials w.r.t. (mu_x, E[x^2], E[xy]) on the
        //    42 x 42 region; zero outside the image (those windows do not exist)
        constexpr int kVS = 7, kVN = kR1 / kVS;
        float ssim_sum = 0.f;
        for (int k = tid; k < kR1 * kVN; k += kLossThreads) {
            const int cidx = k % kR1, r0 = (k / kR1) * kVS;
            float2 m01[kVS], m23[kVS];  // (mu_x, mu_y), (E[x^2 + y^2], E[xy])
            strip11x2<kVS, kR1>(&S.b.h.h01[r0][cidx], m01);
            strip11x2<kVS, kR1>(&S.b.h.h23[r0][cidx], m23);
            const int gx = ox - 5 + cidx;
#pragma unroll
            for (int o = 0; o < kVS; ++o) {
                const int r = r0 + o, gy = oy - 5 + r;
                float dmu = 0.f, dxx = 0.f, dxy = 0.f;
                if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                    const float mx = m01[o].x, my = m01[o].y;
                    const float m2 = mx * mx + my * my;
                    const float sxy = m23[o].y - mx * my;
                    const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
                    // B2 = var x + var y + C2 = E[x^2 + y^2] - mu_x^2 - mu_y^2 + C2
                    const float B1 = m2 + kC1, B2 = m23[o].x - m2 + kC2;
                    // B1 >= C1 and B2 ~ >= C2: the hardware reciprocal (within 2 ulp)
                    const float iB1 = __fdividef(1.0f, B1), iB2 = __fdividef(1.0f, B2);
                    const float iB = iB1 * iB2;
                    const float ss = A1 * A2 * iB;
                    dmu = 2.f * my * (A2 - A1) * iB - 2.f * mx * ss * (iB1 - iB2);
                    dxx = -ss * iB2;
                    dxy = 2.f * A1 * iB;
                    if (r >= 5 && r < 5 + kOut && cidx >= 5 && cidx < 5 + kOut) ssim_sum += ss;
                }
                S.a.part.p01[r][cidx] = make_float2(dmu, dxx);
                S.a.part.p2[r][cidx] = dxy;
            }
        }
        __syncthreads();
        // 4. horizontal pass of the partials: 42 rows x 32 columns in strips of 8,
        //    the first two partials packed (168 strips), the third two rows at a
        //    time (84 strips): 252 strips, one round of the block
        static_assert(kR1 % 2 == 0 && kR1 * 4 + (kR1 / 2) * 4 <= kLossThreads, "one strip per thread");
        if (tid < kR1 * 4) {
            const int r = tid >> 2, c0 = (tid & 3) * 8;
            float2 out[8];
            strip11x2<8, 1>(&S.a.part.p01[r][c0], out);
#pragma unroll
            for (int o = 0; o < 8; ++o) S.b.st.hp01[r][c0 + o] = out[o];
        } else if (tid < kR1 * 4 + (kR1 / 2) * 4) {
            const int rem = tid - kR1 * 4;
            const int r = (rem >> 2) * 2, c0 = (rem & 3) * 8;
            float2 out[8];
            strip11x2<8, 1>(&S.a.part.p2[r][c0], &S.a.part.p2[r + 1][c0], out);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                S.b.st.hp2[r][c0 + o] = out[o].x;
                S.b.st.hp2[r + 1][c0 + o] = out[o].y;
            }
        }
        __syncthreads();
        // the input region and the alpha buffer are free: start the next item
        settled = start_item(next);
        // 5. vertical pass onto the tile (a 4-pixel column strip per thread) and
        //    the gradient
        float l1 = 0.f, la = 0.f;
        {
            const int cidx = tid % kOut, r0 = (tid / kOut) * 4;  // 32 columns x 8 strips = 256
            float2 cmx[4];  // (dSSIM/dmu_x, dSSIM/dE[x^2]) convolved back
            float cxy[4];
            strip11x2<4, kOut>(&S.b.st.hp01[r0][cidx], cmx);
            strip11<4, kOut>(&S.b.st.hp2[r0][cidx], cxy);
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int r = r0 + o;
                const int gy = oy + r, gx = ox + cidx;
                if (gy >= H || gx >= W) continue;
                // the output pixel's render and composited target, again from global memory
                // (the same operations as step 1, so bit-identical; the item's region is in L2)
                const long long q0 = (long long)gy * W + gx;
                const float xv = __ldg(rgb + 3ll * cam.pixel_offset + ch * P + q0);
                const float yv = __ldg(t_rgb + 3ll * cam.pixel_offset + ch * P + q0) + (1.0f - __ldg(At + q0)) * bgc;
                const float dssim = cmx[o].x + 2.f * xv * cmx[o].y + yv * cxy[o];
                const float diff = xv - yv;
                const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
                l1 += fabsf(diff);
                const long long q = (long long)gy * W + gx;
                g_rgb[3ll * cam.pixel_offset + ch * P + q] = ((1.0f - lambda) * sg - lambda * dssim) * inv3PV;
                if (ch == 0) {
                    const float da = alpha[cam.pixel_offset + q] - At[q];
                    la += fabsf(da);
                    g_alpha[cam.pixel_offset + q] =
                        (da > 0.f ? 1.f : (da < 0.f ? -1.f : 0.f)) / ((float)P * (float)n_views);
                }
            }
        }
        block_loss_sums(s_red, acc + 3 * v, l1, ssim_sum, la);
    }
}

__global__ void loss_finalize_kernel(const gsfit_camera* __restrict__ cams, int n_views, float lambda,
                                     const float* __restrict__ acc, float* __restrict__ loss_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float L = 0.f;
    for (int v = 0; v < n_views; ++v) {
        const float P = (float)cams[v].width * (float)cams[v].height;
        const float l1 = acc[3 * v] / (3.f * P), ssim = acc[3 * v + 1] / (3.f * P), la = acc[3 * v + 2] / P;
        L += (1.f - lambda) * l1 + lambda * (1.f - ssim) + la;
    }
    *loss_out = L / (float)n_views;
}

// The loss kernel's dynamic shared memory opt-in, shared by both entry
// points: once per device and context.
ContextOnce g_loss_smem_once;
int enable_loss_smem() { return opt_in_smem(g_loss_smem_once, loss_kernel, sizeof(LossSmem)); }

}  // namespace

}  // namespace gsfit

using namespace gsfit;

extern "C" size_t gsfit_loss_workspace_size(const gsfit_camera* cams, int32_t n_views) {
    if (n_views < 1 || n_views > GSFIT_MAX_VIEWS) return 0;
    if (!cams) return (size_t)(3 * n_views) * sizeof(float);  // the accumulators only
    size_t blocks = 0;
    for (int v = 0; v < n_views; ++v) blocks += (size_t)blocks_of(cams[v]);
    return flags_offset(n_views) + 3 * blocks;
}

extern "C" int gsfit_loss(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
                          const float* target_rgb, const float* target_alpha, const float* bg, float lambda,
                          float* dL_drgb, float* dL_dalpha, float* loss_out, void* ws, size_t ws_bytes,
                          cudaStream_t stream) {
    if (!cams || n_views < 1 || n_views > GSFIT_MAX_VIEWS || !rgb || !alpha || !target_rgb || !target_alpha ||
        !bg || !dL_drgb || !dL_dalpha || !ws || ws_bytes < gsfit_loss_workspace_size(nullptr, n_views))
        return GSFIT_ERR_INVALID_ARG;
    const size_t smem = sizeof(LossSmem);
    const int rc = enable_loss_smem();
    if (rc != GSFIT_OK) return rc;
    int dev = 0, sms = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* acc = static_cast<float*>(ws);
    GSFIT_CUDA_CHECK(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * n_views, stream));
    // the match flags, where the workspace holds them (the kernels check the size)
    uint8_t* flags = nullptr;
    size_t flag_bytes = 0;
    if (ws_bytes > flags_offset(n_views)) {
        flags = static_cast<uint8_t*>(ws) + flags_offset(n_views);
        flag_bytes = ws_bytes - flags_offset(n_views);
        match_kernel<<<8 * sms, 256, 0, stream>>>(cams, n_views, rgb, target_rgb, target_alpha, bg, flags, flag_bytes);
        GSFIT_LAUNCH_CHECK();
    }
    loss_kernel<<<kLossCtasPerSm * sms, kLossThreads, smem, stream>>>(cams, n_views, rgb, alpha, target_rgb, target_alpha, bg,
                                                         lambda, dL_drgb, dL_dalpha, acc, flags, flag_bytes);
    GSFIT_LAUNCH_CHECK();
    if (loss_out) {
        loss_finalize_kernel<<<1, 32, 0, stream>>>(cams, n_views, lambda, acc, loss_out);
        GSFIT_LAUNCH_CHECK();
    }
    return GSFIT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant (no counterpart in the paper): the same kernels with
// the per-view accumulators in a fixed device array of this library, for
// callers that cannot allocate device memory (a real-time frame loop, a
// plug-in whose host application owns all device allocations).
// ---------------------------------------------------------------------------

namespace gsfit {
namespace {

constexpr int kNoAllocMaxViews = GSFIT_MAX_VIEWS;

// 3 accumulators per view: sum|x - y|, sum SSIM, sum|A - A*| (3 KB). Host code
// must not use this name as a pointer: it is a host-side stand-in; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) float g_loss_noalloc_acc[3 * kNoAllocMaxViews];

// Device address of g_loss_noalloc_acc in the current device's current
// context. Looked up (cudaGetSymbolAddress, with that device current) on the
// first call in each context and cached under the context's id: a context
// reset reloads the library's module, and the next call looks the address up
// again instead of writing through a stale one.
struct NoAllocAddress {
    ContextOnce once;
    float* addr[64] = {};
};
NoAllocAddress g_noalloc;

int noalloc_acc_address(float** out) {
    int dev = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GSFIT_ERR_CUDA;
    const int rc = run_once_per_context(g_noalloc.once, [&] {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_loss_noalloc_acc) != cudaSuccess || !p) return GSFIT_ERR_CUDA;
        g_noalloc.addr[dev] = static_cast<float*>(p);
        return GSFIT_OK;
    });
    if (rc != GSFIT_OK) return rc;
    std::lock_guard<std::mutex> lock(g_noalloc.once.m);
    *out = g_noalloc.addr[dev];
    return *out ? GSFIT_OK : GSFIT_ERR_CUDA;
}

}  // namespace
}  // namespace gsfit

extern "C" int gsfit_loss_noalloc(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
                                  const float* target_rgb, const float* target_alpha, const float* bg,
                                  float lambda, float* dL_drgb, float* dL_dalpha, float* loss_out,
                                  cudaStream_t stream) {
    if (!cams || n_views < 1 || n_views > kNoAllocMaxViews || !rgb || !alpha || !target_rgb || !target_alpha ||
        !bg || !dL_drgb || !dL_dalpha)
        return GSFIT_ERR_INVALID_ARG;
    float* acc = nullptr;
    int rc = noalloc_acc_address(&acc);
    if (rc != GSFIT_OK) return rc;
    const size_t smem = sizeof(LossSmem);
    rc = enable_loss_smem();
    if (rc != GSFIT_OK) return rc;
    int dev = 0, sms = 0;
    GSFIT_CUDA_CHECK(cudaGetDevice(&dev));
    GSFIT_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the array keeps the previous call's sums: clear this call's part first
    GSFIT_CUDA_CHECK(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * n_views, stream));
    loss_kernel<<<kLossCtasPerSm * sms, kLossThreads, smem, stream>>>(cams, n_views, rgb, alpha, target_rgb, target_alpha, bg,
                                                         lambda, dL_drgb, dL_dalpha, acc, nullptr, 0);
    GSFIT_LAUNCH_CHECK();
    if (loss_out) {
        loss_finalize_kernel<<<1, 32, 0, stream>>>(cams, n_views, lambda, acc, loss_out);
        GSFIT_LAUNCH_CHECK();
    }
    return GSFIT_OK;
}
