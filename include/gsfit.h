/*
 * gsfit.h -- C ABI of the Gaussian-Splatting periphery fit step (sm_103a).
 *
 * The peripheral model of the paper (Section 4.2) is a 3D Gaussian Splatting
 * model fitted to posed path-traced views with alpha supervision and
 * randomised backgrounds; one fit iteration is
 *
 *   gsfit_project     EWA projection of every Gaussian into every view, with
 *                     spherical-harmonic colour
 *   gsfit_bin_sort    (tile | depth) key generation, radix sort, tile ranges
 *   gsfit_render_fwd  front-to-back alpha compositing per pixel
 *   gsfit_loss        L1 + 0.2 D-SSIM on colour + L1 on alpha, and dL/dimage
 *   gsfit_render_bwd  back-to-front adjoint of the compositing, then the
 *                     adjoint of the projection, summed over views
 *   gsfit_adam_step   Adam update of all parameters
 *
 * (gsfit_blend_bwd followed by gsfit_project_bwd_adam runs the last two
 * stages with the projection adjoint and Adam fused into one pass.)
 *
 * The paper does not write the splatting math out; every convention is that
 * of standard 3DGS (Kerbl et al. 2023, EWA splatting after Zwicker et al.
 * 2001) and is stated at each call below.
 *
 * Conventions shared by every call
 *   - All data pointers are DEVICE pointers owned by the caller unless the
 *     argument says "host". The library allocates nothing; scratch space is
 *     passed in as a workspace whose size a *_workspace_size query returns.
 *   - Every call is asynchronous on the given stream and performs no
 *     host/device synchronisation, so a whole iteration can be captured in a
 *     CUDA graph. Return values report argument errors and launch errors
 *     (GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA) only; conditions found on the
 *     device (instance capacity exceeded, a bounded wait that ran out) are
 *     written to the caller's int32 status word, read after a synchronise.
 *   - Sizes: n Gaussians (n < 2^31), V views (1 <= V <= GSFIT_MAX_VIEWS),
 *     tile size B = 8 or 16 pixels (GSFIT_TILE = 16 is the default; see
 *     gsfit_camera and gsfit_render_opts).
 *
 * Data layouts
 *   Gaussian parameters (and their gradients, and the Adam moments) are
 *   float4 planes: plane p of Gaussian i is at float4 index p * n + i.
 *     plane 0          (mean x, mean y, mean z, opacity logit)
 *     plane 1          rotation quaternion (w, x, y, z), normalised on use
 *     plane 2          (log scale x, log scale y, log scale z, 0)
 *     planes 3 ..      SH coefficients k = 0 .. K-1 (K = (degree+1)^2),
 *                      flattened as k0.r k0.g k0.b k1.r ..., four per plane,
 *                      zero padded: gsfit_num_planes(degree) planes in all.
 *   Images of a view batch are packed view after view. View v starts at
 *   pixel pixel_offset_v (gsfit_camera.pixel_offset); colour images hold
 *   three H x W planes (r, g, b) per view starting at 3 * pixel_offset_v;
 *   single-channel images (alpha, T_final, n_contrib) one plane per view.
 *   Pixel (x, y) of a view samples the image plane at integer (x, y); a
 *   centred camera has cx = W/2 - 0.5, cy = H/2 - 0.5.
 */
#ifndef GSFIT_H_
#define GSFIT_H_

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSFIT_ABI_VERSION 10
#define GSFIT_MAX_VIEWS 256
#define GSFIT_TILE 16
/* Words of a tile_order buffer for total_tiles tiles (gsfit_bin_sort):
 * the heavy-first permutation, the number of non-empty tiles, each tile's
 * furthest contributor and the adjoint's launch order. */
#define GSFIT_TILE_ORDER_WORDS(total_tiles) (3 * (total_tiles) + 2)

/* Return and status codes. */
#define GSFIT_OK 0
#define GSFIT_ERR_INVALID_ARG (-1)
#define GSFIT_ERR_CAPACITY (-2)  /* more (Gaussian, tile) pairs than capacity  */
#define GSFIT_ERR_CUDA (-3)      /* a CUDA launch or runtime call failed        */
#define GSFIT_ERR_TIMEOUT (-4)   /* a bounded device-side wait ran out          */
#define GSFIT_ERR_NONFINITE (-5) /* a non-finite parameter gradient was produced */

/*
 * One pinhole camera: 128 bytes, identical on host and device.
 * viewmat is world -> camera, row-major 3 x 4 [R | t]; camera axes are
 * +x right, +y down, +z forward, so p_cam = R p_world + t. campos is the
 * camera centre in world space (-R^T t), used for the SH view direction.
 * A Gaussian is culled in a view when its float32 depth is <= near_plane
 * (3DGS uses 0.2). tile_offset is the global id of the view's first tile and
 * pixel_offset its first pixel in the packed images; tile is the tile edge
 * B the batch is laid out for (8 or 16, the same in every view of a batch);
 * gsfit_camera_layout fills all three. The projection's tile rectangles and
 * the binning use B; the compositing calls are told B by their options and
 * check it against the cameras.
 */
typedef struct gsfit_camera {
    float viewmat[12];
    float campos[3];
    float fx, fy, cx, cy;
    float near_plane;
    int32_t width, height;
    int32_t tile_offset;
    int32_t pixel_offset;
    int32_t tile;         /* tile edge in pixels, 8 or 16 (any other value reads as 16) */
    int32_t reserved[7];
} gsfit_camera;

/* Storage of the Gaussian features the projection reads (see gsfit_gaussians). */
#define GSFIT_FEATURES_F32 0   /* every plane read from params                    */
#define GSFIT_FEATURES_F16 1   /* SH planes 3.. read from an IEEE half copy         */
#define GSFIT_FEATURES_BF16 2  /* SH planes 3.. read from a bfloat16 copy           */

/*
 * A Gaussian set (device, float4 planes as described above).
 * Mixed-precision form (the precision pattern of the fitting loop, Section
 * 4.2's fitted 3DGS model with 16-bit colour storage): with feature_dtype
 * GSFIT_FEATURES_F16 or GSFIT_FEATURES_BF16 the projection and its adjoint
 * read the SH coefficient planes 3 .. num_planes-1 from `features`, a 16-bit
 * copy laid out as those planes with 4 x 16 bits per entry (plane p of
 * Gaussian i at 8-byte index (p - 3) * n + i, (num_planes - 3) * n * 8
 * bytes). Planes 0-2 (means and opacity logit, rotation, log-scales) are
 * always read in float32 from params: rounding them would move splat
 * footprints and with them the compositing's skip / clamp / stop decisions,
 * while the SH coefficients (48 of the 59 values of a degree-3 Gaussian) only
 * tint colours. Everything computed from the features (colour, transmittance,
 * gradients) stays float32, and the gradients are those of the function of
 * the 16-bit values. The copy is written by gsfit_features_refresh and kept
 * current by gsfit_adam_step.
 */
typedef struct gsfit_gaussians {
    const float* params;    /* gsfit_num_planes(sh_degree) * n float4 (float32 master copy) */
    int32_t n;
    int32_t sh_degree;      /* 0 .. 3 */
    const void* features;   /* 16-bit copy of the SH planes 3.., or null with GSFIT_FEATURES_F32 */
    int32_t feature_dtype;  /* GSFIT_FEATURES_* */
    int32_t reserved;
} gsfit_gaussians;

/*
 * Per-(view, Gaussian) projected records, index r = v * n + i (device).
 *   xyd[r]     float4 (u, v, depth, radius): pixel-space centre, float32
 *              camera-space depth, integer pixel radius ceil(3 sqrt(lambda_max))
 *              stored as a float; radius 0 marks a culled record.
 *   conic[r]   float4 (a', b', c', opacity): inverse 2D covariance and the
 *              activated opacity; power = -1/2 (a' dx^2 + c' dy^2) - b' dx dy.
 *   rgb[r]     float4 (r, g, b, mask): colour after the clamp at 0; mask holds
 *              (clamped r) + 2 (clamped g) + 4 (clamped b) as a float.
 *   tiles[r]   number of tiles the record's rectangle covers (0 if culled).
 */
typedef struct gsfit_proj {
    float* xyd;
    float* conic;
    float* rgb;
    uint32_t* tiles;
} gsfit_proj;

/* Number of float4 parameter planes for an SH degree (3 + ceil(3K/4)). */
int gsfit_num_planes(int sh_degree);

/* ABI version, for a loader to check against GSFIT_ABI_VERSION. */
int gsfit_abi_version(void);

/* Human-readable name of a return / status code (static string). */
const char* gsfit_status_string(int code);

/*
 * Host helper: fills tile_offset, pixel_offset and tile of V HOST cameras for
 * tile size `tile` (8 or 16), laying views out in order, and returns the batch
 * totals. Returns GSFIT_ERR_INVALID_ARG for another tile size, a
 * non-positive image size or V out of range.
 */
int gsfit_camera_layout(gsfit_camera* cams_host, int n_views, int tile, int32_t* total_tiles,
                        int64_t* total_pixels);

/*
 * Host helper, view selection for continual refinement (Section 4.2, Eq. 1):
 * a new view joins the training set only if, for every view i already in
 * it, ||pos_new - pos_i|| > delta_pos or view_new . view_i < cos(theta_view)
 * (the paper uses delta_pos = 0.05 and theta_view = 5 degrees). pos: camera
 * centres, 3 floats each; dir: viewing directions, 3 floats each, normalised
 * here (a zero direction is invalid). HOST pointers; n_set may be 0 (an
 * empty set accepts any view).
 * Returns 1 (novel: add the view), 0 (redundant), GSFIT_ERR_INVALID_ARG for
 * null pointers with n_set > 0, a zero direction or a negative n_set.
 */
int gsfit_view_is_novel(const float* pos_new, const float* dir_new, const float* pos_set, const float* dir_set,
                        int32_t n_set, float delta_pos, float cos_theta);

/*
 * gsfit_project -- EWA projection with SH colour: the first stage of
 * rendering the peripheral 3DGS model that Section 4.2 fits to the
 * path-traced views (alpha training, randomised backgrounds); the splatting
 * conventions are those of 3DGS, which the paper inherits.
 *   Per (view v, Gaussian i): s = exp(log_scale), q normalised, opacity =
 *   sigmoid(logit), Sigma = R(q) diag(s^2) R(q)^T; t = R_v mu + t_v; culled
 *   if t_z <= near. Sigma' = J R_v Sigma R_v^T J^T + 0.3 I with the EWA
 *   Jacobian J at t (t_x/t_z, t_y/t_z clamped to +-1.3 tan(fov/2) inside J);
 *   conic = Sigma'^-1 (culled if det <= 0); radius = ceil(3 sqrt(lambda_max)),
 *   lambda_max = m + sqrt(max(0.1, m^2 - det)), m = (a + c)/2; centre
 *   u = fx t_x/t_z + cx, v = fy t_y/t_z + cy; tile rectangle
 *   [floor((u-r)/B), floor((u+r+B-1)/B)) in x (likewise y) clamped to the
 *   view; colour = max(0, sum_k Y_k(dir) k_k + 0.5), dir = normalise(mu -
 *   campos), real SH with Condon-Shortley phase, m = -l..l per band.
 *   Depth, centre and rectangle are computed with a fixed order of correctly
 *   rounded float32 operations (no contraction) so that keys are
 *   reproducible. A Gaussian with non-finite parameters is culled in every
 *   view (a NaN position, scale or rotation fails the depth or determinant
 *   test; a non-finite opacity or colour is culled explicitly), so it neither
 *   renders nor receives gradients and the rest of the set is unaffected.
 * Arguments: g (device params), cams (device, n_views records laid out by
 *   gsfit_camera_layout), out (device arrays of n_views * n records each).
 * Errors: GSFIT_ERR_INVALID_ARG for null pointers, n <= 0, bad degree or V;
 *   GSFIT_ERR_CUDA if the launch fails.
 */
int gsfit_project(const gsfit_gaussians* g, const gsfit_camera* cams, int32_t n_views, gsfit_proj* out,
                  cudaStream_t stream);

/*
 * Workspace bytes gsfit_bin_sort needs for n_views * n projected records,
 * `capacity` (Gaussian, tile) pairs and `total_tiles` tiles.
 */
size_t gsfit_bin_sort_workspace_size(int64_t n_records, int64_t capacity, int32_t total_tiles);

/*
 * gsfit_bin_sort -- tile binning of the projected records: the depth-ordered
 * per-tile lists from which the peripheral 3DGS model of Section 4.2 is
 * composited (3DGS's tile rasteriser ordering).
 *   Exclusive scan of tiles[]; for every record with tiles > 0 and every
 *   tile (row-major) of its rectangle, one pair key = (global tile id << 32)
 *   | float32 bits of depth, value = Gaussian index i; the pairs sorted by
 *   key, stably with respect to record order (the result is the unique order
 *   by (key, view, Gaussian index); computed as a stable radix sort of the
 *   binned records by depth, emission of their pairs in that order, and a
 *   stable radix sort of the pairs on the tile-id bits); and per global tile t the
 *   range ranges[2t], ranges[2t+1] = [first, last+1) of its pairs, [0, 0)
 *   if empty.
 * Arguments: proj/cams as for gsfit_project (n Gaussians, n_views views,
 *   total_tiles = sum over views of tiles); ws/ws_bytes: device workspace of
 *   at least gsfit_bin_sort_workspace_size bytes (contents need not be
 *   initialised); keys (uint64) and vals (uint32): device, `capacity`
 *   entries each, sorted output; keys may be null when the caller needs only
 *   the lists (vals) and ranges, which are then the same: the tile-bit passes
 *   then sort 32-bit tile ids with the values (8 bytes per pair and pass
 *   instead of 12); n_instances: device uint32, receives the
 *   number of pairs (also when it exceeds capacity); ranges: device uint32,
 *   2 * total_tiles entries; status: device int32, set to GSFIT_ERR_CAPACITY
 *   when the pairs exceed capacity (nothing is then emitted and every range
 *   is empty) and to GSFIT_ERR_TIMEOUT if a bounded wait of the sort ran out;
 *   it is not cleared by this call. tile_order (device uint32,
 *   GSFIT_TILE_ORDER_WORDS(total_tiles) entries, may be null), with
 *   T = total_tiles: entries [0, T) a permutation of the tiles, most work
 *   first (bucketed by quarter octaves of the furthest contributor the last
 *   gsfit_render_fwd recorded in this buffer, capped at the list length, or
 *   of the list length where it recorded none; any order within a bucket),
 *   so the non-empty tiles lead; entry T the number of non-empty tiles;
 *   entries [T + 1, 2T + 1) each tile's furthest contributor, set to zero
 *   here and written by gsfit_render_fwd; entries [2T + 1, 3T + 1) the
 *   adjoint's launch order and entry 3T + 1 the non-empty count again,
 *   written by gsfit_blend_bwd. The forward pass
 *   launches tiles in the heavy-first order, so the longest lists start first
 *   and do not form the tail of the grid; the CTAs of empty tiles leave at
 *   once (the forward pass writing the background first).
 * Errors: GSFIT_ERR_INVALID_ARG (null pointers, sizes, workspace too small,
 *   capacity >= 2^30, n_views * n >= 2^32), GSFIT_ERR_CUDA.
 */
int gsfit_bin_sort(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                   int32_t total_tiles, void* ws, size_t ws_bytes, uint64_t* keys, uint32_t* vals,
                   int64_t capacity, uint32_t* n_instances, uint32_t* ranges, uint32_t* tile_order,
                   int32_t* status, cudaStream_t stream);

/*
 * Options of the compositing calls: the tunables of the batched launch.
 *   tile:  the tile edge the cameras were laid out for by gsfit_camera_layout
 *          (8 or 16); a launch whose cameras say otherwise writes
 *          GSFIT_ERR_INVALID_ARG to the status word and does nothing.
 *   batch: records per shared-memory slot of the producer ring (the number of
 *          Gaussians staged per batch) of the forward passes (gsfit_render_fwd,
 *          gsfit_render_importance): 64, 128 or 256. The ring holds 8 slots of
 *          64 entries or 4 slots of 128 or 256.
 *   batch_bwd: the same for the blend adjoint (gsfit_blend_bwd,
 *          gsfit_render_bwd): 64, 128 or 256. The results do not depend on
 *          either depth beyond the order of the adjoint's atomic sums.
 *   exp_half2: 1 evaluates exp(power) of each (pixel, Gaussian) pair in
 *          packed half precision (f16x2: the forward pass takes two Gaussians
 *          of a pixel per instruction), the half2-exponent option of the
 *          mixed-precision form; 0 (default) in float32. The quadratic form,
 *          alpha, T, colours and gradients stay float32. Each pair's value
 *          depends on its own power only, so the adjoint, which must be called
 *          with the same setting as the forward pass it follows, takes the
 *          same skip and stop decisions. Against the float32 form the result
 *          moves by the half-precision rounding of power and exp (up to about
 *          2^-10 relative in the weight) and by the threshold decisions that
 *          rounding moves.
 * A null pointer or a 0 field selects the default (tile 16, batch 128,
 * batch_bwd 64, float32 exponent).
 * gsfit_render_autotune measures the batch depths on a caller's workload.
 */
typedef struct gsfit_render_opts {
    int32_t tile;
    int32_t batch;
    int32_t exp_half2;
    int32_t batch_bwd;
} gsfit_render_opts;

/*
 * gsfit_render_fwd -- front-to-back compositing (3DGS, with the alpha output
 * used for alpha supervision, Section 4.2).
 *   For each pixel, over its tile's sorted pairs: power as in gsfit_proj,
 *   skipped if power > 0; alpha = min(0.99, opacity exp(power)), skipped if
 *   alpha < 1/255; stop before a Gaussian that would take T below 1e-4;
 *   C = sum c alpha T + T_N bg_v, A = 1 - T_N. n_contrib is one past the
 *   list position (within the tile's range) of the last blended Gaussian.
 * Arguments: bg: device float, 3 per view; rgb: 3 * total_pixels floats,
 *   alpha, T_final: total_pixels floats, n_contrib: total_pixels uint32
 *   (device). vals/ranges/tile_order from gsfit_bin_sort (tile_order may be
 *   null: tiles in id order, every tile composited in full; the results do
 *   not depend on the order). With a tile_order the call also records each
 *   non-empty tile's furthest contributor (the largest n_contrib of its
 *   pixels) in it, from which the adjoint orders its launch; compositing
 *   calls that share a tile_order must therefore not run concurrently.
 *   status: device int32 or null. The kernel's warps hand records to each
 *   other through shared-memory barriers whose waits are bounded (about a
 *   second); if one runs out (which a correct launch never does) the kernel
 *   writes GSFIT_ERR_TIMEOUT there, the affected tiles' outputs are
 *   incomplete, and later tiles of this and the other compositing calls that
 *   see that value skip their work. With a null status a timeout goes
 *   unreported. opts: see gsfit_render_opts (may be null).
 * Errors: GSFIT_ERR_INVALID_ARG (also for unsupported options), GSFIT_ERR_CUDA;
 *   GSFIT_ERR_TIMEOUT, or GSFIT_ERR_INVALID_ARG for a tile mismatch, on the
 *   device, through status.
 */
int gsfit_render_fwd(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                     int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges, uint32_t* tile_order,
                     const float* bg, float* rgb, float* alpha, float* T_final, uint32_t* n_contrib,
                     const gsfit_render_opts* opts, int32_t* status, cudaStream_t stream);

/*
 * gsfit_loss -- photometric loss of a view batch and its gradient.
 *   Target colour y = target_rgb + (1 - target_alpha) bg_v (premultiplied
 *   target composited over the render's background). Per view
 *   L_v = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y))
 *         + mean|A - target_alpha|,  L = (1/V) sum_v L_v,
 *   SSIM with an 11 x 11 Gaussian window (sigma 1.5), zero padding, C1 =
 *   0.01^2, C2 = 0.03^2, averaged over channels and pixels (3DGS). Writes
 *   dL/drgb and dL/dalpha (the L1 subgradient at 0 is 0) and, if loss_out is
 *   not null, the scalar loss (device float). Where render and composited
 *   target are equal (in float32) over a 32 x 32 output tile and the 10
 *   pixels around it, the windows there have SSIM 1 and the colour gradient
 *   is zero: such tiles are written directly, without the SSIM stencil.
 *   With a workspace of gsfit_loss_workspace_size(cams, n_views) bytes a
 *   pre-pass first records, per 16 x 16 pixel block and channel, whether
 *   render and target agree over the block, and tiles whose surrounding
 *   blocks all agree are settled without loading their inputs; with the
 *   accumulators only (gsfit_loss_workspace_size(NULL, n_views) bytes) every
 *   tile tests its own region. The results are the same.
 * Arguments: images in the packed layout (device); ws: device workspace of at
 *   least gsfit_loss_workspace_size(NULL, n_views) bytes; cams of the size
 *   query: the host copy of the camera table (as gsfit_camera_layout fills
 *   it), or NULL for the accumulators only.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
size_t gsfit_loss_workspace_size(const gsfit_camera* cams, int32_t n_views);
int gsfit_loss(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
               const float* target_rgb, const float* target_alpha, const float* bg, float lambda,
               float* dL_drgb, float* dL_dalpha, float* loss_out, void* ws, size_t ws_bytes,
               cudaStream_t stream);

/*
 * gsfit_loss_noalloc -- gsfit_loss for callers that cannot allocate device
 * memory. The paper has no counterpart; this is a deployment convenience.
 *   Some callers must not call cudaMalloc on their path: a real-time frame
 *   loop, where an allocation can synchronise the device and stall the frame,
 *   or a plug-in inside an application that owns every device allocation
 *   (its own pool and accounting). They still pass inputs and outputs, but no
 *   workspace: the per-view accumulators live in a fixed array inside this
 *   library (3 * GSFIT_MAX_VIEWS floats = 3 KB per GPU, held by every GPU that
 *   loads the library until the process exits).
 *   Same arguments and results as gsfit_loss without ws / ws_bytes.
 *   n_views above GSFIT_MAX_VIEWS (256) is rejected with
 *   GSFIT_ERR_INVALID_ARG. The first call on a device looks up the array's
 *   device address (with that device current) and caches it; make that first
 *   call before any stream capture. Every call clears the accumulators it uses
 *   before using them. All calls share the one array: calls whose executions
 *   overlap on the GPU (different streams, or graphs replayed concurrently)
 *   race on it and may return wrong loss values; serialise them.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA (including a failed address
 *   lookup).
 */
int gsfit_loss_noalloc(const gsfit_camera* cams, int32_t n_views, const float* rgb, const float* alpha,
                       const float* target_rgb, const float* target_alpha, const float* bg, float lambda,
                       float* dL_drgb, float* dL_dalpha, float* loss_out, cudaStream_t stream);

/*
 * gsfit_render_bwd -- adjoint of gsfit_render_fwd and gsfit_project: the
 * gradient step of fitting the peripheral 3DGS model to the training views
 * (Section 4.2: alpha training against the views' alpha, randomised
 * backgrounds).
 *   Per pixel, back to front from n_contrib - 1, recovering T_i = T_{i+1} /
 *   (1 - alpha_i) from T_final (no per-(pixel, Gaussian) state is stored):
 *   dC/dc_i = alpha_i T_i; dC/dalpha_i = T_i c_i - (S_i + T_N bg) / (1 -
 *   alpha_i) with S_i the colour composited behind i; dA/dalpha_i = T_N /
 *   (1 - alpha_i); dalpha/d(opacity, power) = 0 where the 0.99 clamp is
 *   active. Per-(view, Gaussian) gradients of (u, v, conic, opacity, rgb) are
 *   accumulated with atomics in grad2d (per lane where few lanes of a warp
 *   blend the Gaussian, else reduced over the warp first), then chained
 *   through the projection (zero derivative where the frustum guard or the
 *   colour clamp is active) and summed over views into `grads`.
 * Arguments: g: the Gaussians that were projected; dL_drgb/dL_dalpha in the
 *   image layout; grad2d: device workspace of 16 floats per record
 *   (n_views * n * 64 bytes) that must be zero before the first call; this
 *   call leaves it zero again. grads: device, same layout as the parameters,
 *   fully overwritten (no zeroing needed). opts, status: as for
 *   gsfit_render_fwd.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA; on the device, through
 *   status: GSFIT_ERR_TIMEOUT, and GSFIT_ERR_NONFINITE when a parameter
 *   gradient written to `grads` is not finite (a non-finite image,
 *   cotangent or 2D gradient upstream; the gradients are still written, and
 *   an earlier error in status is kept).
 */
int gsfit_render_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                     int32_t n_views, int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                     uint32_t* tile_order, const float* bg, const float* T_final, const uint32_t* n_contrib,
                     const float* dL_drgb, const float* dL_dalpha, float* grad2d, float* grads,
                     const gsfit_render_opts* opts, int32_t* status, cudaStream_t stream);

/*
 * gsfit_blend_bwd / gsfit_project_bwd -- the two halves of gsfit_render_bwd,
 * for callers that schedule them separately (gsfit_render_bwd = blend, then
 * project). gsfit_blend_bwd accumulates the per-(view, Gaussian) gradients of
 * (u, v, conic, opacity, rgb) into grad2d (which must be zero on entry);
 * gsfit_project_bwd chains them through the projection, sums them over views
 * into `grads` (fully overwritten) and zeroes grad2d again. Arguments as for
 * gsfit_render_bwd (opts and status only for gsfit_blend_bwd). With a
 * tile_order, gsfit_blend_bwd first orders the non-empty tiles by the
 * furthest contributor the forward pass recorded (descending, in quarter
 * octaves; a tile's adjoint walks its list up to that position), into the
 * order's last region, and launches them in that order, which ends the
 * launch with short tiles (list length predicts a tile's adjoint work less
 * well); the results do not depend on the order. Errors:
 * GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA; GSFIT_ERR_TIMEOUT on the device,
 * through status.
 */
int gsfit_blend_bwd(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                    int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges, uint32_t* tile_order,
                    const float* bg, const float* T_final, const uint32_t* n_contrib, const float* dL_drgb,
                    const float* dL_dalpha, float* grad2d, const gsfit_render_opts* opts, int32_t* status,
                    cudaStream_t stream);
int gsfit_project_bwd(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views,
                      float* grad2d, float* grads, cudaStream_t stream);

/*
 * gsfit_project_bwd_adam -- gsfit_project_bwd and gsfit_adam_step in one
 * pass over the Gaussians: the fit iteration's last two stages (the fitted
 * 3DGS model of Section 4.2, with its Adam rates and restarts as in
 * gsfit_adam_step). Each Gaussian's gradient, summed over the views, goes
 * straight into its Adam update instead of through a gradient buffer, which
 * saves writing and reading n_planes * n float4 and the gradient buffer
 * itself. The gradient equals gsfit_project_bwd's up to rounding (the
 * compiler may contract the chain's products and sums into fused
 * multiply-adds differently in the two kernels); given that gradient, the
 * update equals gsfit_adam_step's bit for bit. On GB300 the two separate
 * calls are faster for the fit step: the fused pass runs at the projection
 * adjoint's register budget, with too few warps in flight for Adam's
 * stream.
 * Arguments: g, proj, cams, n_views, grad2d as for gsfit_project_bwd (grad2d
 *   zeroed again); g->params and, with a 16-bit feature type, g->features
 *   are UPDATED IN PLACE, so both must be writable device memory; grads:
 *   device, n_planes * n float4, or null; when given, it also receives the
 *   gradient as gsfit_project_bwd writes it. m, v, lr, beta1, beta2, eps,
 *   step: as for gsfit_adam_step, with n_planes = gsfit_num_planes
 *   (g->sh_degree); *step is incremented on the device afterwards. status:
 *   device int32 or null; a non-finite gradient sets GSFIT_ERR_NONFINITE
 *   there, as gsfit_render_bwd does. params, grads, m and v are distinct
 *   buffers.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_project_bwd_adam(const gsfit_gaussians* g, const gsfit_proj* proj, const gsfit_camera* cams,
                           int32_t n_views, float* grad2d, float* grads, float* m, float* v, const float* lr,
                           float beta1, float beta2, float eps, int32_t* step, int32_t* status, cudaStream_t stream);

/*
 * gsfit_render_count -- diagnostic: the number of blended (pixel, Gaussian)
 * pairs of a forward pass (pairs with list position < n_contrib, power <= 0
 * and alpha >= 1/255), i.e. the pairs whose adjoint gsfit_blend_bwd evaluates.
 * Adds the count to *count (device uint64; the caller zeroes it). Not part of
 * a fit iteration; used to state achieved arithmetic rates.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_render_count(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                       int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges, const uint32_t* tile_order,
                       const uint32_t* n_contrib, unsigned long long* count,
                       const gsfit_render_opts* opts, cudaStream_t stream);

/*
 * gsfit_render_autotune -- the batching pattern's tuner: picks the batch
 * depth of the compositing kernels for one laid-out view batch by measuring
 * each supported depth (64, 128, 256) on the caller's buffers: `reps`
 * forward launches and `reps` adjoint launches each, timed with CUDA events on
 * `stream`. The adjoint accumulates into grad2d, which this call zeroes again
 * at the end. Unlike the other calls it synchronises the stream (it measures)
 * and must not be captured in a graph. Writes to *best (tile = `tile`) the
 * depth with the smallest forward time as batch and the one with the smallest
 * adjoint time as batch_bwd, and, if times_ms (host) is
 * not null, the mean times per depth: 2 floats per depth (forward, adjoint),
 * depths in increasing order. The tile size itself changes the projection
 * and the binning too; callers compare tile sizes on the whole iteration.
 * Arguments as for gsfit_render_fwd and gsfit_blend_bwd; tile 8 or 16; reps
 * >= 1.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_render_autotune(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                          int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                          uint32_t* tile_order, const float* bg, float* rgb, float* alpha, float* T_final,
                          uint32_t* n_contrib, const float* dL_drgb, const float* dL_dalpha, float* grad2d,
                          int32_t tile, int32_t reps, gsfit_render_opts* best, float* times_ms, int32_t* status,
                          cudaStream_t stream);

/*
 * gsfit_adam_step -- Adam (Kingma & Ba) with bias correction over all
 * parameter planes (the paper raises the scale, opacity and colour rates by
 * about 50% and resets the state on restart, Section 4.2; both are choices of
 * the caller's lr table and moment buffers).
 *   m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
 *   p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 *   with t = *step + 1; *step is incremented on the device afterwards.
 *   Parameters and moments are float32. With feature_dtype
 *   GSFIT_FEATURES_F16 / GSFIT_FEATURES_BF16 the same pass also writes the
 *   updated SH planes 3.. to `features`, rounded to nearest even (the layout
 *   of gsfit_gaussians.features).
 * Arguments: params, grads, m, v: n_planes * n float4 (device); lr: HOST
 *   array of 4 * n_planes floats, the rate of each component of each plane
 *   (0 freezes it); step: device int32 count of completed steps; features:
 *   device, (n_planes - 3) * n * 8 bytes, or null with GSFIT_FEATURES_F32.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, int32_t n_planes,
                    const float* lr, float beta1, float beta2, float eps, int32_t* step, void* features,
                    int32_t feature_dtype, cudaStream_t stream);

/*
 * gsfit_features_refresh -- writes the 16-bit feature copy of
 * gsfit_gaussians.features from the float32 parameters (the SH planes 3 ..
 * n_planes-1, rounded to nearest even): after the parameters were set or
 * changed outside gsfit_adam_step.
 * Arguments: params: n_planes * n float4 (device); features: device,
 *   (n_planes - 3) * n * 8 bytes; feature_dtype GSFIT_FEATURES_F16 or
 *   GSFIT_FEATURES_BF16.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_features_refresh(const float* params, int32_t n, int32_t n_planes, void* features, int32_t feature_dtype,
                           cudaStream_t stream);

/*
 * gsfit_render_importance -- gsfit_render_fwd that also accumulates each
 * Gaussian's importance: the sum over the batch's pixels of its blend weight
 * alpha_i T_i (the weight its colour gets in C). Per pixel these weights sum
 * to 1 - T_N, so the importances of a batch sum to its total alpha. Used for
 * the simplification step of the abbreviated regeneration (Section 4.2).
 * Arguments as for gsfit_render_fwd; importance: device, n floats, added to
 * (the caller zeroes it before the first batch).
 * Errors: as for gsfit_render_fwd.
 */
int gsfit_render_importance(const gsfit_proj* proj, const gsfit_camera* cams, int32_t n_views, int32_t n,
                            int32_t total_tiles, const uint32_t* vals, const uint32_t* ranges,
                            uint32_t* tile_order, const float* bg, float* rgb, float* alpha, float* T_final,
                            uint32_t* n_contrib, float* importance, const gsfit_render_opts* opts, int32_t* status,
                            cudaStream_t stream);

/*
 * gsfit_simplify -- keeps the `keep` most important Gaussians (the
 * simplification of the abbreviated regeneration, Section 4.2; importance as
 * gsfit_render_importance accumulates it). The threshold is the keep-th
 * largest importance; every Gaussian at or above it is kept, so ties at the
 * threshold may keep a few more; with n <= keep every Gaussian is kept.
 * Kept Gaussians are written in index order: plane p of the m-th kept one at
 * float4 index p * n + m of params_out (the input's plane stride n); the count
 * goes to *n_out (device). Negative or NaN importance counts as 0.
 * Arguments: params: n_planes * n float4 (device); importance: n floats;
 *   params_out: n_planes * n float4, distinct from params; ws: device workspace
 *   of gsfit_simplify_workspace_size(n) bytes, 16-byte aligned.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
size_t gsfit_simplify_workspace_size(int32_t n);
int gsfit_simplify(const float* params, int32_t n, int32_t n_planes, const float* importance, int32_t keep,
                   float* params_out, uint32_t* n_out, void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * gsfit_first_hit -- first-hit point-cloud seeding (Section 4.1): rays cast
 * toward the CT volume from the given viewpoints; each ray keeps its first
 * significant hit, the first point where the transfer function's opacity of
 * the (trilinearly interpolated) volume reaches alpha_min.
 *   Volume: int16 HU values hu[z][y][x], nx * ny * nz voxels of edge `voxel`,
 *   corner at `origin` (HOST 3 floats); voxel centres at origin + (i + 0.5)
 *   voxel; samples between centres interpolate trilinearly, clamped at the
 *   faces. Transfer function: n_knots (<= 8) HOST rows (HU, r, g, b, alpha),
 *   HU increasing; linear between knots, clamped outside.
 *   Rays: per view, a rays_x x rays_y grid over the image (ray (i, j) through
 *   pixel ((i + 0.5) W / rays_x - 0.5, (j + 0.5) H / rays_y - 0.5) of the
 *   pinhole camera), from the camera centre, clipped to the volume's box and
 *   sampled every `step` (world units) from the entry point; at the first
 *   sample whose opacity reaches alpha_min the crossing is refined by 12
 *   bisection steps between it and the previous sample (or the entry point).
 *   Ray r = (v * rays_y + j) * rays_x + i writes points[r] = (x, y, z, 1) at
 *   the hit, (0, 0, 0, 0) for a miss, and colour[r] = the transfer function's
 *   (r, g, b, alpha) there (0 for a miss). The paper colours the points by
 *   path tracing; that is not part of this library.
 * Arguments: hu, cams (n_views cameras), points, colour: device; points and
 *   colour 4 * n_views * rays_x * rays_y floats, 16-byte aligned; step > 0.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_first_hit(const int16_t* hu, int32_t nx, int32_t ny, int32_t nz, const float* origin, float voxel,
                    const float* tf_knots, int32_t n_knots, const gsfit_camera* cams, int32_t n_views,
                    int32_t rays_x, int32_t rays_y, float step, float alpha_min, float* points, float* colour,
                    cudaStream_t stream);

/*
 * gsfit_reproject -- depth-guided reprojection of a foveal image to a newer
 * head pose (Section 4.3, Eqs. 2-4), as a headless kernel writing device
 * buffers instead of deforming a mesh in a viewer shader.
 *   Per source pixel (x, y), uv = ((x + 0.5) / W, (y + 0.5) / H) (v grows
 *   with the row index) and its linear depth d (world distance along the ray):
 *     p_far   = (P_old V_old)^-1 (2uv - 1, 1, 1)^T / w   (the far plane, z_ndc = 1)
 *     p_world = pos_old + d (p_far - pos_old) / |p_far - pos_old|
 *     p'_clip = P_new V_new p_world                      (written to clip)
 *   The image is then carried to the new view point by point: the source
 *   pixel lands on the output pixel nearest to its projected centre
 *   ((ndc + 1) / 2 * size - 0.5 rounded half up) if p'_clip.w > 0 and that pixel
 *   exists; among sources landing on one output pixel the smallest w (nearest
 *   to the new camera) wins, ties to the lower source index. Output pixels no
 *   source reaches (disocclusions, which the viewer fills from the Gaussian
 *   model) get covered = 0 and colour 0. Pixels with depth <= 0 or not
 *   finite are skipped (clip = 0).
 * Arguments: rgb: 3 planes of W*H floats; depth: W*H floats (device);
 *   inv_pv_old (the inverse of P_old V_old), pv_new: HOST row-major 4x4
 *   float matrices acting on column vectors; pos_old: HOST 3 floats; clip:
 *   device 4*W*H floats or null; zbuf: device workspace of out_w*out_h
 *   uint64 (contents need not be initialised); out_rgb: 3 planes of
 *   out_w*out_h floats; covered: out_w*out_h bytes (device).
 * Errors: GSFIT_ERR_INVALID_ARG (null pointers, non-positive sizes, clip
 *   not 16-byte aligned, zbuf not 8-byte aligned), GSFIT_ERR_CUDA.
 */
int gsfit_reproject(const float* rgb, const float* depth, int32_t width, int32_t height, const float* inv_pv_old,
                    const float* pos_old, const float* pv_new, int32_t out_w, int32_t out_h, float* clip,
                    unsigned long long* zbuf, float* out_rgb, uint8_t* covered, cudaStream_t stream);

/*
 * Diagnostics of the bounded device waits (failure detection without a GPU
 * fault). gsfit_selftest_wait_timeout launches threads that wait, as the
 * compositing kernels' pixel and producer warps do, on a shared-memory
 * mbarrier phase that never completes, giving up after limit_cycles clock
 * cycles; gsfit_selftest_lookback_timeout polls, as the radix pass's
 * decoupled look-back does, a device word (a zeroed uint32 the caller
 * provides) that nothing sets, giving up after `polls` polls of ~100 ns.
 * Both write GSFIT_ERR_TIMEOUT to *status (device int32) and return; the
 * context stays usable.
 * Errors: GSFIT_ERR_INVALID_ARG, GSFIT_ERR_CUDA.
 */
int gsfit_selftest_wait_timeout(int64_t limit_cycles, int32_t* status, cudaStream_t stream);
int gsfit_selftest_lookback_timeout(uint32_t* word, int32_t polls, int32_t* status, cudaStream_t stream);

/*
 * Diagnostic of the compositing kernels' shared exponent (Section 4.2, the
 * 3DGS splat power -1/2 d^T Sigma'^-1 d). The forward pass evaluates it with
 * scalar operations on records as stored; the adjoint with packed two-lane
 * operations on records rearranged in shared memory. Both must round
 * identically, or the adjoint would not replay the forward's skip and stop
 * decisions. For each i < n: conic[4i..4i+3] = (a', b', c', opacity) and
 * pix[4i..4i+3] = (px, py, u, v); out[2i] is the forward's power and
 * out[2i+1] the adjoint's. All pointers are device float arrays owned by
 * the caller; n >= 0.
 * Errors: GSFIT_ERR_INVALID_ARG (null pointers with n > 0, n < 0),
 *   GSFIT_ERR_CUDA.
 */
int gsfit_selftest_splat_power(const float* conic, const float* pix, int32_t n, float* out, cudaStream_t stream);

/*
 * gsfit_selftest_alu_rate -- diagnostic with no counterpart in the paper: the
 * arithmetic-rate microbenchmark behind the compositing kernels' roofline.
 * Launches `blocks` CTAs of 256 threads; each thread runs 8 independent
 * chains of `iters` operations of one kind: 0 = fma.rn.f32 (2 FLOP), 1 =
 * fma.rn.f32x2 (two FMAs, 4 FLOP), 2 = ex2.approx.f32 (one MUFU operation).
 * The caller times the launch (CUDA events on `stream`) and divides
 * blocks * 256 * 8 * iters operations by the time.
 * Arguments: sink: device, blocks * 256 floats (written, meaningless).
 * Errors: GSFIT_ERR_INVALID_ARG (kind not 0-2, blocks or iters < 1, null
 *   sink), GSFIT_ERR_CUDA.
 */
int gsfit_selftest_alu_rate(int32_t kind, int32_t blocks, int32_t iters, float* sink, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSFIT_H_ */
