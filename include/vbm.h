/*
 * vbm.h -- C ABI of the GB300 (sm_103a) implementation of Variable Basis
 * Mapping (VBM, arXiv 2601.09417): volume -> wavelet coefficients -> 3D
 * Gaussians (Sec. 4.2-4.3) and the image-space fine-tuning step that refines
 * them (Sec. 4.4).
 *
 * Conventions for every entry point
 *   - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never frees them.  Pointers without the prefix are host pointers, read
 *     during the call only.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated
 *     otherwise; no call synchronises the device except vbm_build (which
 *     copies a few counters to the host), vbm_plan_check and vbm_plan_create.
 *   - Argument errors are detected on the host before any launch and return
 *     VBM_ERR_ARG; a failing CUDA runtime call returns VBM_ERR_CUDA.  The
 *     message of the last failure on the calling thread is vbm_last_error().
 *   - Device-side conditions (pair-buffer overflow, non-finite gradients)
 *     are recorded in device words and reported by vbm_plan_check /
 *     the d_nonfinite counter of vbm_adam, never by faulting or trapping.
 *   - Floating point is IEEE float32 on the device unless stated.
 *
 * Data layouts
 *   Gaussian parameters  float P[14][stride], row r, column i = Gaussian i:
 *     rows 0-2 mean (world units = voxels), 3-5 log standard deviation,
 *     6-9 rotation quaternion (w, x, y, z; normalised inside), 10 opacity
 *     logit (opacity = sigmoid), 11-13 colour (r, g, b; no activation).
 *     Gradients use the same layout.
 *   Volume               float F[nz][ny][nx] (x fastest); voxel (i, j, k)
 *     covers [i, i+1) x [j, j+1) x [k, k+1) in world units.
 *   Images               float img[V][3][H][W] (planar RGB), alpha / per-pixel
 *     state [V][H][W]; DVR output float rgba[V][4][H][W].  Pixel (i, j) has
 *     its centre at (i + 1/2, j + 1/2).
 */
#ifndef VBM_H
#define VBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VBM_API __attribute__((visibility("default")))
#else
#define VBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VBM_OK = 0,
    VBM_ERR_ARG = 1,       /* invalid argument, detected on the host           */
    VBM_ERR_CAPACITY = 2,  /* a buffer sized by the caller or plan is too small */
    VBM_ERR_CUDA = 3,      /* a CUDA runtime call failed                        */
    VBM_ERR_TIMEOUT = 4,   /* reserved: a bounded device wait gave up           */
    VBM_ERR_NOMEM = 5,     /* device allocation failed                          */
    VBM_ERR_NUMERIC = 6    /* non-finite values were detected                   */
} vbm_status;

/* Message of the last failed call on this thread ("" if none).  Thread-local,
 * valid until the next failing call on the same thread. */
VBM_API const char *vbm_last_error(void);

/* ABI version (major * 100 + minor). */
VBM_API int vbm_version(void);

/* ------------------------------------------------------------------ types */

/* Pinhole camera, 80 bytes.  World -> camera p_c = R p + t (R row-major);
 * camera frame x right, y down, z forward; image point (fx x/z + cx,
 * fy y/z + cy).  znear: Gaussians with camera z <= znear are culled. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float znear;
    int32_t width, height;
    int32_t pad;
} vbm_camera;

/* Piecewise-linear transfer function (Sec. 3): n_knots in [2, 16], x
 * ascending in [0, 1]; the scalar is clamped to [0, 1] and each RGBA channel
 * interpolated linearly between knots (constant outside). */
typedef struct {
    int32_t n_knots;
    float x[16];
    float rgba[16][4];
} vbm_tf;

/* One transition-bank entry (Sec. 4.2, Eq. 13-18): canonical Gaussian of
 * subband (j, o) with o[d] = 0 (L) or 1 (H) along x, y, z.  u: centroid in
 * grid units relative to the impulse position 2^j k (Eq. 14); cov: xx yy zz
 * xy xz yz (Eq. 14); w: ridge energy weight (Eq. 17); log_scale / quat: the
 * splat shape with R diag(exp(2 log_scale)) R^T = cov. */
typedef struct {
    int32_t j;
    int32_t o[3];
    double u[3];
    double cov[6];
    double w;
    float log_scale[3];
    float quat[4];
} vbm_bank_entry;

/* Transition bank for a J-level transform: 7J + 1 entries (seven detail
 * bands per level plus the approximation band at level J), ordered by j,
 * then by o_x + 2 o_y + 4 o_z.  wavelet: 0 = bior4.4, 1 = Haar. */
typedef struct {
    int32_t levels;
    int32_t wavelet;
    int32_t n_sub;
    int32_t pad;
    double tau;
    double ridge_rel;
    vbm_bank_entry sub[64];
} vbm_bank;

/* Adaptive filtering parameters (Supp. Sec. 1): S = E^alpha_E N^beta_N,
 * K_{j,o} = max(min_per_band, floor(K_tot S / sum S)), MAD threshold
 * T = lambda_mad * MAD / 0.6745.  energy_comp != 0 applies s = 2^{-3j/2}
 * (Eq. 23). */
typedef struct {
    double alpha_E;
    double beta_N;
    double lambda_mad;
    int64_t K_tot;
    int32_t min_per_band;
    int32_t energy_comp;
} vbm_select;

/* --------------------------------------------- setup: bank and Gaussians */

/* Build the transition bank on the host in FP64 (Sec. 4.2): for each
 * subband the IDWT of a unit impulse (Eq. 9-10), the ROI
 * {|psi| > tau max|psi|} (Eq. 13), its W-weighted moments (Eq. 14) and the
 * ridge weight w = sum |Y| G / (sum G^2 + ridge_rel sum G^2) (Eq. 17).
 * levels in [1, 9]; wavelet 0 (bior4.4) or 1 (Haar); tau in (0, 1).
 * Host only; writes *out. */
VBM_API vbm_status vbm_bank_build(int levels, int wavelet, double tau, double ridge_rel, vbm_bank *out);

#define VBM_BANK_ISOTROPIC 1     /* ablation "w/o transition bank": one shared isotropic covariance */
#define VBM_BANK_UNIT_WEIGHT 2   /* ablation "w/o energy projection": w = 1 */

/* Turn a bank into an ablation variant of Sec. 5.4, in place (host only).
 * VBM_BANK_ISOTROPIC: every covariance becomes sigma_iso^2 I, with sigma_iso
 * the mean over the bank's subbands of det(Sigma)^(1/6) (the paper's "average
 * spatial extent in the full model"; centres and weights unchanged).
 * VBM_BANK_UNIT_WEIGHT: every ridge weight w becomes 1.  VBM_ERR_ARG on an
 * unknown flag or an empty bank. */
VBM_API vbm_status vbm_bank_ablate(vbm_bank *bank, int32_t flags);

/* Apply the TF to a volume: d_rf[4][n] = TF(d_volume[n]) (Sec. 3),
 * n = nx ny nz, planar RGBA. */
VBM_API vbm_status vbm_tf_apply(const float *d_volume, int64_t n, const vbm_tf *tf, float *d_rf, void *stream);

/* J-level periodised separable 3D DWT of n_channels planar volumes in place
 * (Sec. 3, Eq. 1-3; Sec. 4.3, Eq. 20-21), Mallat layout: after level j the
 * region [0, n/2^(j-1))^3 holds octants o in {L, H}^3, octant o at
 * [o_d n/2^j, (o_d + 1) n/2^j) per axis; level j+1 recurses into LLL.
 * Analysis a[k] = sum_n ht[n] x[(2k+n) mod L], d[k] = sum_n gt[n]
 * x[(2k+1+n) mod L].  dims[d] must be divisible by 2^levels.  d_tmp: 2 nx ny
 * nz floats of scratch. */
VBM_API vbm_status vbm_dwt3d(float *d_data, int n_channels, const int dims[3], int levels, int wavelet,
                     float *d_tmp, void *stream);

/* Workspace bytes vbm_build needs for a volume of dims and levels. */
VBM_API vbm_status vbm_build_workspace_size(const int dims[3], int levels, size_t *bytes);

/* Volume -> Gaussians (Sec. 4.1: F -> RF -> Phi -> G): TF, J-level DWT,
 * adaptive filtering (Supp. Sec. 1) and the per-coefficient map
 * (Eq. 22-24): amplitude s |A| w, centre u + 2^j k + 1/2, covariance of the
 * bank entry; opacity logit = logit(clamp(amp_alpha, 2/255, 0.99)), colour =
 * amp_rgb.  Gaussians are written subband by subband, each in raster order
 * of k, to d_params[14][capacity] (stride = capacity).  *n_out = number kept;
 * if it exceeds capacity nothing is written and VBM_ERR_CAPACITY is
 * returned with *n_out = the required capacity.  If d_coef is not NULL the
 * coefficient pyramid is also copied there (float[4][nz][ny][nx]) and
 * d_keep (if not NULL) receives one byte per pyramid element (1 = kept).
 * Synchronises the stream (copies the subband energies and counts). */
VBM_API vbm_status vbm_build(const float *d_volume, const int dims[3], const vbm_tf *tf, const vbm_bank *bank,
                     const vbm_select *sel, float *d_params, int64_t capacity, int64_t *n_out,
                     float *d_coef, uint8_t *d_keep, void *d_ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------ DVR target images */

/* Emission-absorption ray marching of the supervision images (Sec. 4.4):
 * ray through each pixel centre, clipped to the box [0,nx]x[0,ny]x[0,nz];
 * segments of length `step` (the last one shorter) sampled at their
 * midpoints by trilinear interpolation at p - 1/2 with clamp-to-edge, TF on
 * the interpolated scalar, opacity correction a' = 1 - (1 - a)^len,
 * front-to-back C += T a' c, T *= 1 - a'; stops once T < 1e-6; black
 * background.  Writes d_rgba[V][4][H][W] = (C, 1 - T).  d_cams: n_views
 * device records; every camera must have the given width and height. */
VBM_API vbm_status vbm_render_dvr(const float *d_volume, const int dims[3], const vbm_tf *tf,
                          const vbm_camera *d_cams, int n_views, int width, int height, float step,
                          float *d_rgba, void *stream);

/* ----------------------------------------------------- fine-tuning step */

/* A raster plan owns every buffer of the splatting forward/backward for a
 * fixed batch: per-(view, Gaussian) projected splats, per-tile pair counts,
 * the (tile, depth, index)-ordered pair lists, tile ranges and per-pixel
 * compositing state (the saved context between forward and backward).  One
 * plan per stream. */
typedef struct vbm_plan vbm_plan;

#define VBM_PLAN_RECOMPUTE 1   /* keep no per-pixel state; backward recomputes it */
#define VBM_PLAN_PERSISTENT 2  /* compositing kernels run as one persistent grid pulling tiles,
                                  longest list first, from a work queue */
#define VBM_PLAN_RADIX_SORT 4  /* order the pairs with device radix sorts instead of the bucketed
                                  per-tile sort: the items are sorted by depth (stable LSD radix
                                  sort on the 32 depth bits), their pairs emitted in that order and
                                  sorted stably by tile (LSD radix sort on ceil(log2 tiles) bits),
                                  which is the sort on (tile | depth) keys with ties in item order;
                                  the lists are identical bit for bit */

/* Batch description.  Scenes are independent Gaussian sets stored as column
 * ranges [scene_offset[s], scene_offset[s+1]) of one parameter array; view v
 * renders scene view_scene[v] (NULL means all views render scene 0).  Every
 * view has the same width x height.  Tiles are tile_w x tile_h pixels
 * (tile_w 8 or 16, tile_h a multiple of 4, tile_w * tile_h in {32, 64, 128,
 * 256}); each compositing
 * thread handles pixels_per_thread pixels of one tile column (at least 32
 * threads per tile), and the threads of a warp form groups of group_lanes
 * lanes that each walk the list entries reaching their own pixel block.
 * pair_capacity bounds the number of (tile, Gaussian) pairs of one call.
 * At most 65535 tiles along each image axis. */
typedef struct {
    int32_t n_scenes;
    int32_t n_views;
    const int64_t *scene_offset;   /* host, n_scenes + 1 entries   */
    const int32_t *view_scene;     /* host, n_views entries or NULL */
    int32_t width, height;
    int32_t tile_w, tile_h;
    int64_t pair_capacity;
    int32_t flags;
    int32_t pixels_per_thread;     /* 0 = default (2); 1, 2 or 4 */
    int32_t group_lanes;           /* 0 = default (32); 4, 8, 16 or 32 lanes per compositing group */
    int32_t segment_len;           /* persistent plans: the backward walks a tile list longer than
                                      this many entries as segments that different warps take at
                                      once (the forward stores each pixel's transmittance and
                                      colour still to come at every segment boundary, and with
                                      VBM_PLAN_RECOMPUTE the tile's final per-pixel state; the
                                      plan holds checkpoints for about 2 pairs per (view, Gaussian)
                                      item, at most 1 GiB; tiles beyond that are walked whole).  0 = default (256); a positive multiple of 32 up to
                                      65536; -1 = never split.  Ignored by other plans.  Results
                                      equal the unsplit walk's up to FP32 rounding of the
                                      transmittance and of the colour sums. */
    int32_t bwd_pixels_per_thread; /* the backward compositing kernel's own pixels per thread and */
    int32_t bwd_group_lanes;       /* lanes per group (0 = the forward's); its warp regions are its
                                      own, so results do not depend on them */
} vbm_plan_desc;

/* Create a plan (allocates device memory, synchronous). */
VBM_API vbm_status vbm_plan_create(const vbm_plan_desc *desc, vbm_plan **out);

/* Free a plan and its device memory (synchronises the device). */
VBM_API vbm_status vbm_plan_destroy(vbm_plan *plan);

/* Synchronise `stream` and read the plan's device status word.  Returns
 * VBM_ERR_CAPACITY if any call since the last check needed more pairs than
 * pair_capacity (that call rendered background only); *pairs_needed (if
 * not NULL) receives the largest pair count required.  Clears the word. */
VBM_API vbm_status vbm_plan_check(vbm_plan *plan, void *stream, int64_t *pairs_needed);

/* Forward splatting of views [view_begin, view_begin + view_count) (Sec. 4.4,
 * 3DGS conventions): per (view, Gaussian) EWA projection (cull z <= znear,
 * x/z and y/z clamped to the image +15% for the Jacobian, 2D covariance
 * J W Sigma W^T J^T + 0.3 I, radius ceil(k sqrt(lambda_max)) with
 * k = min(3, sqrt(2 ln(255 o))), no tiles when o < 1/255), tile binning
 * (of the radius rectangle, the tiles where some pixel centre can see
 * alpha >= 1/255, by the exact minimum of the quadratic form over the tile
 * with a 1e-3 margin in the log) ordered by depth (ties by Gaussian index),
 * front-to-back compositing per
 * pixel (alpha = min(0.99, o e^power), skip alpha < 1/255, stop before T
 * falls below 1e-4).  Writes d_img[V][3][H][W] = C + T bg and, if not NULL,
 * d_alpha[V][H][W] = 1 - T, at absolute view indices.  d_params: P[14]
 * [stride]; d_cams: device array of all views. */
VBM_API vbm_status vbm_raster_fwd(vbm_plan *plan, const float *d_params, int64_t stride, const vbm_camera *d_cams,
                          int32_t view_begin, int32_t view_count, const float bg[3],
                          float *d_img, float *d_alpha, void *stream);

/* Reverse-mode derivative of vbm_raster_fwd for the same views (which must
 * be the last forward call on this plan): from d_dL_dimg[V][3][H][W] (and
 * d_dL_dalpha[V][H][W], may be NULL) to d_grad[14][stride].  With
 * accumulate = 0 the gradient rows of the Gaussians these views see are
 * overwritten; otherwise added to. */
VBM_API vbm_status vbm_raster_bwd(vbm_plan *plan, const float *d_params, int64_t stride, const vbm_camera *d_cams,
                          int32_t view_begin, int32_t view_count, const float bg[3],
                          const float *d_dL_dimg, const float *d_dL_dalpha, float *d_grad,
                          int32_t accumulate, void *stream);

/* The backward of the last forward call fused with the Adam step that
 * follows it in fine-tuning (Sec. 4.4, Sec. 5.2): the result equals, bit for
 * bit, vbm_raster_bwd with accumulate = 0 into a gradient array that is zero
 * outside the rows the call's views see, followed by vbm_adam on d_params,
 * d_m, d_v over the first n columns (every one of them takes its Adam step;
 * columns of scenes no view of the call renders with a zero gradient).  The
 * gradient itself is not written: each Gaussian's gradient, summed over the
 * views in registers, is applied where it is formed, saving the gradient
 * array's write and read and a second read of the parameters.  d_params is
 * updated in place (it is read by the backward first, per Gaussian).
 * Arguments as for vbm_raster_bwd and vbm_adam; stride >= n. */
VBM_API vbm_status vbm_raster_bwd_adam(vbm_plan *plan, float *d_params, int64_t stride, const vbm_camera *d_cams,
                                       int32_t view_begin, int32_t view_count, const float bg[3],
                                       const float *d_dL_dimg, const float *d_dL_dalpha, float *d_m, float *d_v,
                                       int64_t n, int32_t *d_step, const float lrs[5], float beta1, float beta2,
                                       float eps, uint32_t *d_nonfinite, void *stream);

/* Internal buffers of a plan after a forward call (device pointers, read
 * only, valid until the next call on the plan).  Items are numbered view by
 * view over the call's views. */
typedef struct {
    int64_t n_items;          /* (view, Gaussian) items of the last call          */
    const float *rec;         /* [n_items][16], one 64-byte record per item: u, v, conic A, conic B |
                                 r, g, b, opacity | half-widths (x, y) of the alpha >= 1/255 box,
                                 B / C, B / A | conic C, tau = 2 (ln(255 o) + 1e-3) (the binning
                                 tile test's bound; -1 for an item without tiles), camera z, the
                                 radius in pixels (int32 bits) */
    const uint32_t *place;    /* [n_items][4] placement record: x0 | x1 << 16, y0 | y1 << 16 (the
                                 tile rectangle [x0, x1) x [y0, y1)), the listed-tile word (bit k:
                                 the k-th tile of a rectangle of at most 8 tiles, row-major, passed
                                 the tile test; bit 31 alone: a larger rectangle; 0: no tiles),
                                 camera z (float bits) */
    const uint32_t *pair_tile;/* [n_pairs] sorted tile ids (relative to view_begin) */
    const uint32_t *pair_item;/* [n_pairs] item of each pair                       */
    const int32_t *ranges;    /* [tiles][2] start, end                             */
    const int64_t *n_pairs;   /* device scalar                                     */
    const float *T_final;     /* [V][H][W] (absolute views; NULL in recompute mode) */
    const int32_t *n_contrib; /* [V][H][W]                                         */
    const float *g_splat;     /* [n_items][12] after a backward: du dv dA dB dC dopac dr dg db, 3 unused */
    const int32_t *seg_count; /* persistent plans, device [4]: backward units of the segmented tiles,
                                 segmented tiles, checkpoint slots requested (may exceed
                                 checkpoint_slots: the tiles that found none were walked whole), -;
                                 NULL when lists are never split */
    int64_t checkpoint_slots; /* checkpoint slots the plan holds (0 when lists are never split) */
} vbm_plan_buffers;

VBM_API vbm_status vbm_plan_get_buffers(vbm_plan *plan, vbm_plan_buffers *out);

/* Workspace bytes for vbm_loss over n_images planar RGB images of H x W. */
VBM_API vbm_status vbm_loss_workspace_size(int n_images, int height, int width, size_t *bytes);

/* Image loss of the fine-tuning step (Sec. 4.4, "as in" 3DGS) and its
 * gradient: per element e of n_images x 3 x H x W,
 *   L += scale * ((1 - lambda) |x_e - y_e| + lambda (1 - ssim_e)),
 *   d_dL_dimg[e] = dL/dx_e (overwritten),
 * with SSIM over an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2,
 * C2 = 0.03^2, zero padding, per channel; sign(0) = 0.  scale = 1 / (number
 * of elements of the whole batch) gives the mean.  *d_loss (double) is
 * overwritten, or added to when accumulate != 0.  At most 21845 images per
 * call (VBM_ERR_ARG beyond: split the batch and accumulate).  The first call
 * on a device uploads the SSIM window to its constant memory (a synchronous
 * copy): make it before any stream capture. */
VBM_API vbm_status vbm_loss(const float *d_img, const float *d_target, int n_images, int height, int width,
                    float lambda, double scale, double *d_loss, int32_t accumulate, float *d_dL_dimg,
                    void *d_ws, size_t ws_bytes, void *stream);

/* vbm_loss without a workspace argument and without any allocation, for
 * callers that cannot allocate device memory when they compute the loss:
 * code running while a CUDA graph is being captured, loops whose memory
 * budget is fixed at start-up, hosts that own only the image buffers they
 * pass.  The paper has no counterpart; this is a deployment variant of
 * vbm_loss with identical arguments and results minus (d_ws, ws_bytes).
 * Scratch is a static 32 MiB device array of the library (held by every GPU
 * that loads it, until exit): calls whose vbm_loss workspace would exceed
 * 32 MiB return VBM_ERR_CAPACITY without launching (split the batch and use
 * accumulate).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and uploads the SSIM window to that
 * device's constant memory; make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race;
 * nothing in it needs clearing between calls. */
VBM_API vbm_status vbm_loss_static(const float *d_img, const float *d_target, int n_images, int height, int width,
                                   float lambda, double scale, double *d_loss, int32_t accumulate,
                                   float *d_dL_dimg, void *stream);

/* Adam step (Sec. 5.2) on P[14][stride], first n columns: *d_step is
 * incremented on the device and t = the new value drives the bias
 * correction; row groups {0-2, 3-5, 6-9, 10, 11-13} use lrs[0..4].
 * Non-finite gradient elements leave their parameter, m and v unchanged and
 * are counted into *d_nonfinite (if not NULL). */
VBM_API vbm_status vbm_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t n, int64_t stride,
                    int32_t *d_step, const float lrs[5], float beta1, float beta2, float eps,
                    uint32_t *d_nonfinite, void *stream);

/* ------------------------------------------------------------ diagnostics */

/* Number of kernels this library has launched in this process (host counter,
 * all devices and streams).  The difference across a call sequence is the
 * launch count of that sequence. */
VBM_API int64_t vbm_kernel_launches(void);

/* Profiling hooks of a plan (all optional, NULL disables).  events holds
 * n_events (0, 4 or 7) cudaEvent_t handles created by the caller with timing
 * enabled, recorded on the call's stream (under stream capture as external
 * event nodes):
 *   [0], [1]  just before and after the compositing kernel of vbm_raster_fwd;
 *   [2], [3]  just before and after the compositing kernel of vbm_raster_bwd;
 *   [4]       at the start of vbm_raster_fwd (before the projection);
 *   [5]       after the projection kernel (binning and sorting follow, up to [0]);
 *   [6]       at the end of vbm_raster_bwd (after the projection backward).
 * d_n_eval (int32 [V][H][W]) receives, per pixel of a forward call, the number
 * of list entries evaluated (up to and including the one that ended
 * compositing); d_n_contrib (int32 [V][H][W]) receives the contributor count
 * (one past the last blended entry) in plans created with VBM_PLAN_RECOMPUTE,
 * which keep none of their own.  The hooks stay set until changed. */
VBM_API vbm_status vbm_plan_set_profile(vbm_plan *plan, int32_t n_events, void *const *events, int32_t *d_n_eval,
                                        int32_t *d_n_contrib);

/* Throughput probe for the roofline denominators of the compositing kernels
 * (not part of the method): one launch of `blocks` blocks of 256 threads, each
 * thread running 8 independent dependent chains of `iters` links (a multiple
 * of 16) of kind 0: scalar FP32 FMA, 1: packed FP32x2 FMA (fma.rn.f32x2),
 * 2: ex2.approx.ftz.f32 (one FMA beside each).  *ops (host) receives the
 * launch's work: FLOP for kinds 0 and 1 (2 per FMA), ex2 evaluations for kind
 * 2.  The caller times the launch (CUDA events on `stream`) and divides.
 * d_out needs blocks * 256 floats and is written only in a case that does not
 * occur (it keeps the chains from being removed). */
VBM_API vbm_status vbm_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float *d_out, double *ops,
                                  void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBM_H */
