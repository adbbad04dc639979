/*
 * darb.h -- C ABI of libdarb.so, a GB300 (sm_103a) differentiable tile rasterizer for
 * DARB splats: 3D anisotropic splats whose reconstruction kernel is a decaying
 * anisotropic radial basis function F(d_M) of the Mahalanobis distance
 * (arxiv 2501.12369, Sec. 4, Eq. darbf_class, Table 1).
 *
 * Conventions for every entry point
 *   - Pointers named "device" are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns and allocates every
 *     buffer; the library never allocates device memory on these paths and keeps no
 *     pointer after a call returns.
 *   - Device pointers must be 16-byte aligned (any cudaMalloc / PyTorch allocation is).
 *   - All work is enqueued on the given stream (NULL = legacy default stream) and runs
 *     asynchronously unless the entry point says it synchronises.
 *   - Errors are returned as darb_status; nothing is thrown across the ABI.  A status
 *     other than DARB_OK means nothing was enqueued, except DARB_ERR_CUDA (a launch or
 *     copy failed; the stream state is undefined) and the statuses that say otherwise.
 *   - Arrays are row-major, C-contiguous float32 unless stated.  Images are planar
 *     [3][H][W].  Pixel (x, y) has its centre at (x + 0.5, y + 0.5).
 *   - Cameras use OpenCV axes (x right, y down, z forward); viewmat maps world to camera.
 */
#ifndef DARB_H
#define DARB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *darb_stream; /* a cudaStream_t */

typedef enum {
    DARB_OK = 0,
    DARB_ERR_INVALID_ARG = 1, /* bad size, NULL, misaligned pointer, unknown enum */
    DARB_ERR_WORKSPACE = 2,   /* workspace smaller than the size query returned */
    DARB_ERR_CAPACITY = 3,    /* more (splat, tile) instances than the output capacity */
    DARB_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    DARB_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up; results invalid */
    DARB_ERR_ADMISSION = 6,   /* serving: request cannot be admitted */
    DARB_ERR_NOT_FOUND = 7    /* serving: unknown scene or ticket */
} darb_status;

/* Reconstruction kernels.  q = d_M^2 under the psi-corrected, dilated 2D covariance.
 *   GAUSSIAN          exp(-q/2)                        (Table 1, xi = 2)
 *   HALF_COSINE       cos(pi q / 18)                   (Eq. HalfCosine, xi = 18/pi)
 *   RAISED_COSINE     1/2 + 1/2 cos(pi sqrt(q) / 2.5)  (Sec. B.1, xi = 2.5/pi)
 *   MOD_SINC          |sin x| / x, x = pi sqrt(q) / 3  (Sec. B.3, xi = 3/pi)
 *   INV_QUADRIC       1 / (1 + q)                      (Sec. B.4 listing)
 *   INV_MULTIQUADRIC  (1 + q)^(-1/2)                   (Table 1, xi = 1)
 *   PARABOLA          1 - q/9                          (Table 1, Sec. B.5, xi = 9)      */
typedef enum {
    DARB_GAUSSIAN = 0,
    DARB_HALF_COSINE = 1,
    DARB_RAISED_COSINE = 2,
    DARB_MOD_SINC = 3,
    DARB_INV_QUADRIC = 4,
    DARB_INV_MULTIQUADRIC = 5,
    DARB_PARABOLA = 6,
    DARB_GENERIC = 7 /* Table 1's modified family, described by base, xi, beta, lobes below */
} darb_kernel;

/* Bases of the generic member, F = base(u) with u = d_M^beta / xi (Table 1). */
typedef enum {
    DARB_BASE_GAUSSIAN = 0,         /* exp(-u)                               d_M >= 0          */
    DARB_BASE_HALF_COSINE = 1,      /* cos(u)                                u <= pi / 2       */
    DARB_BASE_RAISED_COSINE = 2,    /* 1/2 + 1/2 cos(u)                      u <= n pi         */
    DARB_BASE_MOD_SINC = 3,         /* |sin u| / u                           u <= (n + 1) pi / 2 */
    DARB_BASE_INV_MULTIQUADRIC = 4, /* (u + 1)^(-1/2)                        d_M >= 0          */
    DARB_BASE_PARABOLA = 5          /* 1 - u                                 u <= 1            */
} darb_kernel_base;

/* kind: a darb_kernel.  psi: correction factor multiplying the 2x2 EWA block (Eq.
 * 2x2covProjection, Table 2).  q_max: main-lobe limit on q (Sec. A.3); a pixel is
 * skipped when q > q_max, or q >= q_max when q_max_strict is non-zero.
 * base, xi, beta, lobes: the member of Table 1's family; they define F for DARB_GENERIC and
 * describe the fixed kinds (darb_kernel_defaults fills them; ignored there). */
typedef struct {
    int32_t kind;
    float psi;
    float q_max;
    int32_t q_max_strict;
    int32_t base; /* a darb_kernel_base */
    float xi;     /* > 0 */
    float beta;   /* 0.5 .. 4 */
    int32_t lobes; /* n >= 1: lobes kept by the raised cosine and the modular sinc */
} darb_kernel_params;

/* Parameters of the generic member (base, xi, beta, lobes): q_max = min(9, (xi u_max)^(2/beta))
 * with u_max the domain end of Table 1 (9 for the unbounded bases) -- the tile rectangle's
 * radius 3 sqrt(lambda_max) bounds every footprint at q = 9 (Sec. 4.1).  psi is left 1: set it
 * with darb_kernel_psi or by hand. */
darb_status darb_kernel_generic(int32_t base, float xi, float beta, int32_t lobes, darb_kernel_params *out);

/* psi of any kernel by the moment integral on the device: the per-axis second moment of the
 * truncated 3D kernel with Sigma = I, (1/3) int r^4 F(r^2) dr / int r^2 F(r^2) dr over
 * [0, sqrt(q_max)] -- the quantity the Sec. A.2 grid experiment measures (and, for the fixed
 * kernels, the printed psi to its precision).  Midpoint rule over 2^22 radii in FP64.
 * scratch: device double[2].  Synchronises `stream`; *psi receives the value. */
darb_status darb_kernel_psi(const darb_kernel_params *kparams, double *scratch, double *psi, darb_stream stream);

typedef struct {
    float viewmat[16]; /* world -> camera, row-major [R t; 0 0 0 1] */
    float fx, fy, cx, cy, near_plane;
    int32_t width, height;
    float bg[3]; /* background colour composited behind the splats */
} darb_camera;

/* Splat parameters, device pointers, SoA (the 3DGS parameterisation, Sec. 4.1).
 * means [n][3]; scales [n][3] (activated, > 0); quats [n][4] as (w, x, y, z), any
 * non-zero norm (normalised inside); opacities [n] (activated, in (0, 1));
 * sh [n][(sh_degree+1)^2][3] real SH coefficients, sh_degree in 0..3. */
typedef struct {
    const float *means, *scales, *quats, *opacities, *sh;
    int32_t n, sh_degree;
} darb_splats;

/* Per-splat outputs of darb_preprocess, device pointers, each with n entries.
 * depth [n]: camera-space z.  radius [n]: ceil(3 sqrt(lambda_max)); 0 = culled (behind the
 * near plane, outside the guard band, a degenerate covariance, or no member tile).
 * tile_rect [n][4]: inclusive tile rectangle (tx0, ty0, tx1, ty1) of the pixel centres within
 * radius of the centre.
 * mean2d [n][2]: projected centre in pixels.  conic_o [n][4]: (A, B, C, opacity) with
 * q = A dx^2 + 2 B dx dy + C dy^2.  rgb [n][3]: SH colour.  clamped [n]: bit c set when
 * colour channel c was clamped at 0.
 * tiles_touched [n]: member tiles.  In each tile row of the rectangle they are the run of
 * columns whose pixel centres the ellipse {q <= q_max} reaches over the row's band of
 * pixel-centre heights (the Sec. 3 footprint's support, tested per tile row).
 * tile_runs [n]: the same runs packed, for darb_bin_sort: when the rectangle spans at most 8
 * rows and 15 columns, byte k (from the least significant) holds row ty0 + k's run as
 * (c1 - tx0) << 4 | (c0 - tx0), or 0x0F for a row without member tiles (also for the bytes
 * past the last row); all ones for larger rectangles and culled splats. */
typedef struct {
    float *depth;
    int32_t *radius;
    int32_t *tile_rect;
    float *mean2d;
    float *conic_o;
    float *rgb;
    uint8_t *clamped;
    uint32_t *tiles_touched;
    uint64_t *tile_runs;
} darb_projected;

/* Outputs of darb_bin_sort, device pointers.
 * keys [capacity], values [capacity]: the (splat, tile) instances sorted by
 * key = tile << 32 | bits(depth), ties by splat index; values hold splat indices.
 * ranges [tiles_y * tiles_x][2]: [start, end) of each tile's run in values; [0, 0) if empty.
 * num_instances [1]: M, the number of instances (written even when M > capacity).
 * status [1]: 0, or a darb_status the device detected (DARB_ERR_CAPACITY, DARB_ERR_TIMEOUT). */
typedef struct {
    uint64_t *keys;
    uint32_t *values;
    uint32_t *ranges;
    uint32_t *num_instances;
    uint32_t *status;
} darb_binning;

/* Outputs of darb_render_fwd, device pointers.
 * image [3][H][W]; t_final [H][W]: transmittance left after the last blended splat;
 * last [H][W]: one past the position, within the pixel's tile run, of the last blended
 * splat (0 if none); n_contrib [H][W]: number of blended splats. */
typedef struct {
    float *image;
    float *t_final;
    uint32_t *last;
    uint32_t *n_contrib;
} darb_image;

/* Gradients w.r.t. the splat parameters, device pointers, layouts as darb_splats.
 * dscales and dopacities are w.r.t. the activated values. */
typedef struct {
    float *dmeans, *dscales, *dquats, *dopacities, *dsh;
} darb_splat_grads;

/* Human-readable name of a status.  Never NULL. */
const char *darb_status_string(darb_status s);

/* Paper defaults for a kernel: psi of the Sec. B listings (Table 2 where no listing is
 * printed), q_max and strictness of the listings' main-lobe limits (Sec. A.3).
 * out: host pointer.  DARB_ERR_INVALID_ARG for an unknown kind or NULL out. */
darb_status darb_kernel_defaults(int32_t kind, darb_kernel_params *out);

/* Number of tiles of a camera: tiles_x = ceil(W / tile), tiles_y = ceil(H / tile).
 * Host pointers.  tile must be 8, 16 or 32. */
darb_status darb_tile_grid(const darb_camera *cam, int32_t tile, int32_t *tiles_x, int32_t *tiles_y);

/* Step 1: per-splat preprocessing (Sec. 4.1 "DARB Projection"; Eq. 2x2covProjection;
 * the "cov *= correctionFactor" lines of the Sec. B listings): view transform, near
 * cull (z <= near_plane), Sigma = R S S^T R^T, Sigma2 = psi (J W Sigma W^T J^T)_2x2
 * + 0.3 I, conic, R = ceil(3 sqrt(lambda_max)) (Sec. 4.1), pixel-exact tile rectangle,
 * member tiles (the row runs of the ellipse q <= kparams->q_max; a splat without member
 * tiles is culled), SH colour.  Geometry follows a fixed IEEE FP32 operation sequence, so
 * the results are bit-reproducible.  splats, cam, kparams: host structs holding device pointers
 * (splats) or values.  out: host struct of caller-owned device buffers sized n. */
darb_status darb_preprocess(const darb_splats *splats, const darb_camera *cam,
                            const darb_kernel_params *kparams, int32_t tile,
                            const darb_projected *out, darb_stream stream);

/* Sort strategies of darb_bin_sort.  Both give the same keys, values and ranges, bit for bit.
 *   DARB_SORT_DEPTH_THEN_TILE: sort the n splats by depth once, emit the instances in that order
 *     and sort them stably by tile id only (2 LSD passes of 32-bit keys at 1080p / 16-pixel tiles;
 *     about 36 bytes of traffic per instance).  out->keys is optional (NULL: not written).
 *   DARB_SORT_KEYS64: one stable LSD sort of the 64-bit keys tile << 32 | bits(depth) over their
 *     low 32 + ceil(log2(tiles)) bits (6 passes at 1080p).  out->keys is required. */
typedef enum { DARB_SORT_DEPTH_THEN_TILE = 0, DARB_SORT_KEYS64 = 1 } darb_sort_strategy;

/* Workspace bytes darb_bin_sort needs for n splats, an instance capacity and a strategy.
 * Host pointers; no device work. */
darb_status darb_bin_sort_workspace_size(int32_t n, int32_t tile, const darb_camera *cam,
                                         uint64_t capacity, int32_t strategy, size_t *bytes);

/* Steps 2 and 3: tile/depth key duplication and radix sort (the tile-based
 * rasterization with a bounding box that Sec. A.3 inherits from 3DGS).  Scans
 * tiles_touched, emits one instance per member tile of each splat (the row runs of
 * darb_projected; kparams->q_max sets the ellipse) and sorts them with LSD onesweep radix
 * passes into the order of key = tile << 32 | bits(depth), ties by splat index, then writes
 * the per-tile ranges, [0, 0) for a tile without instances.  strategy: a darb_sort_strategy.
 * proj: darb_preprocess outputs.  workspace: device, at least
 * darb_bin_sort_workspace_size bytes, contents scratch.  capacity: entries of
 * out->keys / out->values (< 2^30).  num_instances_host: if non-NULL the call
 * synchronises the stream once to read M and returns DARB_ERR_CAPACITY when
 * M > capacity (outputs then undefined); if NULL nothing synchronises, the sort is
 * sized by capacity, and an overflow is reported in out->status with every tile range
 * left empty (so a following darb_render_fwd draws only the background).  The per-tile counts
 * run on a side stream of the library (one per device, created by the first call, so make one
 * call before capturing the stream), forked from and joined back to `stream` with events,
 * beside the depth sort: the call stays ordered on `stream` and can be captured in a CUDA graph
 * (with num_instances_host NULL); calls from several host threads on one device are
 * serialised while they enqueue. */
darb_status darb_bin_sort(const darb_projected *proj, int32_t n, int32_t tile,
                          const darb_camera *cam, const darb_kernel_params *kparams,
                          void *workspace, size_t workspace_bytes,
                          uint64_t capacity, int32_t strategy, const darb_binning *out,
                          uint64_t *num_instances_host, darb_stream stream);

/* darb_bin_sort without a caller-supplied workspace, for callers that cannot allocate device
 * memory: for instance a plugin running inside another application's capture or render loop,
 * where a cudaMalloc would synchronise the device, break a memory budget the host application
 * enforces, or is simply not permitted.  The paper has no counterpart; it is an allocation-free
 * form of the same sort with identical results.
 * The scratch is a static device array of 64 MiB inside the library, held by every GPU that
 * loads the library until the process exits.  Sizes whose darb_bin_sort_workspace_size exceeds
 * 64 MiB are rejected with DARB_ERR_WORKSPACE.  The first call on a device resolves the array's
 * device address (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture; the address is kept for the process, so the device must not be reset
 * (cudaDeviceReset) after that first call.  The call itself allocates nothing: no cudaMalloc, no cudaFree.  All calls share the
 * one array and each call clears what must start at zero, so calls that overlap on the GPU (two
 * streams, or two host threads) race and must be serialised by the caller.  Other arguments and
 * results are those of darb_bin_sort. */
darb_status darb_bin_sort_noalloc(const darb_projected *proj, int32_t n, int32_t tile,
                                  const darb_camera *cam, const darb_kernel_params *kparams,
                                  uint64_t capacity, const darb_binning *out,
                                  uint64_t *num_instances_host, darb_stream stream);

/* Step 4: per-pixel front-to-back compositing (Sec. 4.1, "alpha blending ... similar to
 * 3DGS"; forward listings of Sec. B): for each splat of the pixel's tile run in depth
 * order, skip unless 0 <= q <= q_max, alpha = min(0.99, o F(q)), skip alpha < 1/255,
 * stop before T (1 - alpha) < 1e-4, C += c alpha T.  Then C += T bg.
 * q = dx (A dx + 2B dy) + (C dy) dy is evaluated by a fixed FP32 sequence. */
darb_status darb_render_fwd(const darb_projected *proj, const darb_binning *bins,
                            const darb_camera *cam, const darb_kernel_params *kparams,
                            int32_t tile, const darb_image *out, darb_stream stream);

/* Step 4 with the L1 image loss of Sec. 4.2 taken in the same kernel: darb_render_fwd, then
 * for every pixel and channel dL_dimage = sign(C - target) / (3 W H) and *loss = the mean of
 * |C - target|, while the colour is still in registers.  target, dL_dimage: device
 * [3][H][W]; loss: device [1], zeroed by the call, then accumulated (the order of its FP32
 * additions varies from run to run; dL_dimage and every image output equal darb_render_fwd +
 * darb_l1_loss bit for bit).  out->image and out->n_contrib may be NULL (not written): a
 * training step needs only the loss, its gradient, and t_final and last for the backward. */
darb_status darb_render_fwd_l1(const darb_projected *proj, const darb_binning *bins,
                               const darb_camera *cam, const darb_kernel_params *kparams,
                               int32_t tile, const darb_image *out, const float *target,
                               float *dL_dimage, float *loss, darb_stream stream);

/* Backward of step 4 (Sec. 4.2; backward listings of Sec. B): replays each pixel back
 * to front from last / t_final, applies dF/dq of the kernel, and accumulates per-splat
 * gradients.  n: number of splats.  dL_dimage: device [3][H][W].  grad2d: device [n][12],
 * zeroed by the callee,
 * per splat (d mu'x, d mu'y, dA, dB, dC, d opacity, dr, dg, db, 0, 0, 0).  The alpha
 * clamp at 0.99 has zero derivative. */
darb_status darb_render_bwd(const darb_projected *proj, int32_t n, const darb_binning *bins,
                            const darb_camera *cam, const darb_kernel_params *kparams,
                            int32_t tile, const darb_image *fwd, const float *dL_dimage,
                            float *grad2d, darb_stream stream);

/* Backward of step 1: chains grad2d through the conic, psi, the EWA projection, the
 * quaternion normalisation and the SH basis (the conic -> covariance lines of the Sec. B
 * backward listings carry psi).  out: caller-owned device buffers, fully written
 * (zeros for culled splats). */
darb_status darb_preprocess_bwd(const darb_splats *splats, const darb_camera *cam,
                                const darb_kernel_params *kparams, const darb_projected *proj,
                                const float *grad2d, const darb_splat_grads *out,
                                darb_stream stream);

/* L1 photometric term of the training loss (Sec. 4.2): loss = mean |image - target|,
 * dL_dimage = sign(image - target) / (3 H W).  image, target, dL_dimage: device
 * [3][H][W].  loss: device float[1], overwritten. */
darb_status darb_l1_loss(const float *image, const float *target, int32_t width, int32_t height,
                         float *dL_dimage, float *loss, darb_stream stream);

/* The full image loss of Sec. 4.2: L = (1 - lambda) L1 + lambda (1 - SSIM).  The paper takes
 * both terms from 3DGS without printing lambda or the SSIM window; as there: SSIM per channel
 * with an 11 x 11 Gaussian window (sigma 1.5, normalised) over zero-padded images,
 * C1 = 0.01^2, C2 = 0.03^2 (intensities in [0, 1]), averaged over the 3 H W values; lambda 0.2
 * in 3DGS.  image, target, dL_dimage: device [3][H][W].  loss: device float[2], overwritten
 * with L and the mean SSIM.  workspace: device, darb_l1_dssim_workspace_size bytes (three
 * derivative maps and two sums).  lambda in [0, 1]; lambda = 0 gives darb_l1_loss's gradient. */
darb_status darb_l1_dssim_workspace_size(int32_t width, int32_t height, size_t *bytes);
darb_status darb_l1_dssim_loss(const float *image, const float *target, int32_t width, int32_t height,
                               float lambda, void *workspace, size_t workspace_bytes, float *dL_dimage,
                               float *loss, darb_stream stream);

/* Raw (optimised) parameters of a training run, device pointers, layouts as darb_splats
 * except log_scales = log(scales) and opacity_logits = logit(opacities).  scales and
 * opacities are the activated copies that darb_adam_step rewrites after the update. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
    float *scales, *opacities;
    int32_t n, sh_degree;
} darb_train_params;

/* Adam first and second moments, device pointers with the layouts of the raw params. */
typedef struct {
    float *m_means, *v_means, *m_scales, *v_scales, *m_quats, *v_quats;
    float *m_opac, *v_opac, *m_sh, *v_sh;
} darb_adam_state;

typedef struct {
    float lr_means, lr_scales, lr_quats, lr_opacities, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;
    int32_t step; /* 1-based step number, for bias correction */
} darb_adam_config;

/* One Adam step of the 3DGS optimiser (Sec. 5: original hyper-parameters, opacity lr
 * 0.02) on the raw parameters.  grads: w.r.t. the activated values (darb_preprocess_bwd);
 * chained through exp / sigmoid inside.  Updates params, state and the activated copies. */
darb_status darb_adam_step(const darb_train_params *params, const darb_splat_grads *grads,
                           const darb_adam_state *state, const darb_adam_config *cfg,
                           darb_stream stream);

/* darb_preprocess_bwd followed by darb_adam_step, fused per splat: the gradients of one splat
 * stay in registers and go straight into its Adam update, so no darb_splat_grads buffer is
 * written or read.  Same arguments and results as the two calls in sequence (gradients of
 * culled splats are zero; every splat takes the step).  params: read for the forward values
 * (means, scales, quats, sh) and updated in place; every parameter and moment array 16-byte
 * aligned (the Adam pass moves float4 lanes over each group).  proj, grad2d: as for
 * darb_preprocess_bwd.  DARB_ERR_INVALID_ARG on a missing or misaligned pointer. */
darb_status darb_preprocess_bwd_adam(const darb_train_params *params, const darb_camera *cam,
                                     const darb_kernel_params *kparams, const darb_projected *proj,
                                     const float *grad2d, const darb_adam_state *state,
                                     const darb_adam_config *cfg, darb_stream stream);

/* ---- Adaptive density control -----------------------------------------------------------
 * The paper keeps the 3DGS optimisation pipeline (Sec. 4 block diagram), whose density control
 * is: per step, statistics of every visible splat; every few hundred steps, clone small splats
 * with large view-space gradients, split large ones, prune transparent or oversized ones; and a
 * periodic opacity reset.  All decisions are taken in float32 in a fixed operation order. */

/* One step's statistics, for every splat with radius > 0: accum += |(dmean_x W/2, dmean_y H/2)|
 * (the view-space mean gradient in normalised device units), count += 1, max_radius =
 * max(max_radius, radius).  grad2d: device [n][12] from darb_render_bwd; radius: device [n] from
 * darb_preprocess; accum, count (float), max_radius (int32): device [n], updated in place. */
darb_status darb_densify_stats(const float *grad2d, const int32_t *radius, int32_t n, int32_t width,
                               int32_t height, float *accum, float *count, int32_t *max_radius,
                               darb_stream stream);

typedef struct {
    float grad_threshold;    /* grow when accum / count >= this (3DGS: 0.0002) */
    float dense_scale;       /* clone when the largest scale <= this, split above (0.01 x extent) */
    float min_opacity;       /* prune below (0.005) */
    float max_screen_radius; /* prune above, pixels; <= 0 disables */
    float max_world_scale;   /* prune when the largest scale is above; <= 0 disables */
    float split_scale_div;   /* children's scales = parent's / this (1.6) */
} darb_densify_cfg;

darb_status darb_densify_workspace_size(int32_t n, size_t *bytes);

/* One density-control pass from `in` (+ its Adam state) into `out` (+ state), which must not
 * overlap the inputs and must hold capacity >= 2 n rows.  Output rows, in order: the surviving
 * splats in index order (their moments kept), then the kept clones in parent order, then two
 * children per kept split parent (moments zero).  Clones and children start with screen radius
 * 0 for the prune test; children's means are parent + R(q) (s * z) with z = split_normals
 * [n][2][3] (device, standard normal, caller-drawn), their log-scales the parent's minus
 * log(split_scale_div).  n_out: device uint32[3] = rows written, first clone row, first child
 * row.  Asynchronous; statistics of the new set are the caller's to reset. */
darb_status darb_densify(const darb_train_params *in, const darb_adam_state *in_state, const float *accum,
                         const float *count, const int32_t *max_radius, const float *split_normals,
                         const darb_densify_cfg *cfg, void *workspace, size_t workspace_bytes,
                         int32_t capacity, const darb_train_params *out, const darb_adam_state *out_state,
                         uint32_t *n_out, darb_stream stream);

/* Opacity reset: logits clamped to logit(max_opacity), activated opacities refreshed. */
darb_status darb_reset_opacity(const darb_train_params *params, float max_opacity, darb_stream stream);

/* ---- Batched multi-view forward rendering ---------------------------------------------
 * Renders n_views cameras of one splat set: per view, steps 1-3 as darb_preprocess and
 * darb_bin_sort (DARB_SORT_DEPTH_THEN_TILE, asynchronous capacity mode); then step 4 for every
 * view in one persistent launch whose CTAs take (view, tile) items from a device work queue.
 * Views are spread round-robin over `depth` streams (created once per device by the library,
 * joined back into `stream`) so that the preprocessing and sorting of several views overlap.
 * A call neither allocates nor synchronises with the host, so a batch can be captured into a
 * CUDA graph on `stream` (make one call before capturing: the first call on a device creates
 * its streams).  Calls for one device are enqueued one at a time (a per-device lock).
 * Results per view are those of the single-view calls with the same camera, tile and kernel. */
#define DARB_MAX_BATCH_VIEWS 4096

typedef struct {
    int32_t n_views;   /* 1 .. DARB_MAX_BATCH_VIEWS */
    int32_t tile;      /* 8, 16 or 32, shared by all views */
    int32_t depth;     /* streams with views in flight, 1 .. 8 */
    int32_t max_ctas;  /* cap on the persistent launch's CTAs; 0 = SMs x resident CTAs */
    uint64_t capacity; /* instance capacity of each view */
} darb_batch_params;

/* Workspace bytes for darb_render_batch.  cams: host array [n_views]. */
darb_status darb_render_batch_workspace_size(int32_t n, const darb_camera *cams,
                                             const darb_batch_params *params, size_t *bytes);

/* cams: host array [n_views] (read during the call only).  outs: host array [n_views] of
 * device image buffers; image is required, t_final / last / n_contrib may be NULL (then not
 * written).  workspace: device, at least the queried size; it holds every view's projected
 * splats and sorted instances until the call's work completes.  num_instances, status: device
 * u32[n_views] or NULL: each view's instance count M and darb_bin_sort status word.  A view
 * with M > capacity has status DARB_ERR_CAPACITY and renders as background only; rerun it
 * with a larger capacity. */
darb_status darb_render_batch(const darb_splats *splats, const darb_camera *cams,
                              const darb_kernel_params *kparams, const darb_batch_params *params,
                              void *workspace, size_t workspace_bytes, const darb_image *outs,
                              uint32_t *num_instances, uint32_t *status, darb_stream stream);

/* ---- Serving ----------------------------------------------------------------------------
 * A server renders requests (scene, camera, kernel) against resident splat sets on the device
 * that is current at create time.  darb_serve_create allocates the server's whole device pool
 * once (scene_bytes for splat sets plus workspace_bytes split evenly over `slots` batch slots)
 * and starts a worker thread; nothing is allocated afterwards.  The worker batches
 * continuously: whenever a slot is free it takes pending requests in arrival order while their
 * workspace fits the slot (at most max_batch), renders them with darb_render_batch (one call
 * per scene and kernel, the calls of a batch on up to four streams of the slot so that they
 * overlap), and completes their tickets when the batch's work has finished.  Every slot has
 * its own stream, so a batch formed while others render is enqueued at once and its work
 * overlaps theirs on the device; batches retire in whatever order they finish.  A request's
 * instance capacity is capacity_per_pixel x W x H until its scene has been rendered, then the
 * scene's largest instances-per-pixel ratio so far x capacity_margin (at least capacity_min);
 * a view that still overflows is re-queued once, at the head, with the capacity its instance
 * count asks for.  The paper describes no serving system; this is the batched forward path of
 * Sec. 4 behind a request queue. */
typedef struct darb_server darb_server;

#define DARB_MAX_SERVE_SLOTS 8

typedef struct {
    uint64_t scene_bytes;      /* device bytes for resident splat sets */
    uint64_t workspace_bytes;  /* device bytes for the batch slots (an equal share each) */
    int32_t tile;              /* 8, 16 or 32 */
    int32_t max_batch;         /* requests per batch, 1 .. DARB_MAX_BATCH_VIEWS */
    int32_t depth;             /* darb_batch_params.depth of each batch, 1 .. 8 */
    float capacity_per_pixel;  /* first capacity guess, instances per pixel (> 0) */
    float capacity_margin;     /* factor on the observed ratio (>= 1) */
    uint64_t capacity_min;     /* lower bound of any capacity (>= 1) */
    int32_t slots;             /* batches in flight at once, 1 .. DARB_MAX_SERVE_SLOTS (0: 2) */
} darb_serve_cfg;

typedef struct {
    int32_t scene_id;   /* from darb_serve_add_scene */
    int32_t kernel;     /* one of the seven fixed darb_kernel kinds, with its darb_kernel_defaults
                           parameters (a DARB_GENERIC member is not served: DARB_ERR_INVALID_ARG) */
    darb_camera cam;
    float *image;       /* device [3][H][W], caller-owned, written by the server; keep it alive and
                           unread until the ticket completes */
} darb_request;

typedef struct {
    int32_t status;          /* DARB_OK or why the request failed */
    uint32_t num_instances;  /* M of the final attempt */
    uint32_t attempts;       /* 1, or 2 after a capacity retry */
    uint32_t batch_size;     /* requests in the batch that rendered it */
    double queue_us;         /* submit -> batch enqueued */
    double latency_us;       /* submit -> image complete, as seen by the worker */
    uint64_t batch_id;       /* 1, 2, ... in the order batches were enqueued (0: never enqueued) */
    double gpu_begin_us;     /* device time at which the batch's slot stream began it ... */
    double gpu_end_us;       /* ... and finished it, both since the server was created */
} darb_result;
/* DARB_ERR_CUDA if the pool cannot be allocated. */
darb_status darb_serve_create(const darb_serve_cfg *cfg, darb_server **server);

/* Copies a splat set (device pointers, as for darb_preprocess) into the scene region;
 * synchronous.  DARB_ERR_ADMISSION when the region is full. */
darb_status darb_serve_add_scene(darb_server *server, const darb_splats *splats, int32_t *scene_id);

/* Queues a request; returns at once with its ticket.  DARB_ERR_NOT_FOUND for an unknown
 * scene, DARB_ERR_ADMISSION if its workspace exceeds a batch slot even alone. */
darb_status darb_serve_submit(darb_server *server, const darb_request *request, uint64_t *ticket);

/* Queues count requests under one hold of the server's queue, in order, so the worker sees
 * them together (for instance the views of one camera path): tickets[k] is request k's ticket.
 * Stops at the first request that fails (same errors as darb_serve_submit) and returns its
 * status; *submitted is the number queued before it, whose tickets stay valid. */
darb_status darb_serve_submit_many(darb_server *server, const darb_request *requests, int32_t count,
                                   uint64_t *tickets, int32_t *submitted);

/* Waits up to timeout_ms for a ticket.  On DARB_OK the result is stored and the ticket is
 * released; DARB_ERR_TIMEOUT leaves it pending; DARB_ERR_NOT_FOUND for an unknown or already
 * collected ticket. */
darb_status darb_serve_poll(darb_server *server, uint64_t ticket, int32_t timeout_ms, darb_result *result);

/* Finishes every queued and in-flight request, stops the worker and frees the pool. */
void darb_serve_destroy(darb_server *server);

#ifdef __cplusplus
}
#endif

#endif /* DARB_H */
