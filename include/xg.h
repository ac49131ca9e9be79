/*
 * xg.h -- C ABI of the GB300 (sm_103a) radiative Gaussian rasterizer.
 *
 * The library renders X-ray projections of 3-D Gaussians and differentiates them: the
 * Differentiable Radiative Rasterization of X-Gaussian (arXiv 2403.04116, Sec. 3.2,
 * Eq. 5-10), with the cone-beam camera built from the scanner parameters of Sec. 3.3,
 * Eq. 12.  A frame holds one batch of views that share a detector size; the four stages
 * run as stream-ordered launches over every view of the frame at once:
 *
 *     xg_project    -> xg_bin_sort -> xg_render_fwd          (forward, Eq. 7-10)
 *                                  -> xg_render_bwd          (gradients to every parameter)
 *
 * Conventions shared by every call
 *   - Device pointers are CUDA device addresses of the current device; host pointers are
 *     ordinary process memory.  Every array is dense, C order, FP32 unless stated.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - The caller owns every buffer, including the frame's device workspace.  The library
 *     never allocates or frees device memory and never synchronises, except
 *     xg_frame_read_status, which waits for `stream`.  The stage calls contain only kernel
 *     launches and cudaMemsetAsync, so a sequence of them can be captured in a CUDA graph.
 *   - Argument errors are returned at once, before anything is enqueued.  Conditions met on
 *     the device (pair capacity exceeded) are recorded in a status word in the workspace;
 *     after one, the later stages of the frame write zeros.  Read it with
 *     xg_frame_read_status.  Gaussians with a non-finite attribute are skipped and counted.
 *
 * Gaussians (Sec. 3.1, Eq. 1-4) are structure-of-arrays, activated values:
 *   mean[3][n] (mm, world frame whose origin is the rotation centre), scale[3][n] (mm, > 0),
 *   quat[4][n] ((w, x, y, z), any non-zero norm; normalised inside), opacity[n] (the
 *   paper's alpha_i, in [0, 1]), intensity[n] (the radiation intensity i of Eq. 3).
 *
 * Readings of the paper used by the kernels: focal length in pixels L_SD / pitch; pixel
 * (x, y) samples the detector at (x + 1/2, y + 1/2) with the principal point at (W/2, H/2);
 * Sigma'' gets 0.3 px^2 added on its diagonal; Gaussians with t_z <= near_mm are skipped;
 * the opacity of Eq. 10 is sigma = min(0.99, alpha * density) and terms with sigma < 1/255
 * are skipped; blending stops before a term that would take the transmittance below 1e-4;
 * depth order is ascending t_z, ties by ascending Gaussian index; background 0.
 */
#ifndef XG_H
#define XG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  XG_OK = 0,
  XG_ERR_INVALID_ARG = 1, /* a pointer, size or geometry argument is unusable */
  XG_ERR_CAPACITY = 2,    /* the frame's (view, tile, Gaussian) pairs exceed pair_capacity */
  XG_ERR_CUDA = 3,        /* a CUDA launch or copy failed; see cudaGetLastError */
  XG_ERR_WORKSPACE = 4,   /* the workspace is too small or misaligned */
  XG_ERR_CHECK = 5        /* a device-side bounds check failed, or a bounded wait in a kernel expired
                             (a library or device defect, or the XG_SPIN_LIMIT fault injection:
                             that environment variable, read once per process, caps the
                             kernels' first waits, 0 making every one expire); outputs invalid */
} xg_status;

/* One cone-beam projection (Sec. 3.3, Eq. 12).  The source orbits at distance sod_mm from
 * the rotation centre in the z = 0 plane at azimuth angle_rad (elevation 0); the detector
 * is sdd_mm from the source, width x height pixels of pitch_u_mm x pitch_v_mm. */
typedef struct {
  double sod_mm;     /* L_SO, > 0 */
  double sdd_mm;     /* L_SD, > 0 */
  double pitch_u_mm; /* detector pixel width, > 0 */
  double pitch_v_mm; /* detector pixel height, > 0 */
  double angle_rad;  /* azimuth phi of Eq. 9 and 12 */
  int32_t width;     /* W, 1 .. 4096 */
  int32_t height;    /* H, 1 .. 4096 */
} xg_view;

/* Device arrays of n Gaussians (see above).  n >= 1. */
typedef struct {
  const float* mean;
  const float* scale;
  const float* quat;
  const float* opacity;
  const float* intensity;
  int64_t n;
} xg_gaussians;

/* Device arrays receiving dL/d(parameter), same shapes as xg_gaussians; overwritten. */
typedef struct {
  float* mean;
  float* scale;
  float* quat;
  float* opacity;
  float* intensity;
} xg_grads;

/* Frame configuration.  tile_w, tile_h in {8, 16, 32}; pixels_per_thread: pixels each
 * compositing thread owns, 1, 2 or 4 (0 selects 2), with tile_h a multiple of
 * 4 * pixels_per_thread and tile_w * tile_h <= 512 * pixels_per_thread; near_mm > 0;
 * batch: list entries (Gaussians) whose records each warp of the compositing kernels keeps
 * in flight into shared memory, one of 64, 128, 256, 512 (0 selects 64); the shared memory
 * this needs must fit one block (XG_ERR_INVALID_ARG otherwise); 1 <= pair_capacity < 2^31
 * (pairs of one pass).  views_per_pass >= 0: views the per-pass arrays hold; 0, or a value
 * >= the frame's view count, renders every view in one pass.  A smaller value renders a
 * long scan in passes through one workspace (see xg_frame_select_views).  persistent: 0
 * launches the compositing kernels with one block per (view, tile); 1 launches as many
 * blocks as fit on the device at once, whose warps take (view, tile, pixel block) work
 * items from a counter in the workspace, longest tile lists first.  Tile shape, batch,
 * pixels per thread, views per pass and the launch form change speed and memory only:
 * images and gradients do not depend on them. */
typedef struct {
  int32_t tile_w;
  int32_t tile_h;
  float near_mm;
  int32_t batch;
  int64_t pair_capacity;
  int32_t pixels_per_thread;
  int32_t views_per_pass;
  int32_t persistent;
  int32_t reserved;  /* 0 */
} xg_config;

/* Device-side status of a frame, read back by xg_frame_read_status. */
typedef struct {
  int32_t code;      /* XG_OK, XG_ERR_CAPACITY or XG_ERR_CHECK */
  int32_t reserved;
  int64_t pairs;     /* (view, tile, Gaussian) pairs of the last xg_bin_sort */
  int64_t nonfinite; /* Gaussians skipped for a non-finite attribute, summed over xg_project calls */
  /* work done since the last xg_bin_sort, for throughput accounting: (pixel, list entry)
   * pairs whose opacity was evaluated, and how many of them contributed */
  int64_t fwd_evaluated, fwd_contrib;
  int64_t bwd_evaluated, bwd_contrib;
} xg_device_status;

/* Byte offsets, inside the workspace, of the frame's intermediate arrays (for inspection).
 * V views of the current pass, n Gaussians, T tiles per view, cap = pair_capacity; the
 * camera table (at `cameras`) holds every view of the frame:
 *   records    float[V*n][8]  (u_x, u_y, -a/2, -b, -c/2, opacity, intensity, thr): (a, b, c)
 *                             the conic, so the exponent at pixel offset d = u - p is
 *                             (-a/2) dx^2 + (-b) dx dy + (-c/2) dy^2; thr = -ln(255 opacity)
 *                             - 1e-4, below which the opacity stays under 1/255; u centred
 *                             on the principal point; zero where the Gaussian touches no tile
 *   depth      float[V*n]     t_z (0 where it touches no tile)
 *   rect       uint16[V*n][4] tile rectangle (x0, y0, x1, y1), inclusive
 *   count      uint32[V*n]    tiles touched
 *   value      uint32[cap]    the (view, tile, Gaussian) pairs as Gaussian indices, ordered
 *                             by (tile, view, t_z, index): every (view, tile) list is
 *                             contiguous and in depth order (the first `pairs` are valid)
 *   range      uint32[V*S][2] [start, end) in `value` of (view, tile) at view * S + tile,
 *                             S = range_stride, the power of two >= T ([0, 0) if the list
 *                             is empty or tile >= T)
 *   tfinal     float[V][H][W] transmittance after the last contributor
 *   last       uint32[V][H][W] 1-based position in the tile's list of the last contributor
 *   grad2d     float[V*n][8]  per (view, Gaussian): dL/du_x, dL/du_y, dL/da, dL/db, dL/dc,
 *                             dL/dopacity, dL/dintensity, 0 (written by xg_render_bwd)
 *   order      uint32[V*T]    the compositing work items, view * T + tile, by descending
 *                             bucket of list length (four buckets per octave; the order
 *                             inside a bucket is unspecified), written by xg_bin_sort */
typedef struct {
  size_t status, cameras, records, depth, rect, count;
  size_t value, range, tfinal, last, grad2d;
  int64_t tiles_per_view;
  int32_t tiles_x, tiles_y;
  int32_t sort_passes;  /* radix passes over the V*n entries */
  int32_t range_stride; /* S: power of two >= tiles_per_view */
  size_t order;
} xg_layout;

typedef struct xg_frame xg_frame;

/* Bytes of device workspace a frame with these sizes needs (0 if the arguments are
 * invalid).  The workspace must be 256-byte aligned. */
size_t xg_workspace_bytes(const xg_config* cfg, int64_t n, int32_t n_views, int32_t width, int32_t height);

/* Create a frame for `n_views` views (host array, copied; every view must have the same
 * width and height) and n Gaussians, inside the caller's device workspace.  Enqueues on
 * `stream` the upload of the camera table and the clearing of the status word; the host
 * array may be reused as soon as the call returns.  The frame object itself is host memory
 * owned by the library; release it with xg_frame_destroy (the workspace stays the
 * caller's).  Errors: XG_ERR_INVALID_ARG, XG_ERR_WORKSPACE, XG_ERR_CUDA. */
xg_status xg_frame_create(xg_frame** out, const xg_config* cfg, int64_t n, const xg_view* views, int32_t n_views,
                          void* workspace, size_t workspace_bytes, void* stream);
void xg_frame_destroy(xg_frame* frame);

/* Select the views of the next pass: views first_view .. first_view + V - 1 of the frame,
 * V = min(views_per_pass, n_views - first_view), written to *n_selected (may be NULL).
 * A new frame has views 0 .. views_per_pass - 1 selected.  The selection is host state
 * only: it enqueues nothing, so it can sit between graph-captured calls, and it governs
 * the calls made after it (their view index v, image planes and arrays run over the V
 * selected views; xg_render_bwd sums over them only).  Calls already enqueued are not
 * affected.  Errors: XG_ERR_INVALID_ARG (first_view outside [0, n_views)). */
xg_status xg_frame_select_views(xg_frame* frame, int32_t first_view, int32_t* n_selected);

/* Project every Gaussian into every view of the frame (Eq. 7-9 and the 2-D covariance of
 * Sec. 3.2: t = M_ext mu, u = M_int t, Sigma' = J W Sigma W^T J^T, Sigma'' its top-left
 * block, Sigma = R S S^T R^T of Sec. 3.1) and find the tiles its footprint touches.  Writes
 * the frame's records, depth, rect and count arrays.  `g` must have the frame's n. */
xg_status xg_project(xg_frame* frame, const xg_gaussians* g, void* stream);

/* Tile binning and the depth order (Sec. 3.2).  Orders the (view, Gaussian) entries by
 * (view, t_z) with a stable LSD radix sort, counts the pairs every run of sorted entries
 * puts on every tile, turns the counts into positions, and writes one pair per touched tile
 * straight to its place in `value`, with each (view, tile) range: every list is in
 * ascending t_z, ties by ascending Gaussian index.  Sets XG_ERR_CAPACITY in the device
 * status (and leaves every list empty) if the pairs exceed pair_capacity. */
xg_status xg_bin_sort(xg_frame* frame, void* stream);

/* Front-to-back alpha compositing of intensity per detector pixel (Eq. 10).
 *   image      device float[V][H][W], written
 *   n_contrib  device uint32[V][H][W] contributor counts, written; may be NULL */
xg_status xg_render_fwd(xg_frame* frame, float* image, uint32_t* n_contrib, void* stream);

/* Gradients of L = sum_{v,p} grad_image[v][p] * image[v][p] with respect to every
 * Gaussian parameter, for the image of the last xg_render_fwd of this frame (the frame's
 * records, sorted pairs, tfinal and last must be unchanged since).  The compositing is
 * walked back to front, the transmittance recovered by division rather than stored.
 *   g          the same device Gaussians as xg_project
 *   grad_image device float[V][H][W]
 *   out        device gradient arrays, overwritten (sum over the frame's views) */
xg_status xg_render_bwd(xg_frame* frame, const xg_gaussians* g, const float* grad_image, const xg_grads* out,
                        void* stream);

/* Wait for `stream`, then copy the frame's device status to *out.  Returns XG_OK if the
 * copy worked (the device-side code is in out->code), else XG_ERR_CUDA. */
xg_status xg_frame_read_status(const xg_frame* frame, xg_device_status* out, void* stream);

/* Enqueue on `stream` a copy of the frame's device status, in the xg_device_status layout,
 * to device memory `out` (8-byte aligned, caller-owned).  It does not synchronise, so it
 * can be graph-captured, e.g. to keep the status of every pass of a scan rendered in
 * passes.  Errors: XG_ERR_INVALID_ARG, XG_ERR_CUDA. */
xg_status xg_frame_copy_status(const xg_frame* frame, xg_device_status* out, void* stream);

/* Byte offsets of the frame's arrays inside its workspace. */
xg_status xg_frame_layout(const xg_frame* frame, xg_layout* out);

/* The FP32 exponential the compositing kernels use in their opacity decisions (Cody-Waite
 * reduction by ln 2, degree-6 polynomial, argument clamped at -80), evaluated on the device
 * in its scalar form into y_scalar and in its two-lane packed form into y_packed, for tests
 * that hold both to an independent implementation bit for bit.  x, y_scalar, y_packed:
 * device float[n].  Errors: XG_ERR_INVALID_ARG (null pointer, n < 1 or n > 2^38), XG_ERR_CUDA. */
xg_status xg_exp_check(const float* x, float* y_scalar, float* y_packed, int64_t n, void* stream);

/* L1 term of the training objective (Eq. 11):
 *   *loss = scale * sum_i |image[i] - target[i]|,  grad[i] = scale * sign(image[i] - target[i])
 * image, target, grad: device float[count]; loss: one device float, overwritten.  Use
 * scale = 1 / count for the mean.  Not tied to a frame. */
xg_status xg_loss_l1(const float* image, const float* target, int64_t count, float scale, float* grad, float* loss,
                     void* stream);

/* Per-kernel timing of a frame's launches.  While enabled, every launch the frame's stage
 * calls make is bracketed by CUDA events recorded on the launch stream (up to 2048
 * launches between reads; further launches are not timed).  Keep it disabled while a
 * stream is being captured into a CUDA graph. */
typedef struct {
  char name[32];     /* kernel name, e.g. "k_render_fwd" ("memset" for cudaMemsetAsync) */
  int64_t launches;
  double total_ms;   /* summed event-to-event time */
} xg_kernel_time;

xg_status xg_frame_set_timing(xg_frame* frame, int32_t enable);

/* Wait for the recorded events, write one entry per kernel that ran (at most `capacity`)
 * and the number written to *count, and start a new accumulation. */
xg_status xg_frame_read_timing(xg_frame* frame, xg_kernel_time* out, int32_t capacity, int32_t* count);

/* ------------------------------------------------------------------------------------ */
/* The rest of a training step (Sec. 3.1, Eq. 3 and 11; implementation details of Sec. 4.1) */
/* ------------------------------------------------------------------------------------ */

/* Learnable parameters that are activated before projection (mean and quaternion are used
 * as they are).  Device arrays: log_scale[3][n], opacity_logit[n], features[n_features][n]
 * (the feature vector f of Eq. 3), lambda[n_features] (the constant weights of Eq. 3).
 * 1 <= n_features <= 64. */
typedef struct {
  const float* log_scale;
  const float* opacity_logit;
  const float* features;
  const float* lambda;
  int32_t n_features;
  int32_t reserved;
  int64_t n;
} xg_raw_gaussians;

/* Activations of the radiative Gaussian model: scale = exp(log_scale), opacity =
 * sigmoid(opacity_logit), and the radiation intensity response function (Eq. 3),
 * intensity = sigmoid(sum_k lambda_k f_k) -- the weights applied as an inner product.
 * Writes device scale[3][n], opacity[n], intensity[n]. */
xg_status xg_activate(const xg_raw_gaussians* raw, float* scale, float* opacity, float* intensity, void* stream);

/* Chain rule of xg_activate: from dL/dscale[3][n], dL/dopacity[n], dL/dintensity[n] (as
 * xg_render_bwd writes them) to dL/dlog_scale[3][n], dL/dopacity_logit[n],
 * dL/dfeatures[n_features][n] (overwritten). */
xg_status xg_activate_bwd(const xg_raw_gaussians* raw, const float* g_scale, const float* g_opacity,
                          const float* g_intensity, float* g_log_scale, float* g_opacity_logit, float* g_features,
                          void* stream);

/* Device workspace bytes of xg_loss_l1_ssim for n_views images of width x height. */
size_t xg_loss_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/* Training objective of Eq. 11 over n_views images: loss = (1 - gamma) * mean |I - I*| +
 * gamma * (1 - mean SSIM(I, I*)), SSIM with the 11-tap Gaussian window of sigma 1.5, zero
 * padding, C1 = 0.01^2, C2 = 0.03^2 (intensities in [0, 1]); the mean runs over all pixels
 * of all views.  grad[V][H][W] receives dloss/dI; loss (3 device floats) receives the
 * loss, the mean L1 and the mean SSIM.  The workspace (16-byte aligned) is scratch. */
xg_status xg_loss_l1_ssim(const float* image, const float* target, int32_t n_views, int32_t width, int32_t height,
                          float gamma, float* grad, float* loss, void* workspace, size_t workspace_bytes,
                          void* stream);

/* One Adam step (Sec. 4.1) over up to XG_ADAM_MAX_GROUPS parameter groups.  Each group:
 * device param, grad, first and second moments m, v (count floats each, updated in place),
 * the learning rate lr, and, when decay_steps > 0, an exponential decay from lr to lr_final
 * over decay_steps steps.  step points to a device int32 holding the number of steps
 * taken so far; the call uses it for bias correction and the schedule and increments it,
 * so a captured step can be replayed. */
#define XG_ADAM_MAX_GROUPS 8
typedef struct {
  float* param;
  const float* grad;
  float* m;
  float* v;
  int64_t count;
  float lr;
  float lr_final;
  int32_t decay_steps;
  int32_t reserved;
} xg_adam_group;

xg_status xg_adam_step(const xg_adam_group* groups, int32_t n_groups, int32_t* step, float beta1, float beta2,
                       float eps, void* stream);

/* Peak signal-to-noise ratio (peak 1) of each of n_views images of pixels_per_view pixels:
 * psnr[v] = -10 log10(mean (I - I*)^2) (device floats, overwritten). */
xg_status xg_psnr(const float* image, const float* target, int32_t n_views, int64_t pixels_per_view, float* psnr,
                  void* stream);

/* ACUI initialisation of the Gaussian centres (Sec. 3.3, Eq. 13).  A cuboid of
 * size_mm[0] x size_mm[1] x size_mm[2] mm centred on the origin is divided into
 * grid[0] x grid[1] x grid[2] voxels; the centres are the points
 * (n_1 S_1 d / M_1, n_2 S_2 d / M_2, n_3 S_3 d / M_3) for integers n_i with
 * |n_i| <= floor(M_i / (2 d)) + 1 (the bracket of Eq. 13 read as the floor), d = interval
 * in voxels (the paper takes d = 8).
 *
 * xg_acui_count returns the number of points (0 for invalid arguments: sizes not finite
 * and positive, grid < 1, interval not finite and positive, or 2^31 points or more). */
int64_t xg_acui_count(const double size_mm[3], const int32_t grid[3], double interval);

/* Writes the points to `mean` (device, float[3][count], rows x, y, z), n_1 slowest and
 * n_3 fastest, each ascending; every coordinate is ((n S) d) / M in FP64 rounded once to
 * FP32.  size_mm and grid are host arrays.  Enqueued on `stream`.  Errors:
 * XG_ERR_INVALID_ARG, XG_ERR_CAPACITY (count > capacity floats per row), XG_ERR_CUDA. */
xg_status xg_acui_points(const double size_mm[3], const int32_t grid[3], double interval, float* mean,
                         int64_t capacity, void* stream);

/* Adaptive density control.  The paper adjusts the number of Gaussians with the adaptive
 * control of 3D Gaussian splatting (Sec. 3.2) without restating it; these calls follow that
 * method's published rules.  Parameters are raw: centres, log-scales, quaternions, opacity
 * logits and features, device SoA [3][n], [3][n], [4][n], [n], [n_features][n].  The same
 * layout carries Adam's first and second moments. */
typedef struct {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* features;
  int32_t n_features;
  int32_t reserved; /* set to 0 */
  int64_t n;
} xg_param_set;

/* Densify where accum / denom >= grad_thresh (FP32 division; never where denom = 0): a
 * Gaussian whose largest log-scale is <= size_log_thresh is cloned (an identical copy),
 * a larger one is split into two with centres mu + R diag(s) z_k and log-scales reduced by
 * ln 1.6.  Prune where the opacity logit < prune_logit or the largest log-scale >
 * max_log_size (INFINITY: never); children are tested with their own log-scales.  All
 * comparisons are in FP32, none may be NaN. */
typedef struct {
  float grad_thresh;
  float size_log_thresh;
  float prune_logit;
  float max_log_size;
} xg_density_rules;

/* Adds, for every Gaussian and every view of the frame's current pass in which it touches
 * a tile, scale * |dL/du| (the projected-centre gradient written by the last xg_render_bwd)
 * to accum[n] and 1 to denom[n] (device arrays, accumulated, not overwritten).  Enqueued on
 * `stream`; graph-capturable.  Errors: XG_ERR_INVALID_ARG, XG_ERR_CUDA. */
xg_status xg_densify_stats(xg_frame* frame, float scale, float* accum, int32_t* denom, void* stream);

/* Device scratch bytes xg_densify_plan needs on the current device (one partial count
 * per CTA of its scan, 4 CTAs per SM). */
size_t xg_densify_workspace_bytes(void);

/* The plan: offsets[g] (device, n + 1 entries) = first output slot of Gaussian g in the
 * order [g if kept], [its clone], [child 0, child 1]; offsets[n] = the new count.  The
 * caller reads offsets[n] to size the outputs of xg_densify_apply.  Requires 1 <= n <= 2^30.
 * Errors: XG_ERR_INVALID_ARG, XG_ERR_CUDA. */
xg_status xg_densify_plan(const xg_param_set* params, const float* accum, const int32_t* denom,
                          const xg_density_rules* rules, uint32_t* offsets, void* workspace, void* stream);

/* Writes the new parameters and Adam moments (out_* with n = offsets[n], same
 * n_features): kept Gaussians keep their moments, clones and children start from zero
 * moments.  normals: device [2][3][n] standard-normal samples z_k (drawn by the caller).
 * Inputs and outputs must not overlap.  With a new count of 0 the outputs may be empty
 * (NULL pointers) and nothing is written.  Errors: XG_ERR_INVALID_ARG, XG_ERR_CUDA. */
xg_status xg_densify_apply(const xg_param_set* params, const xg_param_set* adam_m, const xg_param_set* adam_v,
                           const float* accum, const int32_t* denom, const xg_density_rules* rules,
                           const uint32_t* offsets, const float* normals, const xg_param_set* out_params,
                           const xg_param_set* out_m, const xg_param_set* out_v, void* stream);

/* Opacity reset: opacity_logit[g] = min(opacity_logit[g], reset_logit) (device, in place),
 * and the opacity logits' Adam moments adam_m[n], adam_v[n] set to zero (either may be
 * NULL).  Errors: XG_ERR_INVALID_ARG, XG_ERR_CUDA. */
xg_status xg_opacity_reset(float* opacity_logit, float* adam_m, float* adam_v, int64_t n, float reset_logit,
                           void* stream);

/* FDK reconstruction (Feldkamp, Davis, Kress) of a volume from projections of a full
 * circular scan: the paper's downstream use of rendered views (Sec. 4, Table 2).  Views
 * are evenly spaced over 2 pi and share one scanner (only the angle changes).  Steps:
 * P_w = P L_SO / sqrt(L_SO^2 + p^2 + zeta^2) at pixel centres scaled to the rotation axis
 * (tau = pitch L_SO / L_SD); Q = tau (h * P_w) along each detector row with the ramp kernel
 * h[0] = 1 / (4 tau^2), h[n odd] = -1 / (pi^2 n^2 tau^2); f(mu) = (pi / V) sum_v U^2 Q_v
 * at mu's projection (bilinear, zero off the detector), U = L_SO / t_z.  The volume is
 * [nz][ny][nx] floats, voxel (i, j, k) centred at ((i + 1/2 - nx/2) s, (j + 1/2 - ny/2) s,
 * (k + 1/2 - nz/2) s) mm, s = voxel_mm. */
typedef struct {
  int32_t nx, ny, nz;
  int32_t reserved; /* set to 0 */
  double voxel_mm;
} xg_volume;

/* Device workspace bytes of xg_fdk (0 for invalid sizes); 256-byte aligned. */
size_t xg_fdk_workspace_bytes(int32_t n_views, int32_t width, int32_t height);

/* views: host array of n_views; projections: device [n_views][H][W]; volume: device,
 * overwritten.  Enqueued on `stream` (the camera constants are uploaded from host memory,
 * so the call is not graph-capturable).  Errors: XG_ERR_INVALID_ARG, XG_ERR_WORKSPACE,
 * XG_ERR_CUDA. */
xg_status xg_fdk(const xg_view* views, int32_t n_views, const float* projections, const xg_volume* vol,
                 float* volume, void* workspace, size_t workspace_bytes, void* stream);

/* Largest pair count xg_sort_pairs_noalloc accepts. */
#define XG_NOALLOC_MAX_PAIRS (1 << 20)

/* Allocation-free pair sort.  The paper has no counterpart of this call: it is the stable
 * radix sort inside xg_bin_sort, offered on its own to callers that cannot allocate device
 * memory -- plugins hosted by an application that owns the GPU's memory pool, and
 * real-time pipelines that forbid allocation after start-up (cudaMalloc can synchronise
 * the device and takes unbounded time).  Such callers could not provide xg_bin_sort's
 * workspace.
 *
 * Sorts `count` (key_tile, key_depth, value) triples stably by key_tile, then key_depth,
 * into out_key_tile, out_key_depth, out_value (all device uint32[count]; the outputs must
 * not overlap the inputs).  Only the low `tile_bits` bits of key_tile may be non-zero
 * (0 <= tile_bits <= 32).  Given the pairs xg_bin_sort emits, the output equals its
 * sorted pairs.
 *
 * Scratch: a static device array of about 12.6 MB inside the library (ping-pong buffers
 * for XG_NOALLOC_MAX_PAIRS pairs, digit histograms, the pair count), held by every GPU that
 * loads the library until the process exits.  The call allocates nothing and frees
 * nothing.  Each call made outside a stream capture looks up the array's device address
 * on the current device (so the address stays valid across cudaDeviceReset); a call made
 * inside a capture reuses the address of the last call outside one, so make a first call
 * on each device before capturing (XG_ERR_CUDA otherwise).  All calls on a device share
 * the array and the last call's contents stay in it: calls whose work overlaps on the GPU
 * (different streams without ordering between them) race and give wrong results; order
 * them on one stream.
 *
 * Errors: XG_ERR_INVALID_ARG if count < 0, count > XG_NOALLOC_MAX_PAIRS, tile_bits is out
 * of range or a pointer is NULL (nothing is enqueued); XG_ERR_CUDA if the address lookup
 * or a launch fails.  count == 0 enqueues nothing.  Failures on the device (a position
 * outside its segment, a bounded wait that gave up) do not reach the return code, which
 * is known before the kernels run: they are recorded in the array's status word, which
 * xg_sort_pairs_noalloc_status reads. */
xg_status xg_sort_pairs_noalloc(const uint32_t* key_tile, const uint32_t* key_depth, const uint32_t* value,
                                int64_t count, int32_t tile_bits, uint32_t* out_key_tile, uint32_t* out_key_depth,
                                uint32_t* out_value, void* stream);

/* Device-side outcome of the last xg_sort_pairs_noalloc on the current device (no
 * counterpart in the paper; it completes the allocation-free sort above).  Waits for
 * `stream` (the stream the sort ran on), then writes to *device_code XG_OK, or
 * XG_ERR_CHECK when a radix pass recorded a failed bounds check or a bounded wait that
 * gave up (the output is then not sorted).  Allocates nothing.  Each sort call starts
 * from XG_OK.  Returns XG_ERR_INVALID_ARG for a NULL device_code, XG_ERR_CUDA if the
 * synchronisation or the read fails. */
xg_status xg_sort_pairs_noalloc_status(void* stream, int32_t* device_code);

/* Measurement aid, no counterpart in the paper: the FP32 pipe's peak rate, the roofline
 * denominator of the compositing kernels (no stage is a dense contraction).  Enqueues on
 * `stream` one launch of 8 CTAs of 256 threads per SM of the current device, each thread
 * running `iters` rounds of 8 independent fused multiply-add chains: scalar FFMA
 * (packed = 0) or two-lane packed FFMA (packed = 1).  *lane_ops (host) receives the FP32
 * multiply-adds the launch performs (a packed one counts two); time the launch with CUDA
 * events on `stream`.  `sink` (device, one float) is written only for inputs that never
 * occur.  Errors: XG_ERR_INVALID_ARG (NULL pointer, iters < 1, packed not 0 or 1),
 * XG_ERR_CUDA. */
xg_status xg_fp32_peak(int32_t packed, int32_t iters, float* sink, int64_t* lane_ops, void* stream);

/* Text for a status code (static storage). */
const char* xg_status_str(xg_status s);

#ifdef __cplusplus
}
#endif

#endif /* XG_H */
