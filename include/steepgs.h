/*
 * steepgs.h -- C ABI of the GB300 (sm_103a) SteepGS splitting path.
 *
 * The path follows "Steepest Descent Density Control for Compact 3D Gaussian
 * Splatting" (arXiv 2505.05587):
 *   sgs_project                    Section 3, Eq. sigma_3D / sigma_2D and the
 *                                  affine-projection footnote: EWA projection.
 *   sgs_bin_sort                   Section 3 ("sorts points according to
 *                                  view-dependent depth"): tile binning and
 *                                  (tile, depth) radix sort.
 *   sgs_render_fwd                 Section 3, Eq. alpha_blend.
 *   sgs_l1_loss_grad               Section 3, Eq. loss with the L1 error.
 *   sgs_render_bwd_with_splitting  Section 4.4 and Algorithm 1 (accumulate
 *                                  gradients and S^(i) = E[dl/dsigma Hess sigma])
 *                                  with the Appendix's closed-form Hessian.
 *   sgs_densify_split              Theorem 2, Algorithm 1 and the Appendix
 *                                  "Eigendecomposition": minimum eigenpair of
 *                                  S/T_split, split into p +- eps v_min with
 *                                  opacity o/2, prefix-sum compaction.
 *
 * Conventions shared by every call
 *   - Every array pointer is a DEVICE pointer owned by the caller, unless a
 *     field says otherwise.  The library never allocates device memory: scratch
 *     comes from a caller workspace sized by the matching *_workspace_size.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) and returns an int status (SGS_OK or an SGS_ERR_*
 *     code).  Argument errors are detected on the host before any launch and
 *     leave every output untouched.  SGS_ERR_CUDA means a launch failed; the
 *     CUDA error code is kept for sgs_get_last_cuda_error().
 *   - Every call that launches work is capture-safe: it allocates nothing,
 *     synchronises nothing and reads nothing back to the host, so a sequence
 *     of calls can be captured into a CUDA graph and replayed (the
 *     allocation-free variant's first call on a device is the exception, see
 *     sgs_densify_split_noalloc).  Kernels are launched with programmatic
 *     dependent launch: each one is scheduled while its predecessor on the
 *     stream drains and waits for that predecessor's results before reading.
 *   - Every call that launches work opens an NVTX range named after itself
 *     for the duration of the host call, so a profiler's timeline groups its
 *     launches; without a tool attached the range costs a pointer check.
 *   - Data-dependent sizes (instance count M, split count) are written to
 *     caller-owned device integers.  When a size exceeds the caller's capacity
 *     the kernels write only within capacity (never out of bounds) and the
 *     caller sees the overflow by comparing the count it reads back with the
 *     capacity it passed.
 *   - Layouts are structure-of-arrays, float32, row-major:
 *       means [N,3], log_scales [N,3], quats [N,4] as (w,x,y,z) (need not be
 *       unit: the rotation uses q/|q|), opacity_logit [N] (opacity =
 *       sigmoid), sh [N,K,3] with K = (sh_degree+1)^2 and sh_degree <= 3;
 *       images [H,W,3]; per-pixel maps [H,W].
 *   - Cameras: x_cam = R x_world + t, OpenCV axes (x right, y down, z
 *     forward), pinhole intrinsics fx, fy, cx, cy; pixel (px,py) is sampled at
 *     its integer coordinates.
 */
#ifndef STEEPGS_H
#define STEEPGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGS_OK 0
#define SGS_ERR_INVALID_ARG 1
#define SGS_ERR_WORKSPACE 2
#define SGS_ERR_CAPACITY 3
#define SGS_ERR_CUDA 4
#define SGS_ERR_TIMEOUT 5
#define SGS_ERR_UNSUPPORTED 6
/* Codes 3, 5 and 6 are reserved; no call of this version returns them: a
 * capacity overflow is reported through the data-dependent counts (see the
 * conventions above), no kernel waits on another agent (every loop is bounded
 * by its input sizes), and settings outside what the kernels handle are
 * argument errors (SGS_ERR_INVALID_ARG). */

/* Gaussian parameters theta^(i) = (p, Sigma via quaternion + log-scale, o, SH
 * colour) (Section 3, "Scene Representation").  Read-only input. */
typedef struct sgs_gaussians {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logit;
    const float *sh;
    int32_t n;
    int32_t sh_degree;
} sgs_gaussians;

/* Writable Gaussian arrays (output of sgs_densify_split), same layouts. */
typedef struct sgs_gaussians_mut {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logit;
    float *sh;
} sgs_gaussians_mut;

/* Pinhole camera, host struct passed by pointer (copied at the call). */
typedef struct sgs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;       /* Gaussians with camera z <= near_z are culled */
} sgs_camera;

/* Rasterisation constants, host struct passed by pointer.
 * tile_w x tile_h must be one of 16x16, 16x8, 8x8, 32x8.
 * alpha = min(alpha_max, o G); a pair is skipped when alpha < alpha_min; the
 * walk of a pixel stops before the Gaussian that would bring transmittance
 * below T_min; the support is the radius_sigma-sigma bounding square of the
 * 2-D covariance (dilated by `dilation` on its diagonal); the Jacobian's
 * tx/tz, ty/tz are clamped to +-fov_clamp * (W/2)/fx, (H/2)/fy. */
typedef struct sgs_settings {
    int32_t tile_w, tile_h;
    float alpha_min, alpha_max, T_min, radius_sigma, dilation, fov_clamp;
    float bg[3];
} sgs_settings;

/* Per-view projected state written by sgs_project, capacity >= n rows.
 *   xy          [N,4] (mu_x, mu_y, mu_x_lo, mu_y_lo): 2-D mean in pixels as an
 *               unevaluated float pair mu = hi + lo (about 44 bits).
 *   conic_opac  [N,4] (Q00, Q01, Q11, opacity), Q = Sigma2D^-1.
 *   rgb         [N,4] (r, g, b, 0) after the SH evaluation and the clamp at 0.
 *   depth       [N]   camera-space z, float32 (the depth sort key).
 *   rect        [N,4] int16 (x_lo, y_lo, x_hi, y_hi), inclusive tile rect;
 *               (0,0,-1,-1) for a culled Gaussian.
 *   tiles_touched [N] number of tiles in rect (0 = culled).
 * xy, conic_opac and rgb are written only for rows with tiles_touched > 0
 * (the only rows an instance refers to); depth, rect and tiles_touched for
 * every row. */
typedef struct sgs_proj {
    float *xy;
    float *conic_opac;
    float *rgb;
    float *depth;
    int16_t *rect;
    uint32_t *tiles_touched;
} sgs_proj;

/* Binned, sorted instances written by sgs_bin_sort.
 *   gids     [capacity]  Gaussian id of each (Gaussian, tile) instance, in
 *                        (tile id, float32 depth bits, Gaussian id) order.
 *   keys     [capacity]  optional (NULL to skip): (tile id << 32) | depth bits.
 *   ranges   [T,2]       per tile [start, end) into gids, T = tiles_x*tiles_y,
 *                        tile id = ty * tiles_x + tx.
 *   count    [1] int32   M, the number of instances (may exceed capacity).
 *   capacity             rows available in gids / keys (< 2^31).
 *   order    [T]         optional (NULL to skip): every tile id once, longest
 *                        lists first (list length in quarter octaves:
 *                        classes of the leading three bits, descending;
 *                        empty tiles last; ties by tile id).
 *                        sgs_render_fwd and sgs_render_bwd_with_splitting
 *                        launch their per-tile blocks in this order when it
 *                        is given (the heavy tiles start first and the short
 *                        ones fill the tail); results do not depend on it.
 *   walk     [W*capacity]  optional (NULL with walk_count): the forward
 *                        pass's walk lists, W = tile pixels / 32 warps per
 *                        tile.  sgs_render_fwd / sgs_render_fwd_l1 write, for
 *                        warp w of tile t (8x4 pixel blocks in row-major
 *                        order within the tile), the positions in t's list
 *                        of the entries it composited in at least one pixel,
 *                        front to back, from element W*start_t +
 *                        w*(end_t - start_t); walk_count [T*W] holds their
 *                        numbers.  Given them,
 *                        sgs_render_bwd_with_splitting walks only those
 *                        entries (recomputing the transmittance back to
 *                        front as always) instead of every entry whose alpha
 *                        support meets the block; its results are the same.
 *                        They must come from the forward pass over the same
 *                        proj, bins and settings.  Not written by
 *                        sgs_bin_sort, ignored by the multi-view calls. */
typedef struct sgs_bins {
    uint32_t *gids;
    uint64_t *keys;
    uint32_t *ranges;
    int32_t *count;
    int64_t capacity;
    uint32_t *order;
    uint32_t *walk;
    uint32_t *walk_count;
} sgs_bins;

/* Parameter gradients written by sgs_render_bwd_with_splitting. */
typedef struct sgs_grads {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logit;
    float *sh;
} sgs_grads;

/* Human-readable name of a status code (static storage). */
const char *sgs_error_string(int status);
/* CUDA error code behind the last SGS_ERR_CUDA returned on this thread. */
int sgs_get_last_cuda_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int sgs_version(void);
/* Number of CUDA kernel launches this library has issued since it was loaded
 * (all threads), for measurement reports.  Memsets are not counted. */
uint64_t sgs_kernel_launches(void);
/* Clears `bytes` bytes of caller device memory at dst on the stream (a
 * memset, no kernel launch; capture-safe): for the accumulators the entry
 * points add into, such as the loss of sgs_render_fwd_l1 / sgs_l1_loss_grad
 * and S_accum when no backward call resets it.  Errors:
 * SGS_ERR_INVALID_ARG on a NULL dst with bytes > 0; SGS_ERR_CUDA. */
int sgs_clear(void *dst, size_t bytes, void *stream);

/* Projection (Section 3, Eq. sigma_2D and the affine-Pi footnote; Pi is the
 * pinhole map, linearised at p as P = J W for the 2-D covariance).
 * Writes `out` rows [0, g->n).  The integer stage (depth, tile rect) uses a
 * fixed sequence of IEEE float32 operations so that it is reproducible
 * bit-for-bit.  Errors: SGS_ERR_INVALID_ARG on NULL arrays, n < 0,
 * sh_degree outside [0,3], non-positive image size or unsupported tile. */
int sgs_project(const sgs_gaussians *g, const sgs_camera *cam, const sgs_settings *st,
                const sgs_proj *out, void *stream);

/* Workspace bytes needed by sgs_bin_sort for n Gaussians, `capacity`
 * instances and `num_tiles` tiles.  Returns SGS_OK or SGS_ERR_INVALID_ARG. */
int sgs_bin_sort_workspace_size(int32_t n, int64_t capacity, int32_t num_tiles, size_t *bytes);

/* Binning and depth sort (Section 3): a stable radix sort of the Gaussians by
 * float32 depth bits, emission of one instance per covered tile in that order,
 * then a stable radix sort of the instances by tile id; equivalent to one
 * stable sort on the key (tile << 32 | depth bits) of instances emitted in
 * Gaussian order.  Reads proj->depth, proj->rect, proj->tiles_touched.
 * Errors: SGS_ERR_INVALID_ARG, SGS_ERR_WORKSPACE when ws_bytes is too small. */
int sgs_bin_sort(const sgs_proj *proj, int32_t n, const sgs_camera *cam, const sgs_settings *st,
                 const sgs_bins *out, void *ws, size_t ws_bytes, void *stream);

/* Forward compositing (Section 3, Eq. alpha_blend), front to back over each
 * tile's list: C = sum c_i alpha_i T_i + T_final bg.
 * Outputs image [H,W,3], final_T [H,W] (transmittance after the last
 * composited Gaussian) and n_contrib [H,W] (1 + list position of the last
 * composited Gaussian, 0 if none), the two maps the backward pass needs.
 * proj and bins are the same view's sgs_project / sgs_bin_sort outputs.
 * Errors: SGS_ERR_INVALID_ARG on a NULL struct or array, an invalid camera or
 * settings, or a tile grid that does not fit; SGS_ERR_CUDA if the launch
 * fails. */
int sgs_render_fwd(const sgs_proj *proj, const sgs_bins *bins, const sgs_camera *cam,
                   const sgs_settings *st, float *image, float *final_T, uint32_t *n_contrib,
                   void *stream);

/* sgs_render_fwd and sgs_l1_loss_grad in one kernel (the loss in the
 * compositing epilogue): the same image, final_T and n_contrib, dL_dimage
 * [H,W,3] = sign(image - target) / (3 H W n_views) bit for bit, and loss +=
 * mean |image - target| / n_views (summed per tile, one atomic each, so the
 * float sum may round differently from sgs_l1_loss_grad's).  target [H,W,3]
 * is read; loss is one device float.  Errors: as sgs_render_fwd, and
 * SGS_ERR_INVALID_ARG on a NULL target, dL_dimage or loss or n_views < 1. */
int sgs_render_fwd_l1(const sgs_proj *proj, const sgs_bins *bins, const sgs_camera *cam,
                      const sgs_settings *st, const float *target, int32_t n_views, float *image,
                      float *final_T, uint32_t *n_contrib, float *dL_dimage, float *loss, void *stream);

/* Photometric loss with the SSIM term of Gaussian-splatting training
 * (Section 3, Eq. loss; the paper's analysis keeps only L1, its footnote sets
 * SSIM aside):  loss += ((1 - lambda) L1 + lambda (1 - SSIM)) / n_views, with
 * L1 as in sgs_l1_loss_grad and SSIM after Wang et al. (2004): per channel,
 * 11x11 Gaussian window of sigma 1.5 with zero padding, C1 = 0.01^2,
 * C2 = 0.03^2, averaged over pixels and channels.  dL_dimage [H,W,3] is
 * overwritten with the gradient of that loss; lambda_dssim in [0, 1]
 * (0.2 in Gaussian-splatting training).  ws: sgs_ssim_l1_workspace_size bytes
 * (nine float maps of H x W).  Errors: SGS_ERR_INVALID_ARG on NULL arrays,
 * non-positive sizes, n_views < 1 or lambda_dssim outside [0, 1];
 * SGS_ERR_WORKSPACE when ws_bytes is too small; SGS_ERR_CUDA if a launch
 * fails. */
int sgs_ssim_l1_workspace_size(int32_t height, int32_t width, size_t *bytes);
int sgs_ssim_l1_loss_grad(const float *image, const float *target, int32_t height, int32_t width,
                          int32_t n_views, float lambda_dssim, float *dL_dimage, float *loss, void *ws,
                          size_t ws_bytes, void *stream);

/* L1 photometric loss (Section 3, Eq. loss, l = |.|):
 * loss += mean over pixels and channels of |image - target| / n_views and
 * dL_dimage = sign(image - target) / (3 H W n_views).  loss is one device
 * float, accumulated (+=); dL_dimage [H,W,3] is overwritten.  Errors:
 * SGS_ERR_INVALID_ARG on NULL arrays, non-positive sizes or n_views < 1;
 * SGS_ERR_CUDA if the launch fails. */
int sgs_l1_loss_grad(const float *image, const float *target, int32_t height, int32_t width,
                     int32_t n_views, float *dL_dimage, float *loss, void *stream);

/* Workspace bytes for sgs_render_bwd_with_splitting with n Gaussians. */
int sgs_render_bwd_workspace_size(int32_t n, size_t *bytes);

/* Backward pass fused with the splitting-matrix accumulation (Section 4.4,
 * Algorithm 1).  Back to front over each pixel's list, recomputing the
 * transmittance by division; dL/dalpha is reduced per Gaussian with warp
 * shuffles and one atomic per warp.  With w = dL/dalpha * alpha and
 * u = Q (x - mu) per composited, unclamped pair, the splitting matrix of this
 * view is S += P^T (sum w u u^T - (sum w) Q) P (the Appendix's Hessian
 * sigma (Y Y^T - P^T Q P), Y = P^T u, summed over pixels).
 * flags (a bit set; 0 = overwrite the gradients, add to S):
 *   SGS_BWD_ACCUMULATE_GRADS  grads are accumulated (+=); without it they are
 *                             overwritten (every row, zeros for Gaussians
 *                             this view does not reach; no prior zeroing
 *                             needed);
 *   SGS_BWD_RESET_S           this call starts a new accumulation period of
 *                             the splitting matrices (Algorithm 1 resets S
 *                             after each densification): S_accum (and
 *                             S_po_accum, S_ls_accum when given) are
 *                             overwritten with this call's matrices, zeros
 *                             where nothing composited; no prior zeroing
 *                             needed.
 *   Other bits: SGS_ERR_INVALID_ARG.
 * Without SGS_BWD_RESET_S, S_accum [N,6] = (xx, xy, xz, yy, yz, zz) is
 * accumulated (+=), so calling once per view (or per training step) sums over
 * them.
 * S_po_accum [N,3] (may be NULL): when given, the position-opacity block of
 * the splitting matrix over theta = (p, o) is accumulated (+=) too:
 * sum dL/dsigma G P^T u = P^T Q (sum w (x - mu)) / o (the opacity-opacity
 * entry is 0, sigma being linear in o); with S_accum it forms the 4x4
 * splitting matrix [[S, S_po], [S_po^T, 0]] that sgs_densify_split takes.
 * S_ls_accum [N,18] (may be NULL; requires S_po_accum): when given, the
 * blocks of the splitting matrix over theta = (p, l, o), l the log-scales, are
 * accumulated (+=) as well, with the projection Jacobian P held fixed (as for
 * S): columns 0-8 the p-l block (row p, column l), 9-14 the l-l upper
 * triangle (xx xy xz yy yz zz), 15-17 the l-o column.  With a_k = P R e_k,
 * b_k = Q a_k, t_k = b_k . (x - mu) and s_k = exp(l_k):
 *   p-l[j][k] = sum w (s_k^2 t_k^2 (Q P e_j).(x - mu) - 2 s_k^2 (P^T b_k)_j t_k)
 *   l-l[k][l] = sum w (s_k^2 s_l^2 t_k^2 t_l^2 + 2 delta_kl s_k^2 t_k^2
 *                      - 4 s_k^2 s_l^2 (a_k . b_l) t_k t_l)
 *   l-o[k]    = sum w s_k^2 t_k^2 / o
 * (the pixel moments of w (x - mu) up to fourth order are reduced per
 * Gaussian in the workspace).  The multi-view entry point below has no
 * such argument.
 * Errors: SGS_ERR_INVALID_ARG, SGS_ERR_WORKSPACE. */
int sgs_render_bwd_with_splitting(const sgs_gaussians *g, const sgs_proj *proj, const sgs_bins *bins,
                                  const sgs_camera *cam, const sgs_settings *st,
                                  const float *final_T, const uint32_t *n_contrib,
                                  const float *dL_dimage, const sgs_grads *grads, int32_t flags,
                                  float *S_accum, float *S_po_accum, float *S_ls_accum, void *ws,
                                  size_t ws_bytes, void *stream);
#define SGS_BWD_ACCUMULATE_GRADS 1
#define SGS_BWD_RESET_S 2

/* Several views of one scene in one pass (the batched densification step):
 * projection of every (view, Gaussian) pair, one binning and depth sort over
 * all views (global tile ids, view v's tiles following view v-1's), forward
 * compositing and its backward pass as persistent kernels that pull tiles of
 * all views from a work counter, the L1 loss of every view, and the
 * projection adjoint summing each Gaussian's views: gradients overwritten
 * or added and splitting matrices added to S_accum (and the position-opacity
 * blocks to S_po_accum when it is not NULL) or written, by `flags` as in
 * sgs_render_bwd_with_splitting.
 *   cams[n_views]      host array, 1 <= n_views <= 16, resolutions may differ;
 *   batch              Gaussians staged per shared-memory batch: 64, 128 or
 *                      256 (0 = min(tile pixels, 256));
 *   targets, images    concatenated [sum_v H_v W_v, 3] float, view v starting
 *                      at pixel sum_{u<v} H_u W_u; images is written;
 *   loss               device float, += mean over views of each view's mean
 *                      |C - Chat| (L1 over pixels and channels);
 *   d_count            device int32 receiving the instance count M of all
 *                      views; capacity = instance rows of the workspace.  When
 *                      M > capacity the results are not valid (no access goes
 *                      out of bounds); read d_count and retry with more.
 * Errors: SGS_ERR_INVALID_ARG, SGS_ERR_WORKSPACE, SGS_ERR_CUDA. */
int sgs_render_views_workspace_size(int32_t n, const sgs_camera *cams, int32_t n_views, const sgs_settings *st,
                                    int64_t capacity, size_t *bytes);
int sgs_render_views_with_splitting(const sgs_gaussians *g, const sgs_camera *cams, int32_t n_views,
                                    const sgs_settings *st, int32_t batch, const float *targets, float *images,
                                    float *loss, const sgs_grads *grads, int32_t flags, float *S_accum,
                                    float *S_po_accum, int32_t *d_count, int64_t capacity, void *ws,
                                    size_t ws_bytes, void *stream);

/* The binning that the last sgs_render_views_with_splitting call with the
 * same n, cameras, settings and capacity left in `ws`, for inspection (no
 * work is launched): out->gids [capacity] projection rows v*n + i in (global
 * tile id, float32 depth bits, row) order, out->ranges [T_total, 2] per global
 * tile (view v's tiles follow view v-1's), out->order the tile schedule,
 * out->capacity; out->keys, out->count, out->walk and out->walk_count are
 * NULL.  The pointers point into ws and stay valid while ws holds that call's
 * results.  Errors: SGS_ERR_INVALID_ARG as sgs_render_views_workspace_size,
 * or a NULL out; SGS_ERR_WORKSPACE when ws_bytes is too small. */
int sgs_render_views_bins(int32_t n, const sgs_camera *cams, int32_t n_views, const sgs_settings *st,
                          int64_t capacity, void *ws, size_t ws_bytes, sgs_bins *out);

/* Forward-only render of a batch of views whose scenes may differ (the
 * render-serving batch): scenes[v] is the scene of view v (sh_degree must be
 * equal across the batch), images as in sgs_render_views_with_splitting.
 * Each view's image is bit-identical to rendering it alone with the same
 * settings.  d_count / capacity: instance count of the whole batch, as above.
 * Errors: SGS_ERR_INVALID_ARG (also when the scenes' SH degrees differ),
 * SGS_ERR_WORKSPACE, SGS_ERR_CUDA. */
int sgs_render_batch_workspace_size(const sgs_gaussians *scenes, const sgs_camera *cams, int32_t n_views,
                                    const sgs_settings *st, int64_t capacity, size_t *bytes);
int sgs_render_batch_fwd(const sgs_gaussians *scenes, const sgs_camera *cams, int32_t n_views,
                         const sgs_settings *st, int32_t batch, float *images, int32_t *d_count, int64_t capacity,
                         void *ws, size_t ws_bytes, void *stream);

/* Adam step on one parameter array of `count` floats (the optimiser of the
 * training loop around the path; Algorithm 1's "standard gradient descent"
 * step): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * When grad_accum is not NULL it also adds g into it (Algorithm 1's
 * G <- G + grad).  step >= 1.  Errors: SGS_ERR_INVALID_ARG on count < 0,
 * step < 1, lr < 0, beta outside [0, 1), eps <= 0 or a NULL array when
 * count > 0; SGS_ERR_CUDA if the launch fails. */
int sgs_adam_step(float *param, const float *grad, float *m, float *v, int64_t count, float lr, float beta1,
                  float beta2, float eps, int32_t step, float *grad_accum, void *stream);
/* The same update with the step count read from device memory (d_step, one
 * int32 >= 1 when the kernel runs), so that a captured graph can replay it
 * while the caller advances the count on the device.  Errors: as
 * sgs_adam_step, with a NULL d_step in place of step < 1. */
int sgs_adam_step_dev(float *param, const float *grad, float *m, float *v, int64_t count, float lr, float beta1,
                      float beta2, float eps, const int32_t *d_step, float *grad_accum, void *stream);

/* Workspace bytes for sgs_densify_split with n Gaussians. */
int sgs_densify_split_workspace_size(int32_t n, size_t *bytes);

/* Steepest density control (Theorem 2, Algorithm 1, Appendix
 * "Eigendecomposition").  For each Gaussian: S_bar = S_accum * inv_T_split;
 * lambda_min, v_min by the trigonometric root formula (float32) refined by
 * one Rayleigh quotient; flag = lambda_min < eps_split, and, when grad_norm is
 * not NULL, grad_norm[i] <= eps_grad (the "compactest" condition).  When
 * max_splits > 0 and more Gaussians are flagged, only the max_splits with the
 * least lambda_min stay flagged, ties by index (the "increment budget"
 * variant); max_splits <= 0 means no budget.
 * Output rows: row i = Gaussian i, moved to p + eps_i v_min with opacity o/2
 * when flagged; row N + excl[i] = its second offspring p - eps_i v_min with
 * opacity o/2 (excl = exclusive prefix sum of the flags); scales, rotation and
 * SH are copied; eps_i = step_scale * max_k exp(log_scale_ik).
 * d_n_out (device int32) receives N + number of flags; rows at or beyond
 * `capacity` are not written.  parent_index [capacity] (int32, may be NULL),
 * lam_min_out [N] and v_min_out [N,3] (may be NULL) are written.
 * With S_po_accum [N,3] not NULL the split runs over theta = (p, o) (dim
 * Theta = 4): lambda_min, v_min (4 components, v_min_out [N,4]) of
 * [[S, S_po], [S_po^T, 0]] * inv_T_split by cyclic Jacobi rotations (float32)
 * refined by one Rayleigh quotient, same sign convention; the offspring take
 * p +- eps_i v_p and opacities (o +- eps_i v_o) / 2, each clamped to
 * [1e-4, 1 - 1e-4].
 * With S_ls_accum [N,18] also given (layout as in
 * sgs_render_bwd_with_splitting; requires S_po_accum) the split runs over
 * theta = (p, l, o) (dim Theta = 7): the 7x7 matrix with blocks p-p, p-l,
 * l-l, p-o, l-o and o-o = 0, times inv_T_split, by the same Jacobi rotations;
 * v_min_out [N,7] = (v_p, v_l, v_o); the offspring also take log-scales
 * l +- eps_i v_l.
 * `out` must not alias `in`.  Errors: SGS_ERR_INVALID_ARG, SGS_ERR_WORKSPACE. */
int sgs_densify_split(const sgs_gaussians *in, const float *S_accum, const float *S_po_accum,
                      const float *S_ls_accum, float inv_T_split,
                      float eps_split, float step_scale, const float *grad_norm, float eps_grad,
                      int64_t max_splits, const sgs_gaussians_mut *out, int64_t capacity, int32_t *d_n_out,
                      int32_t *parent_index, float *lam_min_out, float *v_min_out,
                      void *ws, size_t ws_bytes, void *stream);

/* Allocation-free variant of sgs_densify_split (the paper has no counterpart:
 * this is an interface convenience).  For callers that cannot give the
 * library a workspace -- code running where cudaMalloc is not allowed or not
 * wanted (a host callback, a real-time loop in which an allocation would
 * synchronise the device, a plugin whose host owns every device allocation and
 * passes only input and output buffers).  Same arguments, semantics and
 * results as sgs_densify_split, minus the workspace: the scratch is a fixed
 * SGS_NOALLOC_SCRATCH_BYTES array inside the library's device image, reserved
 * on every GPU that loads the library until the process exits.
 *   - n must not exceed SGS_NOALLOC_MAX_GAUSSIANS; larger n returns
 *     SGS_ERR_INVALID_ARG before anything is launched.
 *   - It works on the calling thread's current device.  The first call on a
 *     device looks up the array's device address (cudaGetSymbolAddress) and
 *     caches it; make that first call before any stream capture begins.
 *   - Every call shares the one array, so calls whose work overlaps on the GPU
 *     (other streams, other threads) race: serialise them.  The array keeps the
 *     last call's contents; the call clears what it needs cleared itself.
 *   - The cached address belongs to the device's current context: do not use
 *     this entry point on a device after cudaDeviceReset in the same process.
 *   - Scratch: 44 bytes per Gaussian plus the scan's partials (about 44 MB at
 *     the maximum n); a build whose workspace layout outgrew the array returns
 *     SGS_ERR_WORKSPACE for every call.
 *   - It calls no cudaMalloc, cudaFree or allocating routine. */
#define SGS_NOALLOC_MAX_GAUSSIANS 1000000
#define SGS_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
int sgs_densify_split_noalloc(const sgs_gaussians *in, const float *S_accum, const float *S_po_accum,
                              const float *S_ls_accum, float inv_T_split,
                              float eps_split, float step_scale, const float *grad_norm, float eps_grad,
                              int64_t max_splits, const sgs_gaussians_mut *out, int64_t capacity, int32_t *d_n_out,
                              int32_t *parent_index, float *lam_min_out, float *v_min_out, void *stream);

/* ------------------------------------------------------------------------
 * Measurement instrumentation.  Not steps of the method and not used by its
 * path: the benchmark calls them to count the rasteriser's work units and to
 * measure the FP32 roofline it quotes.
 * ------------------------------------------------------------------------ */

/* Pair counts of the forward walk: counts [H,W,2] uint32 = (pairs evaluated,
 * pairs composited) per pixel, the work units behind the rasteriser's
 * algorithmic FLOP count; warp_union [T * tile pixels / 32] (may be NULL): per
 * 8x4 pixel block of each tile, the number of list entries at least one of
 * its pixels composites (what the forward's walk lists hold).  A walk over
 * every list entry without culling.  Errors: as sgs_render_fwd. */
int sgs_render_stats(const sgs_proj *proj, const sgs_bins *bins, const sgs_camera *cam,
                     const sgs_settings *st, uint32_t *counts, uint32_t *warp_union, void *stream);

/* FP32 FMA throughput probe: `blocks` blocks of 256 threads, each thread runs
 * `iters` rounds of 8 independent fused multiply-adds (16 FLOP per round) and
 * writes one float to out[blocks * 256].  Timing it gives the attainable FP32
 * peak that the rasteriser's ALU roofline is quoted against.  Errors:
 * SGS_ERR_INVALID_ARG on a NULL out or non-positive blocks or iters. */
int sgs_fma_probe(float *out, int32_t blocks, int32_t iters, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* STEEPGS_H */
