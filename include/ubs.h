/*
 * ubs.h -- C-ABI of the Universal Beta Splatting differentiable rasterizer
 * (arXiv 2510.03312) for NVIDIA GB300 (sm_103a).
 *
 * The library renders N-dimensional anisotropic Beta kernels (N = 3, 4, 6, 7:
 * 3 spatial dimensions plus C = N - 3 query dimensions, time and/or view
 * direction) and differentiates the rendering.  Each entry point is one step
 * of the path:
 *
 *   ubs_preprocess  kernel construction (Sec. 4.2), Beta-modulated
 *                   conditioning on each view's query (Sec. 4.3, 4.4) and EWA
 *                   projection with the compact Beta support (Sec. 3)
 *   ubs_bin_sort    tile binning and the front-to-back depth order
 *                   ("standard splatting", Sec. 4.5; ordering of Sec. 3)
 *   ubs_render_fwd  per-tile front-to-back alpha compositing (Sec. 3)
 *   ubs_render_bwd  gradients of the rendered images with respect to every
 *                   primitive parameter (differentiable rendering, Sec. 4.5)
 *
 * and the training step around it: ubs_image_loss (the image loss of
 * Sec. 4.5 and its gradient), ubs_adam_step (the optimiser of Sec. 5.1
 * with the penalties and noise of Sec. 4.5) and ubs_mcmc_relocate (the
 * primitive management of Sec. 4.5).
 *
 * Conventions shared by every call
 * --------------------------------
 * Memory: every pointer in ubs_scene, ubs_scene_grad, the image and dL/dimage
 *   arguments and the workspace is a DEVICE pointer owned by the caller.  The
 *   ubs_problem, ubs_scene/ubs_scene_grad and ubs_view arrays themselves are
 *   HOST memory, read during the call only.  The library allocates nothing
 *   and frees nothing.
 * Streams: every call is asynchronous on `stream`; nothing synchronises
 *   except ubs_read_status.  The sequence preprocess -> bin_sort ->
 *   render_fwd -> render_bwd on one workspace must be issued in that order on
 *   one stream (or with equivalent dependencies); it can be captured in a
 *   CUDA graph.
 * Workspace: all state between calls lives in the caller's workspace of at
 *   least ubs_workspace_size(problem) bytes, 256-byte aligned.  Calls of the
 *   same problem on different workspaces may run concurrently.
 * Errors: argument errors (null pointers, unsupported N, misalignment, a
 *   workspace that is too small) are returned synchronously and nothing is
 *   launched.  Errors found on the device (instance capacity exceeded, a
 *   bounded wait that gave up) are recorded in the workspace and reported by
 *   ubs_read_status; kernels never trap.
 * Floating point: parameters and images are IEEE binary32.
 */
#ifndef UBS_H
#define UBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t; /* the CUDA runtime's stream handle */

typedef enum {
  UBS_OK = 0,
  UBS_ERR_INVALID_ARG = 1, /* null pointer, bad size, unsupported N or mode */
  UBS_ERR_ALIGNMENT = 2,   /* a pointer or the workspace is misaligned */
  UBS_ERR_CAPACITY = 3,    /* more tile instances than instance_capacity */
  UBS_ERR_CUDA = 4,        /* a CUDA launch or copy failed */
  UBS_ERR_TIMEOUT = 5,     /* reserved: no kernel of this library waits on another block,
                              so no call returns it; the value is kept so that codes stay stable */
  UBS_ERR_INTERNAL = 6,
  UBS_ERR_WORKSPACE = 7    /* workspace smaller than ubs_workspace_size */
} ubs_status;

/* Spatial rotation R_x of the spatial-orthogonal Cholesky factor (Sec. 4.2 and
 * the appendix's table of rotation parameterisations): the normalised 3DGS
 * quaternion, or from omega with the skew matrix A(omega) = [[0,-w3,w2],
 * [w3,0,-w1],[-w2,w1,0]]: R = I + A (first-order Taylor of exp A, the paper's
 * choice), R = I + A + A^2/2 (second-order Taylor) or the Cayley transform
 * R = (I - A)^-1 (I + A) = I + 2 (A + A^2) / (1 + |omega|^2).  UBS_ROT_CHOL is
 * the table's plain Cholesky row: no rotation, the spatial block of L is a
 * general lower-triangular factor with diagonal scale_x and strictly-lower
 * entries (l10, l20, l21) = rot.  UBS_ROT_EXP is the table's matrix
 * exponential R = exp(A(omega)) (Rodrigues' form; the decision stage takes
 * sin and cos from the library's own binary32 functions). */
enum { UBS_ROT_QUAT = 0, UBS_ROT_SKEW1 = 1, UBS_ROT_SKEW2 = 2, UBS_ROT_CAYLEY = 3, UBS_ROT_CHOL = 4, UBS_ROT_EXP = 5 };

enum {
  UBS_FLAG_TIGHT_CUT = 1, /* cut each footprint at r_cut = 1-(a_min/o(q))^(1/beta_x) */
  UBS_FLAG_COUNT_PAIRS = 2, /* diagnostic: ubs_render_fwd runs a variant that also counts,
                               per pixel, the pairs with r < 1 and the evaluated entries
                               (ubs_export 9 and 10) */
  UBS_FLAG_ACCUMULATE_GRADS = 4, /* ubs_render_bwd / ubs_render_bwd_params ADD the parameter
                                   gradients to the ubs_scene_grad buffers instead of
                                   overwriting them: a scene rendered by several problems
                                   (launches) gets the sum over all of its views */
  UBS_FLAG_PERSISTENT = 8, /* the blend kernels run as persistent grids (one CTA per resident
                              slot) that take tiles or 8x8 blocks from a counter in the same order,
                              instead of one CTA per tile or block; the results are the same */
  UBS_FLAG_SPLIT_LISTS = 16, /* tile lists longer than 2048 entries are split into segments of 2048
                               blended by separate CTAs and merged front to back with the over
                               operator (C = C_1 + T_1 C_2, T = T_1 T_2), walking a segment again
                               for the pixels whose transmittance falls below T_min inside it; the
                               backward walks the segments in parallel from each segment's end.
                               Images and gradients agree with the unsplit form up to float
                               rounding.  Takes precedence over UBS_FLAG_PERSISTENT; ignored by
                               the UBS_FLAG_COUNT_PAIRS variant.  Needs a larger workspace (see
                               ubs_workspace_size) */
  UBS_FLAG_NO_THRESHOLDS = 32, /* the gradient-check mode (central differences across a skip or
                                  stop decision are meaningless): alpha_min = 0, alpha_max = 1
                                  and T_min = 0 override the configuration's values, so every
                                  pair with r < 1 is composited and no pixel stops early */
  UBS_FLAG_CHECKED = 64 /* the blend kernels also record a record id of a tile list outside the
                           problem's records (impossible in a consistent workspace) as the device
                           status UBS_ERR_INTERNAL, which ubs_read_status reports; without it such
                           an id is only clamped.  Results are otherwise the same */
};

/* One primitive set (Sec. 4.1-4.3).  Structure of arrays: every block below
 * is `rows` consecutive planes of P floats (plane r of a block starts at
 * block + r * P).  All blocks are device pointers, 4-byte aligned.
 *   mean_x  [3][P]        spatial mean mu_x
 *   mean_q  [C][P]        query mean mu_q; rows ordered q = [t, d] (N=7),
 *                         [d] (N=6), [t] (N=4); unused for N=3 (may be NULL)
 *   rot     [4][P] quaternion (w,x,y,z), normalised inside (UBS_ROT_QUAT), or
 *           [3][P] omega of A(omega) (UBS_ROT_SKEW1, UBS_ROT_SKEW2,
 *           UBS_ROT_CAYLEY, UBS_ROT_EXP; Sec. 4.2), or [3][P] (l10, l20, l21) of the
 *           spatial Cholesky factor (UBS_ROT_CHOL)
 *   scale_x [3][P]        spatial scales s_x > 0
 *   L_qx    [3C][P]       C x 3 cross block, row-major: (k, j) at row 3k + j
 *   L_q     [C(C+1)/2][P] lower-triangular query block, packed row-major:
 *                         (i, j <= i) at row i(i+1)/2 + j; diagonal s_q > 0
 *   b       [1+C][P]      Beta parameters b_x, b_q1..b_qC (beta_x = 4 e^b_x,
 *                         beta_q = e^b_q)
 *   opacity [P]           o in [0, 1]
 *   rgb     [3][P]        colour                                          */
typedef struct {
  int32_t N;        /* 3, 4, 6 or 7 */
  int32_t rot_mode; /* UBS_ROT_* */
  int64_t P;        /* number of primitives, >= 0 */
  const float* mean_x;
  const float* mean_q;
  const float* rot;
  const float* scale_x;
  const float* L_qx;
  const float* L_q;
  const float* b;
  const float* opacity;
  const float* rgb;
} ubs_scene;

/* Gradient buffers with the layout of ubs_scene (device pointers, 4-byte
 * aligned).  ubs_render_bwd OVERWRITES them, unless the problem's config has
 * UBS_FLAG_ACCUMULATE_GRADS, in which case it adds to them. */
typedef struct {
  float* mean_x;
  float* mean_q;
  float* rot;
  float* scale_x;
  float* L_qx;
  float* L_q;
  float* b;
  float* opacity;
  float* rgb;
} ubs_scene_grad;

/* A pinhole view (Sec. 3: viewing transform W and projection).  x_cam =
 * R x_world + t with camera axes x right, y down, z forward; pixel (i, j)
 * has its centre at (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy.
 * `time` is the temporal query of N = 4 and N = 7 scenes (Sec. 4.4);
 * `scene_id` selects the primitive set the view renders. */
typedef struct {
  float R[9]; /* row-major */
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float time;
  int32_t scene_id;
} ubs_view;

/* Rasterizer constants ("standard splatting", Sec. 4.5; 3DGS practice). */
typedef struct {
  int32_t tile_w, tile_h; /* 8x8, 16x16, 16x32 (w x h = 16 x 32) or 32x32 */
  float alpha_min;        /* skip a pair when alpha < alpha_min (1/255) */
  float alpha_max;        /* alpha = min(alpha_max, o(q) (1 - r)^beta_x) (0.99) */
  float T_min;            /* stop before T (1 - alpha) < T_min (1e-4) */
  float eps2d;            /* screen-space dilation added to Sigma' (0.3 px^2) */
  float near_plane;       /* cull when camera-space z <= near_plane (0.2) */
  float jac_clip;         /* Jacobian ray clamp, multiple of tan(fov/2) (1.3) */
  float bg[3];            /* background colour */
  int32_t flags;          /* UBS_FLAG_* */
} ubs_config;

/* The whole problem of one call sequence: n_scenes primitive sets and
 * n_views views (each view renders scenes[views[v].scene_id]).  Records are
 * numbered record_offset(v) + p, views in order; tiles are numbered
 * tile_offset(v) + ty * tiles_x(v) + tx.  Images of all views are packed:
 * view v occupies 3 * height * width floats starting at pixel_offset(v) * 3,
 * planar [3][height][width]. */
typedef struct {
  const ubs_scene* scenes; /* host array [n_scenes] */
  int32_t n_scenes;        /* 1 .. 64 */
  const ubs_view* views;   /* host array [n_views] */
  int32_t n_views;         /* 1 .. 256 */
  ubs_config cfg;
  int64_t instance_capacity; /* maximum (tile, record) instances */
} ubs_problem;

/* Device-side status read back by ubs_read_status. */
typedef struct {
  int32_t status;              /* ubs_status of the device-side work */
  int32_t reserved;
  int64_t visible_records;     /* records with a non-empty tile rectangle */
  int64_t instances;           /* (tile, record) instances required */
} ubs_device_status;

/* Bytes of workspace the problem needs (0 on invalid arguments).  Pure host
 * arithmetic. */
size_t ubs_workspace_size(const ubs_problem* problem);

/* P1-P3 of Sec. 4.2-4.4 and Sec. 3: for every (view, primitive) record,
 * builds Sigma from the spatial-orthogonal Cholesky factor, conditions it on
 * the view's query (Beta-modulated mean, covariance and opacity), projects
 * it (mean, conic, depth) and computes its tile rectangle under the compact
 * Beta support.  Also resets the workspace's device status. */
ubs_status ubs_preprocess(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                          cudaStream_t stream);

/* B1-B3: lists every (tile, record) instance, orders each tile's list front
 * to back by (float32 depth, record index) and finds each tile's range.
 * Must follow ubs_preprocess on the same workspace (it reads the records
 * and visibility that call writes, and the counters it zeroes).  If the
 * instances exceed problem->instance_capacity the device status becomes
 * UBS_ERR_CAPACITY (with the required count) and every list is left
 * empty; later calls on this workspace then do nothing. */
ubs_status ubs_bin_sort(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                        cudaStream_t stream);

/* R1 (Sec. 3): per pixel, alpha = min(alpha_max, o(q) (1 - r)^beta_x) for
 * r < 1, blended front to back into colour and transmittance; writes the
 * packed images (device, float32, see ubs_problem) and keeps the per-pixel
 * final transmittance and last contributor in the workspace. */
ubs_status ubs_render_fwd(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                          float* image, cudaStream_t stream);

/* G1-G2: given dL/dimage (device, packed like the images), writes dL/dparams
 * of every scene into grads[0 .. n_scenes-1] (host array of device buffers,
 * overwritten).  Must follow ubs_render_fwd on the same workspace. */
ubs_status ubs_render_bwd(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                          const float* dL_dimage, const ubs_scene_grad* grads, cudaStream_t stream);

/* G1 alone: the backward blend.  Accumulates dL/d(mu', conic, log2 o(q),
 * beta_x, rgb) of every record into the workspace (zeroed first). */
ubs_status ubs_render_bwd_blend(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                                const float* dL_dimage, cudaStream_t stream);

/* G2 alone: chains the workspace's per-record screen gradients back to the
 * parameters of every scene (grads overwritten, or added to with
 * UBS_FLAG_ACCUMULATE_GRADS).  ubs_render_bwd is
 * ubs_render_bwd_blend followed by ubs_render_bwd_params. */
ubs_status ubs_render_bwd_params(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                                 const ubs_scene_grad* grads, cudaStream_t stream);

/* Synchronises `stream` and copies the device status into *out (host). */
ubs_status ubs_read_status(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                           ubs_device_status* out, cudaStream_t stream);

/* Copies internal per-record and per-instance arrays out of the workspace
 * (for tests and diagnostics).  `what` selects: 0 = depth keys [R] u32,
 * 1 = tiles_touched [R] u32, 2 = rectangles [R] x 2 u32 (x0|y0<<16,
 * x1|y1<<16), 3 = render records [R] x 12 f32, 4 = sorted instance records
 * [instances] u32, 5 = tile starts [tiles + 1] u32, 6 = final T [pixels]
 * f32, 7 = last contributor [pixels] u32, 8 = per-record screen gradients
 * [R] x 12 f32 (3 and 8 are defined for the visible records, those with
 * tiles_touched > 0); written only by the UBS_FLAG_COUNT_PAIRS variant of
 * ubs_render_fwd: 9 = per pixel, the pairs with r < 1 on its tile's list
 * visited before the pixel terminated [pixels] u32 (without
 * UBS_FLAG_TIGHT_CUT every record with r < 1 at the pixel is on that list,
 * so this is the tile-free count), 10 = per pixel, the list entries its
 * warp evaluated (those passing the blend's support cull, walked before the
 * warp's 64 pixels were all done) [pixels] u32.  `dst` is device memory of
 * at least `dst_bytes`; returns the bytes needed in *bytes_needed. */
ubs_status ubs_export(const ubs_problem* problem, void* workspace, size_t workspace_bytes,
                      int32_t what, void* dst, size_t dst_bytes, size_t* bytes_needed,
                      cudaStream_t stream);

const char* ubs_status_string(ubs_status status);

/* ---------------------------------------------------------------------------
 * The training step around the rasterizer (Sec. 4.5 loss, Sec. 5.1 optimiser)
 * ------------------------------------------------------------------------- */

/* Image loss of Sec. 4.5, (1 - lambda_ssim) L1 + lambda_ssim (1 - SSIM), and
 * its gradient.  Readings: L1 is the mean |C - C*| over a view's pixels and
 * channels; SSIM is the mean structural-similarity map of Wang et al. (2004)
 * per channel, with an 11 x 11 Gaussian window of standard deviation 1.5,
 * C1 = 0.01^2, C2 = 0.03^2 and zero padding at the border (a map of the
 * image's size); over several views the loss is the mean of the views'.
 * Images and targets are packed like the rasterizer's (view v planar
 * [3][heights[v]][widths[v]], views back to back).  widths/heights are host
 * arrays [n_views], 1 <= n_views <= 256.
 *
 * ubs_loss_workspace_size: bytes of workspace (0 on invalid arguments).
 * ubs_image_loss: writes dL/dimage (device, packed like the images; it may
 *   not alias image or target) and loss (device float[1 + n_views]: the
 *   total, then each view's loss).  workspace: device, 256-byte aligned, at
 *   least ubs_loss_workspace_size bytes, holding the per-pixel partial
 *   derivatives of SSIM and per-block sums between the kernels.  The sums are
 *   reduced in a fixed order: results are deterministic.  Asynchronous on
 *   `stream`; allocates nothing. */
size_t ubs_loss_workspace_size(int32_t n_views, const int32_t* widths, const int32_t* heights);
ubs_status ubs_image_loss(int32_t n_views, const int32_t* widths, const int32_t* heights, const float* image,
                          const float* target, float lambda_ssim, float* dL_dimage, float* loss,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream);

enum { UBS_ACT_IDENTITY = 0, UBS_ACT_SIGMOID = 1, UBS_ACT_EXP = 2 };

/* One parameter plane of the optimiser step. */
typedef struct {
  float lr;           /* Adam learning rate of the plane (Sec. 5.1: 1.6e-4 positions,
                         5e-2 opacity, 5e-3 scales, 1e-3 the rest) */
  int32_t activation; /* UBS_ACT_*: the renderer reads act(raw) */
  float l1_weight;    /* weight of an L1 penalty on the activated value
                         (Sec. 4.5: lambda_o on opacity, lambda_Sigma on scales) */
  int32_t noise_row;  /* row of `noise` added after the update, or -1 */
} ubs_adam_plane;

typedef struct {
  float beta1, beta2, eps; /* Adam constants (0.9, 0.999, 1e-15) */
  int32_t step;            /* t >= 1, for the bias corrections 1 - beta^t */
  float lambda_eps;        /* weight of the injected noise (Sec. 4.5: 1) */
} ubs_adam_config;

/* One Adam step (Kingma and Ba 2015) over K planes of P parameters, fused
 * with the activation and the penalties of Sec. 4.5:
 *   a = act(raw);  g = grad + l1_weight sign(a);  g_raw = g act'(raw)
 *   m = beta1 m + (1 - beta1) g_raw;  v = beta2 v + (1 - beta2) g_raw^2
 *   raw -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
 *   raw += lambda_eps noise[noise_row]     (the spatial noise of Sec. 4.5)
 *   act_out = act(raw)
 * raw, act_out, grad, m, v: device [K][P] planes (plane k at k * P), 4-byte
 * aligned; grad is dL/d(activated value), as ubs_render_bwd writes it.
 * act_out is the buffer the rasterizer reads (it may not alias raw).
 * planes: host array [K], 1 <= K <= 64.  noise: device [rows][P], or NULL
 * when no plane has noise_row >= 0.  Asynchronous on `stream`; allocates
 * nothing. */
ubs_status ubs_adam_step(int32_t K, int64_t P, const ubs_adam_plane* planes, const ubs_adam_config* cfg,
                         float* raw, float* act_out, const float* grad, float* m, float* v, const float* noise,
                         cudaStream_t stream);

/* MCMC relocation of dead primitives (Sec. 4.5 primitive management, the
 * kernel-agnostic scheme of Deformable Beta Splatting).  A primitive is dead
 * when its opacity act[opacity_row] <= dead_threshold (3DGS-MCMC: 0.005).
 * Each dead slot j is moved onto a live source drawn with probability
 * proportional to opacity, exactly: live weights are the integers
 * floor(o * 2^24), and the source is the first primitive whose inclusive
 * cumulative weight exceeds rand[j] mod (total weight).  A source drawn n
 * times and its n copies take the opacity 1 - (1 - o)^(1/(n+1)) (Sec. 4.5),
 * which keeps their composited density; every other row of act and raw is
 * copied from the source, and m and v of every touched primitive are
 * zeroed.  Nothing moves when no primitive is alive.
 * act, raw, m, v: device [K][P] planes (the layout of ubs_adam_step; raw of
 *   the opacity row is its logit), 4-byte aligned, updated in place.
 * rand: device uint64 [P], drawn by the caller, 8-byte aligned.
 * sources: device int32 [P] or NULL: the source of each slot (-1: kept).
 * n_relocated: device int64 or NULL: the number of slots moved.
 * workspace: device, 256-byte aligned, >= ubs_mcmc_workspace_size(P).
 * Asynchronous on `stream`; allocates nothing. */
size_t ubs_mcmc_workspace_size(int64_t P);
ubs_status ubs_mcmc_relocate(int32_t K, int64_t P, int32_t opacity_row, float dead_threshold, float* act,
                             float* raw, float* m, float* v, const uint64_t* rand, int32_t* sources,
                             int64_t* n_relocated, void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Forward rendering that allocates nothing.  (The paper has no counterpart:
 * this serves callers that cannot allocate device memory when they render,
 * such as plugin hosts without an allocator, processes confined to a
 * pre-sized memory pool, or loops that forbid allocation after start-up.)
 * Runs preprocess -> bin_sort -> render_fwd exactly like the entry points
 * above, but takes the workspace from a fixed 32 MiB array in the library's
 * own device memory instead of a caller-supplied buffer; the caller passes
 * only the problem (device scene buffers as usual) and the output image.
 * - Returns UBS_ERR_WORKSPACE, launching nothing, when
 *   ubs_workspace_size(problem) exceeds 32 MiB.
 * - Uses the array of the current device.  The first call on a device looks
 *   up the array's device address with that device current; make that first
 *   call before any stream capture.
 * - Every call on a device shares the one array, which keeps the previous
 *   call's contents (each step clears what must start at zero); calls whose
 *   work overlaps on the GPU race on it.
 * - As with ubs_bin_sort, if problem->instance_capacity is too small the
 *   image is left unwritten (its previous contents stay) and the device
 *   status becomes UBS_ERR_CAPACITY with the required instance count; read
 *   it with ubs_read_status_static.
 * - Calls no cudaMalloc, cudaFree or allocating library routine.  The array
 *   stays allocated on every GPU that loaded this part of the library until
 *   the process exits. */
ubs_status ubs_render_fwd_static(const ubs_problem* problem, float* image, cudaStream_t stream);

/* The device status of the last ubs_render_fwd_static on the current
 * device, as ubs_read_status gives it for a caller workspace: synchronises
 * `stream` and copies the status header of the fixed array into *out (host).
 * `problem` must be the problem of that call (its layout locates the
 * header); returns UBS_ERR_WORKSPACE when it exceeds the array.  Allocates
 * nothing. */
ubs_status ubs_read_status_static(const ubs_problem* problem, ubs_device_status* out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* UBS_H */
