/*
 * s3r.h -- C ABI of the GB300 (sm_103a) S3R-GS render-and-backprop hot path.
 *
 * One timestep of the streamlined pipeline of S3R-GS (Sec. 3.3, "Streamlined
 * Reconstruction Stage"):
 *   1. temporal selection of the Gaussians whose visibility window contains t
 *      (Sec. 3.3, "Temporal separation");
 *   2. projection of each selected Gaussian straight into every camera through
 *      one composed matrix per instance, W_{t,i} = W_t W_{t,i2g} (Sec. 3.3,
 *      "Instance-specific projection"), with the EWA 2D covariance of Eq. 1;
 *   3. the frustum mask M_t and the point-life update of Eq. 5;
 *   4. the adaptive-LOD cull of Gaussians whose 2D scale is below r
 *      (Sec. 3.3, "Adaptive LOD", deterministic threshold form);
 *   5. SH colour, tile|depth key duplication, radix sort, and 16x16-tile
 *      front-to-back alpha blending (Eq. 2);
 *   6. the exact gradient of the images w.r.t. all Gaussian parameters and the
 *      per-instance poses (the training step the paper's reconstruction runs);
 *   7. Eq. 6 and the periodic reset of the visibility record.
 *
 * Conventions (every entry point):
 *   - All array arguments are DEVICE pointers on the workspace's device,
 *     caller-owned, FP32/uint32/int64 as stated, C-contiguous, and 16-byte
 *     aligned where a 128-bit load is used (marked "16-B"). A misaligned or
 *     null required pointer returns S3R_ERR_INVALID and launches nothing.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream). They perform no host synchronisation
 *     and allocate nothing, so a sequence of them can be captured into a CUDA
 *     graph. Only s3r_workspace_create/destroy allocate and free, and only
 *     s3r_query_counts / s3r_sync_status and the resume call s3r_set_epoch
 *     synchronise.
 *   - Data-dependent sizes (selected Gaussians, splats, duplicates) stay on
 *     the device; every kernel reads its own extent from there.
 *   - Device-side failures (a capacity overflow, an exhausted spin budget) are
 *     latched into a status word in the workspace; the work that overflowed is
 *     dropped, never written out of bounds. The next s3r_sync_status (or
 *     s3r_query_counts) returns S3R_ERR_CAPACITY / S3R_ERR_TIMEOUT and clears it.
 *   - Nothing aborts. s3r_last_error() returns a thread-local message for the
 *     most recent non-OK status of the calling thread.
 *   - A sequence captured into a CUDA graph for replay starts at s3r_project:
 *     some set-up of a call is done by the launches of the calls before it
 *     (the forward clears the per-splat adjoints that the backward after it
 *     sums into; a backward that does not follow a forward clears them with a
 *     launch of its own), so a graph of a later call alone would replay
 *     without it.
 *
 * Camera model: OpenCV pinhole (x right, y down, z forward). Pixel (x, y) is
 * sampled at (x + 0.5, y + 0.5). Tiles are 16x16 pixels. Gaussian i of
 * segment k (k = 0 static, k >= 1 instance k) is expressed in that segment's
 * local frame; instance k's pose at time t maps local to world coordinates.
 */
#ifndef S3R_H_
#define S3R_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  S3R_OK = 0,
  S3R_ERR_INVALID = 1,   /* bad argument: null, misaligned, out of range */
  S3R_ERR_CAPACITY = 2,  /* a device count exceeded the workspace capacity */
  S3R_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  S3R_ERR_TIMEOUT = 4,   /* a bounded device-side wait gave up */
  S3R_ERR_STATE = 5      /* calls out of order (e.g. sort before project) */
} s3r_status;

#define S3R_MAX_VIEWS 32
#define S3R_TILE 16

/* Pinhole camera. world_to_cam is the 3x4 row-major matrix [R | t] of the
 * world-to-camera transform W_t (Eq. 1). near_z <= 0 means 0.2. */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy, near_z;
  float world_to_cam[12];
} s3r_camera;

/* The Gaussians (Sec. 3.3: position, covariance as scale + rotation, opacity;
 * colour as SH coefficients). Device pointers, all of length n along dim 0:
 *   means          [n,3]  FP32
 *   log_scales     [n,3]  FP32  (scale = exp(log_scale))
 *   quats          [n,4]  FP32  (w, x, y, z), any norm > 0; 16-B
 *   opacity_logits [n]    FP32  (opacity = sigmoid(logit))
 *   sh             [n,K,3] FP32, K = (sh_degree+1)^2; 16-B
 *   inst_offsets   [n_inst+2] int64: segment k covers [off[k], off[k+1]),
 *                  off[0] = 0, off[n_inst+1] = n; segment 0 is static.
 * The library never writes these. */
typedef struct {
  int64_t n;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  int32_t sh_degree;
  const int64_t* inst_offsets;
  int32_t n_inst;
} s3r_scene;

/* Per-instance pose at time t, the W_{t,i2g} of Sec. 3.3 (local -> world):
 * rotation R(q/|q|) and translation. Device pointers [n_inst,4] (16-B) and
 * [n_inst,3]. */
typedef struct {
  const float* quat;
  const float* trans;
} s3r_poses;

/* Gradient outputs with the layouts of s3r_scene / s3r_poses, device
 * buffers. By default ACCUMULATED (+=) into caller-zeroed buffers, so that
 * calls over different cameras sum; in the overwrite mode of
 * s3r_set_grad_mode every element of every non-NULL buffer is written
 * instead (zeros for the Gaussians kept in no view), so the caller zeroes
 * nothing. Any pointer may be NULL to skip it (its work is still done where
 * other outputs need it). */
typedef struct {
  float* means;           /* [n,3] */
  float* log_scales;      /* [n,3] */
  float* quats;           /* [n,4] */
  float* opacity_logits;  /* [n]   */
  float* sh;              /* [n,K,3] */
  float* inst_quat;       /* [n_inst,4] */
  float* inst_trans;      /* [n_inst,3] */
} s3r_grads;

typedef struct {
  int64_t max_gaussians;   /* n of the largest scene */
  int64_t max_splats;      /* kept (Gaussian, view) pairs per call */
  int64_t max_duplicates;  /* (tile, splat) pairs per call, < 2^31 */
  int32_t max_views;       /* cameras per call, <= S3R_MAX_VIEWS */
  int32_t max_instances;   /* dynamic instances (static segment not counted) */
  int64_t max_tiles;       /* 16x16 tiles summed over the cameras of a call */
  int64_t max_pixels;      /* pixels summed over the cameras of a call */
  int64_t max_rows;        /* row-table entries of s3r_sort's tile counts (one per row of
                              tiles of a splat's rectangle past its third); 0: 4 x
                              max_splats. A splat whose rows do not fit is expanded from
                              its stored alpha region instead: the same pairs, computed
                              again. */
} s3r_capacity;

typedef struct {
  int64_t n_selected;      /* Gaussians whose window contains t */
  int64_t n_splats;        /* kept (Gaussian, view) pairs */
  int64_t n_duplicates;    /* (tile, splat) pairs */
  int64_t n_frustum;       /* selected Gaussians inside at least one frustum */
  int64_t n_blend_pairs;   /* counting mode: (pixel, splat) pairs of the tile lists the last
                              counted forward walked (each pixel up to its stop) */
  uint32_t device_status;  /* latched bits: 1 capacity, 2 timeout */
  uint32_t epoch;          /* call counter of the last s3r_project (stochastic-LOD draws) */
  int64_t n_eval_fwd;      /* counting mode: pairs the last counted forward evaluated (its
                              warp's footprint test passed and the pixel had not stopped) */
  int64_t n_eval_bwd;      /* counting mode: pairs the last counted backward evaluated (in its
                              warp's recorded contributors, up to the pixel's last one) */
} s3r_counts;

typedef struct s3r_workspace s3r_workspace;

/* Allocate a workspace for the given capacities on `device` (the current
 * device is restored afterwards). The workspace owns every intermediate of a
 * call sequence: the selected index list, the projected splats, keys, tile
 * ranges, the final transmittance and contributor counts of each pixel, and
 * per-splat gradients. Returns S3R_ERR_CUDA if the allocation fails. */
s3r_status s3r_workspace_create(const s3r_capacity* cap, int device, s3r_workspace** out);
s3r_status s3r_workspace_destroy(s3r_workspace* ws);
/* Bytes of device memory held by the workspace. */
int64_t s3r_workspace_bytes(const s3r_workspace* ws);

/*
 * Steps 1-4 + colour for one timestep over n_views cameras (Sec. 3.3).
 *   cams        HOST array [n_views] (copied into kernel parameters).
 *   t           normalised rendering time in [-1, 1] (Sec. 3.3).
 *   vis_window  [n,2] FP32 (v_s, v_e); selected iff v_s <= t <= v_e (FP32).
 *   point_life  [n,2] FP32 (l_s, l_e), updated in place by Eq. 5 for every
 *               selected Gaussian inside at least one camera's frustum
 *               (M_t, before the LOD cull); NULL skips the update.
 *   lod_threshold  r in pixels: a Gaussian is culled from a view iff the
 *               square root of the largest eigenvalue of its 2D covariance
 *               (before the 0.3 px^2 dilation) is < r. r <= 0 culls nothing.
 * Writes only workspace state. Sizes: n <= max_gaussians, n_views <=
 * max_views, n_inst <= max_instances, tiles/pixels within capacity. */
s3r_status s3r_project(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                       const s3r_camera* cams, int32_t n_views, float t,
                       const float* vis_window, float* point_life, float lod_threshold,
                       void* stream);

/* Step 5a: duplicate every kept splat into one (tile, splat) pair per 16x16
 * tile its 3-sigma rectangle touches, and sort the pairs by the 64-bit key
 * (view-tile id << 32 | FP32 depth bits), stably in projection order (a
 * least-significant-digit radix sort: the depth digits run on the splats
 * before duplication, the tile digits on the pairs). Then the [start, end)
 * range of every tile. Reads and writes workspace state only. */
s3r_status s3r_sort(s3r_workspace* ws, void* stream);

/* Step 5b: front-to-back alpha blending of every tile (Eq. 2) with the 3DGS
 * thresholds (alpha = min(0.99, o G), skipped below 1/255, stop before T
 * would fall under 1e-4).
 *   background  [3] FP32 composited with the final transmittance.
 *   out_rgb     [sum_v 3*H_v*W_v] FP32: view v's planar [3,H_v,W_v] image
 *               at offset 3 * (sum of the pixel counts of views < v).
 * Keeps the final T and the contributor count of each pixel for the
 * backward pass. */
s3r_status s3r_render_fwd(s3r_workspace* ws, const float* background, float* out_rgb, void* stream);

/* Step 6: gradient of sum(dL_drgb * rgb) w.r.t. all parameters and poses.
 * Must follow s3r_render_fwd on the same workspace with the same scene and
 * poses. Walks each tile back to front from its stored final transmittance
 * (no per-pixel lists), reduces per warp before global atomics, then chains
 * the 2D gradients through Eq. 1 to the parameters and through the composed
 * matrices W_t W_{t,i2g} to every instance pose.
 *   dL_drgb     same layout as out_rgb.
 *   grads       accumulated (+=).
 * Adjoints of clamped quantities (alpha at 0.99, the x/z and y/z clamp of the
 * Jacobian, negative colours) are zero, as in the exact derivative. */
s3r_status s3r_render_bwd(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                          const float* background, const float* dL_drgb,
                          const s3r_grads* grads, void* stream);

enum {
  S3R_VIS_RECORD = 0,    /* Eq. 5 on the Gaussians whose mask bit is set */
  S3R_VIS_FINALIZE = 1,  /* Eq. 6: v = (l_s - 0.1, l_e + 0.1), FP32 */
  S3R_VIS_RESET = 2      /* v = (-1, 1), l = (1, -1): visible at all times */
};

/* The temporal-visibility record (Sec. 3.3, Eqs. 5-6) over n Gaussians.
 *   mask        RECORD only: [ceil(n/32)] uint32 bitmask, bit i = M_t[i].
 *   point_life  [n,2] FP32 (l_s, l_e); vis_window [n,2] FP32 (v_s, v_e).
 * RECORD updates point_life; FINALIZE writes vis_window from point_life;
 * RESET writes both (new Gaussians appended at the end are reset by passing
 * pointers offset to their first index). */
s3r_status s3r_update_visibility(int64_t n, float t, const uint32_t* mask, float* point_life,
                                 float* vis_window, int32_t mode, void* stream);

/* Photometric L1 loss of a rendered batch (the paper does not state its
 * loss; this is the plain mean absolute error a training step can use):
 *   loss = sum |pred - target| / n   (written to *loss_out, one FP32 scalar)
 *   dL_dpred[i] = sign(pred[i] - target[i]) / n   (written)
 * pred, target, dL_dpred: [n] FP32 device arrays; loss_out: device FP32. */
s3r_status s3r_l1_loss(int64_t n, const float* pred, const float* target, float* dL_dpred,
                       float* loss_out, void* stream);

/* One Adam step over several parameter tensors in a single launch (the
 * optimiser of the training configuration; the paper states none and uses
 * the density control and optimiser of its baseline). For each element:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * (PyTorch's Adam without weight decay). `tensors` is a HOST array of up to
 * S3R_ADAM_MAX_TENSORS descriptors of device arrays (FP32, n elements each,
 * 4-byte aligned); param, exp_avg and exp_avg_sq are updated in place.
 * `gate` (may be NULL) is a device uint32 read by the kernel: if it is not 0
 * the step changes nothing. Passing s3r_device_status(ws) skips the update
 * whenever a call of the workspace has latched a failure (dropped splats or
 * pairs, a wait that gave up) since the status was last read, so that a
 * truncated render never reaches the parameters, with no host
 * synchronisation. */
#define S3R_ADAM_MAX_TENSORS 8
typedef struct {
  float* param;
  const float* grad;
  float* exp_avg;
  float* exp_avg_sq;
  int64_t n;
} s3r_adam_tensor;
s3r_status s3r_adam_step(const s3r_adam_tensor* tensors, int32_t count, float lr, float beta1,
                         float beta2, float eps, int32_t step, const uint32_t* gate, void* stream);

/* Device address of the workspace's latched status word (0 while no failure
 * is latched; bits 1 capacity, 2 timeout), for s3r_adam_step's gate. Valid
 * for the workspace's lifetime; NULL for a NULL workspace. */
const uint32_t* s3r_device_status(const s3r_workspace* ws);

/* The conventional pipeline of Fig. 1(a), the comparator that the
 * instance-specific projection of Sec. 3.3 replaces: every Gaussian of a
 * dynamic instance k is moved to the world frame by its pose at time t,
 *   mu_w = R(q_k/|q_k|) mu + t_k,   q_w = (q_k/|q_k|) (x) (q/|q|)
 * (Hamilton product, so R(q_w) = R(q_k) R(q)), and with sh_out its SH
 * coefficients are rotated so that the world-frame view direction gives the
 * colour the object-frame direction gives: band l (1 <= l <= sh_degree)
 * becomes D_l^T c_l per channel, Y_l(R_k^T d) = D_l Y_l(d) (D_l from an exact
 * 26-point Lebedev quadrature of the rotated basis against the basis); band
 * 0 is copied. scene and poses as for s3r_project. Only the rows of the
 * dynamic Gaussians ([inst_offsets[1], n)) of means_out [n,3] (4-B aligned),
 * quats_out [n,4] (16-B aligned) and sh_out [n,K,3] (16-B aligned, like the
 * scene's SH; or NULL) are written:
 * static Gaussians do not move, so the caller fills their rows once (a copy).
 * A scene of these arrays with no instances (inst_offsets {0, n}) then
 * renders the same image through s3r_project. S3R_ERR_INVALID on NULL or
 * misaligned arrays, nothing launched. */
s3r_status s3r_to_world(const s3r_scene* scene, const s3r_poses* poses, float* means_out,
                        float* quats_out, float* sh_out, void* stream);

/* Backward of s3r_to_world, in place: on entry grads->means, grads->quats and
 * grads->sh (each may be NULL; quats and sh 16-byte aligned) hold, at the
 * rows of dynamic Gaussians, the
 * adjoints of the world-frame means, quaternions and rotated SH (as the
 * backward of the world-frame render writes them); on return those rows
 * hold the adjoints of the object-frame parameters (the static rows, whose
 * transform is the identity, are not touched). grads->inst_quat [n_inst,4]
 * and grads->inst_trans [n_inst,3] are WRITTEN with the pose adjoints. The
 * per-instance sums use the workspace (its max_instances bounds n_inst);
 * calls on one workspace must not overlap on the GPU. */
s3r_status s3r_to_world_bwd(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                            const s3r_grads* grads, void* stream);

/* Level of detail (Sec. 3.3 "Adaptive LOD", Eq. 7). In the default
 * S3R_LOD_THRESHOLD mode every in-frustum Gaussian whose projected 2D scale
 * (square root of the largest eigenvalue of the undilated 2D covariance, in
 * pixels) is below the lod_threshold r of s3r_project is culled. In
 * S3R_LOD_STOCHASTIC mode those Gaussians are instead dropped with the
 * depth-dependent probability of Eq. 7,
 *   p = p_max + (p_max - 0.01) * min(0, (d - distance) / distance),
 * d the camera-space depth, and the survivors are rendered at a noisy mean
 *   mu + offset * min(1, d / distance) * (n0, n1, n2),  n ~ N(0, 1) per axis,
 * in the Gaussian's own frame (the noise is a constant for the gradient).
 * Draws are Philox4x32-10 of the counter (Gaussian id, view index in the
 * call, call epoch, block 0/1) under the key (seed low, seed high); the
 * epoch increments with every s3r_project of the workspace (and with every
 * replay of a captured sequence) and is reported by s3r_query_counts. The
 * setting applies to the following s3r_project and s3r_render_bwd calls of
 * the workspace; params NULL restores the threshold mode. Requires
 * 0 <= p_max <= 1 and distance > 0. */
#define S3R_LOD_THRESHOLD 0
#define S3R_LOD_STOCHASTIC 1
typedef struct {
  int32_t mode;
  float p_max;
  float distance;
  float offset[3];
  uint64_t seed;
} s3r_lod_params;
s3r_status s3r_set_lod(s3r_workspace* ws, const s3r_lod_params* params);

/* Gradient output mode of the following s3r_render_bwd calls of the
 * workspace. S3R_GRAD_ACCUMULATE (the default): the gradients are added to
 * the caller's buffers. S3R_GRAD_OVERWRITE: the call writes every element of
 * the n rows of each non-NULL Gaussian buffer and of the n_inst rows of the
 * pose buffers: the gradient rows of the Gaussians kept in at least one view
 * are written once, by the thread that computes them (no read of the old
 * contents), and the other rows are set to zero by a coalesced pass over a
 * per-Gaussian bitmap of the kept ones. The result equals accumulation into
 * zeroed buffers. */
#define S3R_GRAD_ACCUMULATE 0
#define S3R_GRAD_OVERWRITE 1
s3r_status s3r_set_grad_mode(s3r_workspace* ws, int32_t mode);

/* Work accounting: with counting enabled the blend kernels also count the
 * (pixel, splat) pairs they walk and evaluate (reported by s3r_query_counts;
 * the counts persist until the next counted call). Counting runs a separate
 * instantiation of each blend kernel with a few more instructions per pair,
 * so it is off by default and off while timing. */
s3r_status s3r_set_counting(s3r_workspace* ws, int32_t enable);

/* Failure-detection test hook: every device-side wait of the library (the
 * decoupled look-back of the scans and radix passes) is bounded, and on
 * give-up latches a timeout into the workspace status instead of hanging.
 * This call makes both look-back waits run out on purpose: one warp waits,
 * as tile 1, on a tile-0 word that nothing publishes, giving up after
 * `max_polls` polls (1 .. S3R_MAX_PROBE_POLLS; each poll sleeps ~20-40 ns, so
 * at most a few tens of milliseconds). Asynchronous on `stream`; the next
 * s3r_sync_status returns S3R_ERR_TIMEOUT and clears the status, and the
 * workspace stays usable (the hook writes only four look-back words that no
 * pass reads with a matching tag). Returns S3R_ERR_INVALID for a NULL
 * workspace or `max_polls` out of range, launching nothing. */
#define S3R_MAX_PROBE_POLLS (1 << 20)
s3r_status s3r_check_wait_timeout(s3r_workspace* ws, int32_t max_polls, void* stream);

/* Per-kernel device timing (tracing). With timing enabled, every kernel the
 * workspace's calls launch is bracketed by a pair of CUDA events owned by the
 * workspace (recorded on the caller's stream, so this also works inside a
 * captured CUDA graph). After the stream has been synchronised,
 * s3r_kernel_times writes the duration in milliseconds of the most recent
 * launch of each kernel id into ms[0..n) (-1 where it never ran).
 * s3r_kernel_name gives the name of an id in [0, s3r_kernel_count()). */
s3r_status s3r_set_timing(s3r_workspace* ws, int32_t enable);
int32_t s3r_kernel_count(void);
const char* s3r_kernel_name(int32_t id);
s3r_status s3r_kernel_times(s3r_workspace* ws, float* ms, int32_t n);

/* Allocation-free temporal selection. The paper has no counterpart: this is
 * a convenience for callers that cannot allocate device memory at all, e.g.
 * code running inside a host framework whose caching allocator owns the
 * whole device, or a real-time loop that may not call cudaMalloc after
 * start-up. It computes the same list as the selection step of s3r_project
 * (ascending ids i with vis_window[i] = (v_s, v_e), v_s <= t <= v_e, FP32)
 * without a workspace:
 *   n           number of Gaussians, 0 <= n <= S3R_STATIC_MAX_GAUSSIANS;
 *               larger n returns S3R_ERR_INVALID (nothing is launched).
 *   vis_window  [n,2] FP32 device array, 16-byte aligned.
 *   out_idx     [n] uint32 device array (caller-owned), receives the list.
 *   out_count   one uint32 in device memory, receives its length, or
 *               S3R_STATIC_TIMEOUT if a bounded look-back wait of the call
 *               gave up (out_idx is then not valid; the call itself cannot
 *               return S3R_ERR_TIMEOUT, which is only known on the device).
 * The look-back scratch is a fixed array in the library's device image
 * (about 128 KB, held by every GPU that loads the library until the process
 * exits); every call shares it and clears the part it uses on entry, so
 * calls that overlap on the GPU (e.g. on two streams at once) race and must
 * be serialised by the caller. The first call on a device looks up the
 * array's device address and the device's SM count (once per device); make
 * that first call before any stream capture. No allocation or free happens
 * in any call. */
#define S3R_STATIC_TIMEOUT 0xffffffffu
#define S3R_STATIC_MAX_GAUSSIANS (1LL << 26)
s3r_status s3r_select_visible_static(int64_t n, float t, const float* vis_window, uint32_t* out_idx,
                                     uint32_t* out_count, void* stream);

/* NeuralODE object poses (Sec. 3.2, Eqs. 3-4). Each dynamic instance's state
 * z(t) = [position (3), rotation vector r (3)] follows dz/dt = f(z, t, c) (Eq. 3),
 * f(z, t, c) = W3 tanh(W2 tanh(W1 [z, t, c] + b1) + b2) + b3 with hidden width
 * S3R_ODE_HIDDEN and c the instance's embedding (embed_dim <= S3R_ODE_MAX_EMBED
 * floats); Eq. 4's integral from z(t0) is taken with classical fourth-order
 * Runge-Kutta steps, `substeps` equal steps between consecutive output times.
 * The pose at an output time (the instance pose W_{t,i2g} of s3r_poses) is
 * the unit quaternion (cos(|r|/2), sin(|r|/2) r/|r|) (w, x, y, z) and the
 * translation z[0:3]. The paper names neither the network nor the
 * integrator: these are this library's choices.
 *   params  device [s3r_ode_param_count(embed_dim)] FP32: W1 (H x (7 + D),
 *           row-major), b1 (H), W2 (H x H), b2 (H), W3 (6 x H), b3 (6).
 *   embed   device [n_inst, embed_dim] FP32 (may be NULL when embed_dim = 0). */
#define S3R_ODE_HIDDEN 64
#define S3R_ODE_MAX_EMBED 16
typedef struct {
  int32_t embed_dim;
  const float* params;
  const float* embed;
} s3r_ode_net;
int64_t s3r_ode_param_count(int32_t embed_dim);

/* Forward (Eq. 4) for n_inst instances at once:
 *   z0      device [n_inst, 6] states at times[0];
 *   times   device [n_times] output times, ascending (n_times >= 1);
 *   states  device [(n_times - 1) * substeps + 1, n_inst, 6]: the state after
 *           every Runge-Kutta step (kept for s3r_ode_poses_bwd);
 *   quat    device [n_times, n_inst, 4] (16-byte aligned), trans [n_times,
 *           n_inst, 3]: the poses, so that quat + 4 n_inst j and trans +
 *           3 n_inst j are timestep j's s3r_poses.
 * S3R_ERR_INVALID on bad sizes or pointers, nothing launched. */
s3r_status s3r_ode_poses(const s3r_ode_net* net, int32_t n_inst, const float* z0,
                         const float* times, int32_t n_times, int32_t substeps, float* states,
                         float* quat, float* trans, void* stream);

/* Reverse mode of s3r_ode_poses (the exact derivative of its Runge-Kutta
 * steps): given dL/dquat and dL/dtrans at every output time (device, the
 * layouts of quat and trans; zeros where a time is not used), ADDS dL/dparams
 * [param_count], dL/dembed [n_inst, embed_dim] and dL/dz0 [n_inst, 6] into
 * caller-zeroed device buffers. `states` is the forward's output. The pose
 * adjoints of one timestep are the inst_quat / inst_trans gradients of
 * s3r_render_bwd. */
s3r_status s3r_ode_poses_bwd(const s3r_ode_net* net, int32_t n_inst, const float* times,
                             int32_t n_times, int32_t substeps, const float* states,
                             const float* g_quat, const float* g_trans, float* g_params,
                             float* g_embed, float* g_z0, void* stream);

/* Synchronise `stream`, then return the device counts of the last call
 * sequence and the latched device status (which it clears). Tests and logs
 * only. */
s3r_status s3r_query_counts(s3r_workspace* ws, void* stream, s3r_counts* out);
/* Synchronise `stream` and convert the latched device status into a return
 * value (S3R_ERR_CAPACITY / S3R_ERR_TIMEOUT), clearing it. */
s3r_status s3r_sync_status(s3r_workspace* ws, void* stream);

/* Resume support: set the workspace's call counter (s3r_counts.epoch) so that
 * the next s3r_project draws the stochastic-LOD numbers (Eq. 7) of call
 * `epoch` + 1, as the run that saved the counter would have. The counter
 * also tags the scans' look-back words, so the call clears those words (one
 * memset of the workspace's look-back array) and any value is accepted.
 * Synchronises `stream`. */
s3r_status s3r_set_epoch(s3r_workspace* ws, uint32_t epoch, void* stream);

/* Read-only views of workspace intermediates, for tests and tools (device
 * pointers, valid until the next s3r_project on the workspace).
 *   name: "selected" u32[n_selected] ascending Gaussian ids;
 *         "frustum_mask" u32[n_selected] bit v = inside camera v's frustum;
 *         "keep_mask" u32[n_selected] bit v = kept (frustum and LOD) in v;
 *         "splat_start" u32[n_selected] first splat of each selected Gaussian;
 *         "splat_record" 8 x 32-bit [n_splats]: float u, v, conic a, b, c
 *         (power = -0.5 (a dx^2 + c dy^2) - b dx dy), opacity, then x0|y0<<16
 *         and w|h<<13|view<<26|moved<<31 (all ones for views of more than
 *         8190 tiles in x or y); "splat_rgb_depth" float4;
 *         "splat_rect" uint2 (x0|y0<<16, x1|y1<<16,
 *         tiles, half-open); "splat_view" uint8;
 *         "sorted_splats" u32[n_duplicates] splat id per pair in key order;
 *         "sorted_tiles" u32[n_duplicates] view-tile id per pair;
 *         "tile_ranges" uint2[tiles]; "final_T" float[pixels];
 *         "n_contrib" u32[pixels]; "splat_grads" float[n_splats*12]
 *         (du, dv, dA, dB, dC, dopacity, dr, dg, db, 0, 0, 0);
 *         "pose_grad_matrix" float[n_views*(n_inst+1)*12] dL/dW_{t,i}.
 * Returns NULL for an unknown name. */
const void* s3r_debug_buffer(const s3r_workspace* ws, const char* name);

/* Thread-local message of the last non-OK status returned on this thread. */
const char* s3r_last_error(void);

/* Library version and the compute capability it was built for (e.g. 103). */
int32_t s3r_version(void);
int32_t s3r_built_arch(void);

#ifdef __cplusplus
}
#endif

#endif /* S3R_H_ */
