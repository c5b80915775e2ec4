/*
 * scgr.h - C ABI of the GB300 shape-constrained gravitational registration
 * library (method of Agarwal & Bhowmick, "3D Point Cloud Registration with
 * Shape Constraint", arXiv 1902.01061).
 *
 * The library registers a rigid template cloud Y (M points) to a reference
 * cloud X (N points) by translation, rotation and scale (Sec. I, problem
 * statement), without colour, correspondences or topology.  Every reference
 * point pulls every template point with a force weighted by the similarity of
 * their local curvature descriptors (Eq. 2-5, Eq. 10, Eq. 11); the per-point
 * forces give a displacement (Eq. 5.5), a Kabsch rotation (Eq. 6) and an
 * eigenvalue-ratio scale (Sec. III-B, Eq. 8), applied by Eq. 9 each
 * iteration with the gravitational-constant schedule of Eq. 12.
 *
 * Conventions (all calls):
 *  - Points are float32, row-major [n][3] (x, y, z), row-vector convention:
 *    the moved template is s * Y0 @ R + t (Eq. 9), R row-major 3x3 doubles.
 *  - "_dev" pointers are CUDA device pointers on the context's device;
 *    "_host" pointers are host memory (pageable or pinned).  The caller owns
 *    every pointer it passes.  Inputs are copied into context-owned device
 *    buffers before the call returns (stream-ordered on the context stream);
 *    outputs are caller-allocated.  The context owns all workspace and frees
 *    it in scgr_destroy.
 *  - Every call returns a status; nothing throws or aborts across the ABI.
 *    Kernels report through a device error word that is read at the next
 *    synchronising call (scgr_get_result, scgr_get_state, scgr_sync); its
 *    message is available from scgr_last_error until the next call on the
 *    same context.
 *  - Calls are enqueued on the stream given to scgr_create (NULL: the legacy
 *    default stream) and return without synchronising unless stated.
 *  - One context per host thread at a time; distinct contexts are independent.
 */
#ifndef SCGR_H
#define SCGR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SCGR_EXPORT __attribute__((visibility("default")))
#else
#define SCGR_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scgr_ctx scgr_ctx; /* opaque; owns all device workspace */

typedef enum {
  SCGR_OK = 0,
  SCGR_ERR_INVALID_ARG = 1, /* null pointer, bad size (n < k, m < 3), bad parameter */
  SCGR_ERR_STATE = 2,       /* call out of order (e.g. run before descriptors) */
  SCGR_ERR_NONFINITE = 3,   /* an input coordinate is NaN/Inf or |x| > 1e18 */
  SCGR_ERR_OOM = 4,         /* device allocation failed */
  SCGR_ERR_CUDA = 5,        /* a CUDA runtime call or a launch failed */
  SCGR_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  SCGR_ERR_NUMERIC = 7      /* the step became non-finite (e.g. zero total weight) */
} scgr_status;

/* Method parameters (Sec. III, Sec. IV). */
typedef struct {
  int k;           /* neighbours per curvature descriptor, self included (>= 3; default 16) */
  double p;        /* distance exponent of h(d) = d^p, Eq. 11, p >= 1 (default 1) */
  double sigma;    /* RBF spread of Eq. 3; <= 0: population std of the reference curvatures */
  int g_mode;      /* 0: g = s (equal weight, Sec. IV); 1: g = aX aY s (Eq. 10, default) */
  double G1;       /* Eq. 12 (default 10000) */
  int E;           /* Eq. 12 horizon; <= 0: the iteration count of the first scgr_run */
  int step_mode;   /* 0: normalized step kappa = eta0 (G/G1) M / W (default); 1: literal Eq. 5.5,
                      kappa = G time^2 */
  double eta0;     /* normalized step fraction, 0 < eta0 (default 0.5) */
  double time;     /* literal-mode time step of Eq. 5.5 (default 1) */
  int scale_mode;  /* 0: c = sqrt(eX/eY) (default); 1: c = eX/eY as printed; 2: c = 1 (rigid) */
  int use_graph;   /* 1: scgr_run captures its iteration loop in a CUDA graph and replays it */
  int neigh_mode;  /* curvature neighbourhood: 0 the k nearest neighbours (default); 1 all points within
                      radius radius_scale * sqrt(e) of the point, e the largest covariance eigenvalue of its
                      cloud (Sec. IV: radius sqrt(eX) for the reference, sqrt(eY) for the template) */
  double radius_scale; /* radius multiplier of neigh_mode 1 (default 1) */
} scgr_params;

/* Result of a registration (Eq. 6, Eq. 8, Eq. 9): moved = s * Y0 @ R + t. */
typedef struct {
  double R[9];          /* row-major, row-vector convention */
  double t[3];
  double s;
  int iterations;       /* iterations run so far on this context */
  int degenerate_steps; /* iterations whose cross-covariance had rank < 2 (rotation kept) */
} scgr_result;

/* Checkpoint of the iteration state (pose, position in the Eq. 12 schedule,
 * and sigma).  scgr_set_state + scgr_run continues bit-identically. */
typedef struct {
  double R[9];
  double t[3];
  double s;
  int iteration; /* next iteration index t of Eq. 12 */
  int E;         /* Eq. 12 horizon in use (0: not fixed yet) */
  int degenerate_steps;
  double sigma;  /* RBF spread in use (read-only on set: must match the context's) */
} scgr_state;

/* Fill *out with the defaults listed above.  Returns INVALID_ARG on NULL. */
SCGR_EXPORT scgr_status scgr_default_params(scgr_params* out);

/* Create a context bound to the current CUDA device and `cuda_stream`
 * (a cudaStream_t; NULL for the default stream).  *out is set to NULL on
 * failure.  Parameters are validated here (k >= 3, p >= 1, eta0 > 0, ...). */
SCGR_EXPORT scgr_status scgr_create(const scgr_params* params, void* cuda_stream, scgr_ctx** out);

/* Release every device buffer of the context.  NULL is ignored. */
SCGR_EXPORT void scgr_destroy(scgr_ctx* ctx);

/* Text of the last error on this context ("" if none).  Valid until the next
 * call on the same context.  NULL ctx: the last scgr_create failure. */
SCGR_EXPORT const char* scgr_last_error(const scgr_ctx* ctx);

/* Reference cloud X (Sec. II: absolute coordinates r^{Xj}), n >= k points.
 * Copied and validated on device; a non-finite coordinate is reported as
 * SCGR_ERR_NONFINITE at the next synchronising call.  Resets descriptors. */
SCGR_EXPORT scgr_status scgr_set_reference(scgr_ctx* ctx, const float* xyz_dev, int64_t n);
SCGR_EXPORT scgr_status scgr_set_reference_host(scgr_ctx* ctx, const float* xyz_host, int64_t n);

/* Template cloud Y0, m >= max(k, 3) points.  Same rules as the reference.
 * Resets descriptors and the pose to identity. */
SCGR_EXPORT scgr_status scgr_set_template(scgr_ctx* ctx, const float* xyz_dev, int64_t m);
SCGR_EXPORT scgr_status scgr_set_template_host(scgr_ctx* ctx, const float* xyz_host, int64_t m);

/* One-time descriptor pass (Sec. III-A, Sec. IV): k-nearest neighbours of
 * every point of X and of Y0 (exact float32 key (dx*dx+dy*dy)+dz*dz, no fused
 * multiply-add, self included, ties to the lower index; brute force for
 * small clouds, an exact uniform-grid search for large ones, which waits once
 * for the bounding box), the curvature
 * a = lambda_min / (lambda_1+lambda_2+lambda_3) of each neighbourhood's
 * covariance (float64), sigma, and the cloud statistics used by the scale
 * model (means, covariances, largest eigenvalues).  Resets the pose to
 * identity and the iteration counter to 0.  STATE if a cloud is missing. */
SCGR_EXPORT scgr_status scgr_compute_descriptors(scgr_ctx* ctx);

/* Enqueue `iterations` iterations (Eq. 5 - Eq. 12) on the context stream.
 * Resumable: consecutive calls continue the schedule.  The pose stays on the
 * device; no host synchronisation happens inside the loop.  STATE before
 * descriptors; INVALID_ARG for iterations < 0. */
SCGR_EXPORT scgr_status scgr_run(scgr_ctx* ctx, int iterations);

/* Synchronise the stream, check the device error word and copy the pose. */
SCGR_EXPORT scgr_status scgr_get_result(scgr_ctx* ctx, scgr_result* host_out);

/* Moved template s * Y0 @ R + t (Eq. 9) as float32 [m][3].  Enqueued. */
SCGR_EXPORT scgr_status scgr_get_moved(scgr_ctx* ctx, float* xyz_dev_out);
/* Same into host memory; synchronises. */
SCGR_EXPORT scgr_status scgr_get_moved_host(scgr_ctx* ctx, float* xyz_host_out);

/* Descriptors of the reference (which = 0) or the template (which = 1):
 * neighbour indices int32 [n][k] sorted by (key, index) and curvature
 * float32 [n].  Either output may be NULL.  Enqueued.  STATE before
 * descriptors. */
SCGR_EXPORT scgr_status scgr_get_descriptors(scgr_ctx* ctx, int which, int32_t* knn_dev, float* a_dev);

/* sigma in use and the float64 curvature of either cloud (a64_dev may be
 * NULL; [n] doubles).  Synchronises. */
SCGR_EXPORT scgr_status scgr_get_sigma(scgr_ctx* ctx, double* sigma_out);
SCGR_EXPORT scgr_status scgr_get_curvature64(scgr_ctx* ctx, int which, double* a64_dev);

/* Replace the curvature of the reference (which = 0) or the template
 * (which = 1) by caller-supplied float64 values a64_dev [n] (each in [0, 1];
 * non-finite values are rejected with SCGR_ERR_NONFINITE at the next
 * synchronising call).  sigma is recomputed from the reference curvatures
 * unless params.sigma > 0, the force records are rebuilt, and the pose and
 * iteration counter are reset to identity / 0.  The neighbour lists are kept.
 * For descriptors from another source (priors, a coarser neighbourhood) and
 * for tests whose oracle cannot afford the neighbour search.  STATE before
 * scgr_compute_descriptors. */
SCGR_EXPORT scgr_status scgr_set_curvature(scgr_ctx* ctx, int which, const double* a64_dev);

/* Pyramidal schedule (Sec. IV: for noisy data the neighbourhood size and
 * sigma shrink as the iterations proceed).  Recompute both clouds'
 * curvature with a new neighbourhood - k nearest (neigh_mode 0; 3 <= k <= 32)
 * or radius_scale * sqrt(e) (neigh_mode 1) - and set
 * sigma = sigma_scale * (params.sigma if > 0, else the population std of the
 * new reference curvatures).  The pose and the position in the Eq. 12
 * schedule are kept, so scgr_run continues the registration with the new
 * descriptors.  STATE before scgr_compute_descriptors; INVALID_ARG for
 * k outside [3, 32] or non-positive scales. */
SCGR_EXPORT scgr_status scgr_set_neighbourhood(scgr_ctx* ctx, int k, double radius_scale, double sigma_scale);

/* Nearest reference point of q_dev [nq][3] (float32): index int32 [nq] and
 * float32 key (squared distance, the kNN key of R1) [nq]; either output may
 * be NULL.  Ties go to the lower index.  References of at least
 * SCGR_TUNE_KNN_GRID_MIN points are searched through an exact uniform grid
 * (same result as brute force; queries may lie outside the reference's box),
 * which synchronises the stream once for the bounding box; smaller ones by
 * brute force, enqueued.  STATE without a reference. */
SCGR_EXPORT scgr_status scgr_nearest(scgr_ctx* ctx, const float* q_dev, int64_t nq, int32_t* idx_dev,
                                     float* key_dev);

/* Change detection after registration (abstract; Sec. V, real scenes: parts
 * of the template that moved between captures stay unaligned).  For every
 * point of the moved template s Y0 R + t, mask_dev[i] = 1 (uint8) if its
 * nearest reference point is farther than `threshold`, else 0; dist_dev
 * (nullable, float32 [m]) receives that distance.  The search is that of
 * scgr_nearest.  STATE before descriptors. */
SCGR_EXPORT scgr_status scgr_change_mask(scgr_ctx* ctx, double threshold, uint8_t* mask_dev, float* dist_dev);

/* Forces at the current pose without updating it: per template point
 * (fx, fy, fz, W) as float32 [m][4], where f is Eq. 5 without the factor G
 * (f_i = -sum_j g(s_ij) h(d_ij) n_ij) and W_i = sum_j g(s_ij) d_ij^(p-1).
 * Enqueued.  STATE before descriptors. */
SCGR_EXPORT scgr_status scgr_forces(scgr_ctx* ctx, float* f4_dev);

/* Differentiation form.  The shape-weighted potential
 *   U = sum_i sum_j g(s_ij) d_ij^(p+1) / (p+1)
 * whose negative gradient with respect to Y_i is the force of Eq. 5 (Eq. 3,
 * Eq. 10, Eq. 11; descriptors held fixed), evaluated at the pose
 * pose7 = (omega[3], t[3], s): Y = s * Y0 @ R + t with R = exp([omega]_x)^T
 * (axis-angle, row-vector convention).  Optional outputs: grad_pose7 (host,
 * 7 doubles: dU/domega, dU/dt, dU/ds) and grad_xyz_dev (device float32
 * [m][3]: dU/dY0).  The gradient pass recomputes the pair tiles of the force
 * kernel (no N x M storage); sums are float64 in a fixed order.  The
 * registration pose is not touched.  Synchronises.  STATE before
 * descriptors; INVALID_ARG for a non-finite pose or s <= 0. */
SCGR_EXPORT scgr_status scgr_potential(scgr_ctx* ctx, const double pose7[7], double* U_out,
                                       double* grad_pose7, float* grad_xyz_dev);

/* Same outputs as scgr_potential, computed the other way round for
 * comparison: the forward pass stores every pair weight w_ij (float32, M rows
 * of N rounded up to a multiple of 256, so 4 x M x ceil(N/256) x 256 bytes of
 * device memory, allocated on first use and kept by the context; OOM if it
 * does not fit) and the backward pass streams them back from HBM instead of
 * recomputing the tiles.  The weights use the special-function unit's ex2 and
 * lg2 like the force kernel.  Synchronises. */
SCGR_EXPORT scgr_status scgr_potential_stored(scgr_ctx* ctx, const double pose7[7], double* U_out,
                                              double* grad_pose7, float* grad_xyz_dev);

/* Vector-Jacobian product of the force field at the current pose:
 * grad_i = (d f_i / d Y_i)^T v_i with f_i of Eq. 5 (without G; descriptors
 * fixed).  f_i depends only on Y_i, and
 * d f_i / d Y_i = -aY_i sum_j w_ij [I + (p - 1) r_ij r_ij^T / d_ij^2].
 * v_dev and grad_dev are float32 [m][3] device arrays.  The reference tiles
 * are recomputed (no N x M storage).  Enqueued.  STATE before descriptors. */
SCGR_EXPORT scgr_status scgr_force_vjp(scgr_ctx* ctx, const float* v_dev, float* grad_dev);

/* Checkpoint / resume of the iteration state.  Both synchronise. */
SCGR_EXPORT scgr_status scgr_get_state(scgr_ctx* ctx, scgr_state* host_out);
SCGR_EXPORT scgr_status scgr_set_state(scgr_ctx* ctx, const scgr_state* host_in);

/* Wait for all work on the context stream and check the device error word. */
SCGR_EXPORT scgr_status scgr_sync(scgr_ctx* ctx);

/* Device timing of the all-pairs force kernel (diagnostic).  While enabled,
 * every force-kernel launch enqueued outside graph capture is bracketed by
 * CUDA events on the context stream.  scgr_set_force_timing(ctx, 1) enables
 * and resets the tally, (ctx, 0) disables it.  scgr_get_force_timing
 * synchronises and returns the number of timed launches and the sum of their
 * durations in milliseconds since the last reset. */
SCGR_EXPORT scgr_status scgr_set_force_timing(scgr_ctx* ctx, int enable);
SCGR_EXPORT scgr_status scgr_get_force_timing(scgr_ctx* ctx, int64_t* launches, double* total_ms);

/* Allocation-free force evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory - hosts whose
 * device memory is owned by another allocator (a framework's caching pool,
 * a fixed budget on an embedded robot) and real-time loops that cannot take
 * cudaMalloc's latency or the device-wide synchronisation a cudaFree can
 * cause.  It needs no context.
 *
 * Computes what scgr_forces computes at the identity pose - per template
 * point (fx, fy, fz, W) as float32 [m][4] - for the caller's clouds
 * x_dev [n][3], y_dev [m][3] (float32) and curvatures ax_dev [n], ay_dev [m]
 * (float64, each in [0, 1]).  sigma <= 0 selects the population std of ax;
 * p >= 1; g_mode as in scgr_params.  All intermediate buffers live in one
 * file-scope device array of fixed size (about 25 MB, held by every GPU that
 * loads the library until the process exits); nothing is allocated.
 *
 * Limits: 1 <= n, m <= 131072 points; larger sizes return
 * SCGR_ERR_INVALID_ARG.  A non-finite coordinate or a curvature outside
 * [0, 1] returns SCGR_ERR_NONFINITE.  The call runs on `cuda_stream` and
 * synchronises it before returning.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  Every call shares the
 * array, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The looked-up address
 * is kept for the life of the process: after a cudaDeviceReset (which
 * destroys the device's primary context, and the array with it) do not call
 * this entry point again in that process. */
SCGR_EXPORT scgr_status scgr_forces_static(const float* x_dev, int64_t n, const float* y_dev, int64_t m,
                                           const double* ax_dev, const double* ay_dev, double sigma,
                                           double p, int g_mode, float* f4_dev, void* cuda_stream);

/* Batching form: npairs independent registrations of uneven sizes in one
 * call, with the context's parameters.  Pair p's reference is rows
 * [ref_off[p], ref_off[p+1]) of ref_xyz_dev and its template rows
 * [tmp_off[p], tmp_off[p+1]) of tmp_xyz_dev (float32 [.][3] device arrays;
 * ref_off/tmp_off are host int64 arrays of npairs + 1 offsets starting at 0).
 * Descriptors for all clouds run in one launch per stage; each iteration is
 * three launches for all pairs (force work items sorted longest first, one
 * block per item or a persistent grid taking items from a queue, see
 * SCGR_TUNE_BATCH_PERSISTENT, with one kernel shape for all pairs or a shape
 * per pair, see SCGR_TUNE_BATCH_P; a per-pair fixed-order combine; one
 * float64 finalize block per pair); with
 * params.use_graph the iteration loop is captured in a CUDA graph and
 * replayed.  results_host[p] receives pair p's pose (as scgr_get_result).
 * The single-registration state of the context is not touched.
 * Synchronises.  INVALID_ARG for bad offsets (a reference with fewer than k
 * points, a template with fewer than max(k, 3)). */
SCGR_EXPORT scgr_status scgr_batch_run(scgr_ctx* ctx, int npairs, const int64_t* ref_off_host,
                                       const float* ref_xyz_dev, const int64_t* tmp_off_host,
                                       const float* tmp_xyz_dev, int iterations, scgr_result* results_host);

/* Template-row sharding of one registration over several processes (one
 * GPU each).  scgr_set_row_range restricts the force pass of this context
 * to template rows [row0, row0 + rows) (call after scgr_set_template and
 * before scgr_compute_descriptors; statistics still use the whole template).
 * An iteration is then split in two: scgr_step_partials computes this
 * rank's 13 float64 partial sums (total force F[3], total weight W, moment
 * T[3][3] = sum_i f_i (Y_i - ybar)^T over its rows; synchronises), the caller
 * adds the ranks' partials in a fixed order (an all-reduce of 13 doubles),
 * and scgr_step_apply(totals) performs the pose update (Eq. 5.5 - Eq. 12) from
 * the totals (synchronises).  Ranks that apply identical totals hold
 * identical poses.  Stepwise iteration needs params.E > 0.  With a row range
 * set, scgr_run and scgr_potential return STATE and scgr_forces writes the
 * range's rows only ([rows][4]). */
SCGR_EXPORT scgr_status scgr_set_row_range(scgr_ctx* ctx, int64_t row0, int64_t rows);
SCGR_EXPORT scgr_status scgr_step_partials(scgr_ctx* ctx, double out13[13]);
SCGR_EXPORT scgr_status scgr_step_apply(scgr_ctx* ctx, const double tot13[13]);

/* Stream-ordered forms of the same two halves, for an exchange that stays on
 * the device (an NCCL all-gather enqueued on the context stream between
 * them).  Neither copies to or from the host nor synchronises; device-side
 * errors surface at the next synchronising call.
 * scgr_step_partials_dev writes this rank's 13 float64 partial sums (F[3], W,
 * T[3][3] row-major, as scgr_step_partials) to out13_dev (device, 13 doubles,
 * 8-byte aligned, owned by the caller).
 * scgr_step_apply_dev takes the ranks' partial sums gathered in rank order,
 * parts_dev = [nparts][13] doubles on the device (1 <= nparts <= 65536), adds
 * them in that order on the device and performs the pose update of
 * Eq. 5.5 - Eq. 12 with the totals.  Ranks that pass identical parts hold
 * identical poses.  STATE before descriptors or without params.E > 0;
 * INVALID_ARG for NULL or a bad nparts. */
SCGR_EXPORT scgr_status scgr_step_partials_dev(scgr_ctx* ctx, double* out13_dev);
SCGR_EXPORT scgr_status scgr_step_apply_dev(scgr_ctx* ctx, const double* parts_dev, int nparts);

/* Tuning knobs (set by the autotuner; defaults are sensible). */
#define SCGR_TUNE_BATCH_CHUNK_TILES 1 /* reference tiles (256 points) per batched work item, default 16 */
#define SCGR_TUNE_KNN_GRID_MIN 2      /* clouds of at least this many points use the exact grid kNN in
                                         scgr_compute_descriptors (default 20000, where the two cost the
                                         same on GB300; 0: always); the result is identical */
#define SCGR_TUNE_NEAREST_GRID_MIN 14 /* references of at least this many points answer scgr_nearest and
                                         scgr_change_mask through the exact grid search (default 65536:
                                         below it the brute force is faster, also for queries far off
                                         the surface; 0: always); the result is identical */
#define SCGR_TUNE_FORCE_P 3           /* force kernel template points per thread: 0 auto, 1, 2, 4 */
#define SCGR_TUNE_FORCE_TPB 4         /* force kernel threads per block: 0 auto, 128, 256 */
#define SCGR_TUNE_FORCE_SPLITS 5      /* force kernel reference splits: 0 auto (wave-filling), >= 1 */
#define SCGR_TUNE_BATCH_P 8           /* template points per thread in the batched force kernel: 1 (default)
                                         or 2 (128 threads per block), or 4 (64 threads per block, running
                                         sums in shared memory); 0 mixed: per pair, 4 points x 128 threads
                                         (512-point template blocks, running sums in shared memory) where
                                         that padding costs less than the shape gains, else 2 x 128, both
                                         in one launch (the persistent form is not used with 0) */
#define SCGR_TUNE_FORCE_OCC 7         /* force kernel variant: 0 registers only, 2 resident blocks per SM;
                                         1 a tighter register budget and more resident blocks per SM (3 at
                                         256 threads, 4 at 128); 2 the per-point running sums in shared
                                         memory and 512 reference points staged per step (for 4 points x
                                         128 threads, 3 blocks per SM, and 2 points x 256 threads; other
                                         shapes use 0).  Until set: 2 for the 4 x 128 shape that templates
                                         of >= 311,296 points get (152 SMs), else 0 */
#define SCGR_TUNE_FORCE_RSQRT 9       /* p = 2 distance factor d = sqrt(d^2): 0 automatic (the square
                                         root), 1 d^2 * rsqrt(d^2), 2 the square root; all-pairs and
                                         batched force kernels; results agree to rounding.  On GB300
                                         rsqrt costs the special-function unit as much as sqrt, so form 1
                                         only adds a multiply; the autotuner times both */
#define SCGR_TUNE_BATCH_PERSISTENT 10 /* batched force pass: 0 (default) one block per work item, the
                                         items ordered longest first; 1 one persistent block per resident
                                         slot, each taking the next item (same order) from a queue head in
                                         device memory that is cleared before every launch.  Results are
                                         bit-identical: an item's sums do not depend on which block takes it */
#define SCGR_TUNE_FORCE_EX2POLY 11   /* p = 2 with the shared-memory-sum shapes (variant 2): 0 (default) every
                                         pair's similarity factor 2^-e from the special-function unit's ex2;
                                         1 or 2: for that many template points per thread, one of the two
                                         packed pair updates of each 4-point step evaluates it on the FP32
                                         pipe instead (range reduction to [-1/2, 1/2] and a degree-5 minimax
                                         polynomial, relative error < 2^-22; 2^-e below 2^-125.5 reads 0),
                                         which moves a fraction value / (2 P) of the exponentials off the
                                         special-function unit.  Results agree with 0 to rounding */
#define SCGR_TUNE_NEAREST_LEVELS 12  /* nearest-point search over a gridded reference (scgr_nearest,
                                         scgr_change_mask): 2 (default) fine cells around the query, then
                                         coarse cells of 4 x 4 x 4 fine cells that skip empty ones and ones
                                         beyond the best distance so far; 1 fine shells only.  The result
                                         is the same */
#define SCGR_TUNE_FUSED_TAIL 13      /* 1 (default): for templates of at most 2,048 padded slots one launch
                                         per iteration combines the split partials and updates the pose
                                         (one block); 0: the combine kernel and the finalize kernel, as for
                                         larger templates.  The two group the float32 per-point terms
                                         differently before the float64 sums, so poses agree to rounding */
#define SCGR_TUNE_REUSE_POSE_FREE 6   /* 1 (default): odd integer p skips the per-iteration all-pairs pass.
                                         p = 1: the pair weights do not depend on the pose, so scgr_run
                                         computes the force sums once per call and reuses them
                                         (bit-identical).  p = 3: the sums are a quadratic form in the
                                         template point over 14 moments of the similarity weights,
                                         computed once per call (equal up to rounding).  0: the all-pairs
                                         pass in every iteration */
/* Set one knob.  A force-plan knob re-plans at once when descriptors exist
 * (records and workspace are rebuilt; descriptors and pose are kept),
 * otherwise at scgr_compute_descriptors.  INVALID_ARG for an unknown key or
 * value. */
SCGR_EXPORT scgr_status scgr_set_tuning(scgr_ctx* ctx, int key, int value);
/* The force plan in use: out = {points per thread, threads per block,
 * reference splits, template blocks, occupancy variant}.  STATE before
 * descriptors. */
SCGR_EXPORT scgr_status scgr_get_plan(scgr_ctx* ctx, int out[5]);
/* The automatic force plan for n reference and m template points at
 * distance exponent p on a GPU with num_sms SMs where the planned kernel
 * keeps blocks_per_sm blocks resident (host-only arithmetic, no device
 * call; a context queries the device for blocks_per_sm).  out = {points per
 * thread, threads per block, occupancy variant, reference splits, tiles of
 * 256 reference points per split, template blocks, half-tile splits (0/1)}.
 * INVALID_ARG for n, m < 1, p < 1, num_sms < 1 or blocks_per_sm < 1. */
SCGR_EXPORT scgr_status scgr_plan_preview(int64_t n, int64_t m, double p, int num_sms, int blocks_per_sm,
                                          int out[7]);

/* Throughput microbenchmark of the units that bound the force kernel (no
 * paper counterpart; roofline evidence).  kind: 0 scalar FFMA, 1 packed
 * fma.f32x2, 2 MUFU ex2, 3 MUFU sqrt, 4 MUFU lg2.  Runs `blocks` x 256
 * threads (8 x the SM count fills the GPU) on the caller's scratch out_dev
 * (blocks x 256 floats); returns the FP32 lane operations (a packed FMA
 * counts 2) or special-function results of one launch and the best device
 * time (ms) of three launches.  Synchronises the stream. */
SCGR_EXPORT scgr_status scgr_microbench(int kind, int blocks, float* out_dev, void* cuda_stream,
                                        int64_t* lane_ops, double* ms);

/* Test hook (host-side fault injection): the next `count` workspace
 * allocations of any context fail as if the device were out of memory
 * (SCGR_ERR_OOM), without asking the device.  0 switches it off. */
SCGR_EXPORT scgr_status scgr_debug_fail_allocations(int count);

/* Number of kernel launches this context has issued so far (diagnostic). */
SCGR_EXPORT int64_t scgr_launch_count(const scgr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SCGR_H */
