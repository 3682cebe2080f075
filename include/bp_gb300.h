/*
 * bp_gb300 -- motion-compensated cone-beam backprojection and its analytic
 * vector-Jacobian products on NVIDIA GB300 (sm_103a).
 *
 * The operations follow arXiv 2401.09283 (Thies et al., "A gradient-based
 * approach to fast and accurate head motion compensation in cone-beam CT"):
 *   - Eq. 1   rigid motion composition  Phat_j = P_j T(theta_j);
 *   - Eq. 3   voxel-driven backprojection I(p) = sum_j d_j(g(Phat_j p~));
 *   - Eqs. 4-5 the derivative of a backprojected value with respect to the
 *             twelve entries of Phat_j, evaluated only as vector-Jacobian
 *             products (Sec. II-B.2, last paragraph);
 *   - Eq. 2   the chain rule down to the six motion parameters per view;
 *   - Eq. 6   gradient descent with an exponentially decaying step.
 *
 * Conventions shared by every call:
 *   - world coordinates in mm.  Voxel (i,j,k) sits at origin + (i,j,k)*spacing
 *     and volumes are stored [nz][ny][nx], x fastest, float32, contiguous;
 *   - projections are stored [nviews][nv][nu] with element strides
 *     row_stride (between detector rows) and view_stride (between views);
 *     u is the fastest axis; integer detector coordinates are pixel centres;
 *     samples outside the detector read zero (zero padding);
 *   - projection matrices are 3x4 row-major float64, (u,v,w) = P (x,y,z,1);
 *     a view whose w <= 0 at a voxel contributes nothing there;
 *   - motion parameters theta_j = (tx,ty,tz [mm], rx,ry,rz [rad]) define
 *     T = [[R t],[0 1]] with R = Rz(rz) Ry(ry) Rx(rx), rotation about the
 *     world origin (the isocenter);
 *   - with BP_WEIGHT_FDK each sample is weighted c_j * (sid / w)^2, with
 *     BP_WEIGHT_NONE by c_j alone (the paper's Eq. 3 has c_j = 1).
 *
 * Memory and ownership: every array argument is caller-owned and may be
 * either device memory or host memory (pageable or pinned); the library
 * tells them apart with cudaPointerGetAttributes.  Host inputs are copied to
 * a device staging area owned by the context; host outputs are copied back
 * and the call synchronises its stream before returning.  With only device
 * pointers, calls are asynchronous on `stream` (a cudaStream_t, NULL for the
 * legacy default stream).  The library never frees caller memory.
 *
 * Errors: every call returns a bp_status.  Invalid arguments are reported
 * before any work is queued; CUDA launch or copy failures return
 * BP_ERR_CUDA.  bp_last_error() gives a message for the last failure on the
 * context.  Nothing in the library aborts, traps or spins without a bound.
 *
 * Thread safety: a context may be used by one host thread at a time.
 */
#ifndef BP_GB300_H
#define BP_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BP_OK = 0,
  BP_ERR_INVALID_ARG = -1,
  BP_ERR_OOM = -2,
  BP_ERR_CUDA = -3,
  BP_ERR_UNSUPPORTED = -4,
  BP_ERR_TIMEOUT = -5,
  BP_ERR_CANCELLED = -6
} bp_status;

typedef enum { BP_F32 = 0, BP_F16 = 1, BP_BF16 = 2 } bp_dtype;

/* Eq. 3 literally (NONE) or with the FDK distance weight (sid/w)^2. */
typedef enum { BP_WEIGHT_NONE = 0, BP_WEIGHT_FDK = 1 } bp_weight;

/* How g_u, g_v of Eq. 4 are obtained: CENTRAL = bilinear interpolation of
 * gradient images made by central differences (second order in the
 * interior, one-sided first order on the two edge pixels), as Sec. II-B.2
 * describes; BILINEAR_EXACT = the exact partial derivatives of the bilinear
 * interpolant (the true derivative of Eq. 3, used for gradient checks). */
typedef enum { BP_DERIV_CENTRAL = 0, BP_DERIV_BILINEAR_EXACT = 1 } bp_deriv;

typedef struct {
  int nx, ny, nz;
  double spacing[3]; /* mm */
  double origin[3];  /* centre of voxel (0,0,0), mm */
} bp_vol_desc;

typedef struct {
  int nu, nv, nviews;
  int dtype;                   /* bp_dtype */
  long long row_stride;        /* elements between detector rows (>= nu) */
  long long view_stride;       /* elements between views (>= nv*row_stride) */
  const float* view_scale;     /* optional per-view dequantisation scale,
                                  value = scale[j] * stored; NULL = 1 */
  double sid;                  /* source-isocenter distance, mm (FDK weight) */
} bp_proj_desc;

typedef struct bp_ctx bp_ctx;

/* Create a context bound to CUDA device `device`.  The context owns only
 * workspace (per-view tables, gradient images, partial sums, staging).
 * Returns BP_ERR_INVALID_ARG for a bad device, BP_ERR_CUDA if the device
 * cannot be used (including a device that is not sm_103). */
int bp_ctx_create(int device, bp_ctx** out);
void bp_ctx_destroy(bp_ctx* ctx);
/* Message of the last failure on ctx ("" if none); valid until the next call. */
const char* bp_last_error(const bp_ctx* ctx);
/* Bytes of device workspace currently held by the context. */
long long bp_ctx_workspace_bytes(const bp_ctx* ctx);

/* Kernel accounting.  bp_ctx_launch_count: number of kernels the context
 * has launched since it was created.  bp_ctx_set_timing(ctx, 1) resets the
 * per-kernel totals and brackets every later launch with a pair of CUDA
 * events on the launching stream; bp_ctx_timing() then waits for the
 * recorded events and returns the summed device time (ms) and the number of
 * launches of one kernel: "compose", "forward", "grad_images",
 * "vjp_motion", "reduce_chain", "vjp_proj", "vjp_fused" (motion and data VJP
 * in one pass, used when bp_vjp is asked for both), "sharpness",
 * "optimizer", "spline" (Akima motion model) or "fdk_filter".
 * The paper has no counterpart; this is instrumentation for benchmarks. */
long long bp_ctx_launch_count(const bp_ctx* ctx);
int bp_ctx_set_timing(bp_ctx* ctx, int enable);
int bp_ctx_timing(bp_ctx* ctx, const char* kernel, double* total_ms, long long* launches);

/* Throughput probes behind the roofline figures (instrumentation; the paper
 * has no counterpart).  *result, per second on the context's device:
 *   kind 0  FP32 FMA lane operations with scalar FFMA;
 *   kind 1  FP32 FMA lane operations with packed f32x2 FMA (two per lane and
 *           instruction) -- the packed form halves the issue slots, not the
 *           FP32 pipe's lane rate;
 *   kind 2  FP32 atomic adds in L2, lanes of a warp on consecutive words;
 *   kind 3  FP32 atomic adds in L2 in the data VJP's pattern (the 2 x 2 taps
 *           of samples ~2.6 px apart).
 * Synchronous (waits for `stream`); uses 64 MiB of context workspace. */
int bp_probe(bp_ctx* ctx, int kind, double* result, void* stream);

/* Bounds checking (debug builds).  A library compiled with -DBP_BOUNDS_CHECK
 * (paper_2401_09283_gb300.build.build_library(variant="bounds")) checks every
 * staged, gathered and scattered index of the backprojection kernels against
 * the range it must lie in; a failed check sets bit `code` of a device flag
 * word (0 staged tap, 1 global tap, 2 scatter, 3 staging destination, 7 self
 * test), records the first failure (*first_failure = code << 56 | a << 28 | b,
 * the two offending coordinates; -1 when none), and redirects the access to
 * a safe position -- nothing traps and nothing outside the buffers is
 * touched.  op: 0 read, 1 read and clear, 2 record a synthetic failure first
 * (tests the reporting path without touching memory).  Synchronises the
 * device's legacy default stream.  Release builds return BP_ERR_UNSUPPORTED.
 * The paper has no counterpart (a debugging aid). */
int bp_bounds_check(bp_ctx* ctx, int op, unsigned int* flags, long long* first_failure);

/* Eq. 1 for every view: Phat[j] = P[j] T(motion[j]) (float64, [V][12]).
 * motion may be NULL (identity; Phat is then P bit for bit). */
int bp_compose(bp_ctx* ctx, int nviews, const double* P, const double* motion, double* Phat,
               void* stream);

/* Eq. 3: vol[k][j][i] = sum_j c_j * omega_j * d_j(u/w, v/w) with
 * (u,v,w) = P_j T(motion_j) (x,y,z,1), bilinear interpolation, zero padding.
 *   proj         projections, layout and dtype per pdesc;
 *   P            float64 [V][12] calibrated matrices;
 *   motion       float64 [V][6] or NULL (identity);
 *   view_weight  float64 [V] (c_j) or NULL (all 1);
 *   weight       bp_weight; FDK uses pdesc->sid;
 *   vol          float32 output, overwritten.
 * Accumulation is FP32 per voxel; coordinates are computed relative to an
 * FP64 anchor per tile of voxels and view.  Deterministic. */
int bp_forward(bp_ctx* ctx, const void* proj, const bp_proj_desc* pdesc, const double* P,
               const double* motion, const double* view_weight, int weight,
               const bp_vol_desc* vdesc, float* vol, void* stream);

/* Vector-Jacobian products of bp_forward for an upstream gradient dL_dvol
 * (float32, volume layout):
 *   dL_dmotion  float64 [V][6]: Eq. 4 per voxel-view, summed per view
 *               (FP32 within a tile, FP64 across tiles, deterministic), then
 *               chained through Eq. 1 (Eq. 2);
 *   dL_dPhat    float64 [V][12]: the per-view sum of Eq. 4 itself, i.e. the
 *               gradient with respect to Phat_j = P_j T(motion_j);
 *   dL_dproj    float32 [V][nv][nu] (contiguous): the adjoint of Eq. 3 in
 *               the data, overwritten (FP32 atomics: not bitwise
 *               deterministic).  The context holds a scratch block image
 *               of 16 bytes per detector pixel of every view for it (4x the
 *               size of dL_dproj; see bp_ctx_workspace_bytes), kept between
 *               calls -- when dL_dproj comes with the motion gradients, only
 *               for projections with 16-byte aligned rows.
 * Any output may be NULL to skip it (dL_dmotion needs motion or treats it as
 * zero).  With BP_WEIGHT_FDK the derivative of (sid/w)^2 is included. */
int bp_vjp(bp_ctx* ctx, const float* dL_dvol, const void* proj, const bp_proj_desc* pdesc,
           const double* P, const double* motion, const double* view_weight, int weight,
           int deriv, const bp_vol_desc* vdesc, double* dL_dmotion, double* dL_dPhat,
           float* dL_dproj, void* stream);

/* Sharpness loss of a volume (stands in for the learned quality metric of
 * Sec. II-B.3): L = -(1/K) sum over the three axes of the squared forward
 * differences of all voxel pairs inside the volume, K = nx*ny*nz.
 *   loss     float64 scalar output (host or device);
 *   dL_dvol  float32 volume output (may be NULL).
 * The FP64 sum is deterministic. */
int bp_sharpness(bp_ctx* ctx, const float* vol, const bp_vol_desc* vdesc, double* loss,
                 float* dL_dvol, void* stream);

/* Smoothed isotropic total variation of a volume, the classical autofocus
 * metric the paper compares against (Sec. IV-A, "TV"):
 *   L = (1/K) sum over voxels x with all three forward neighbours inside of
 *       sqrt(|grad+ I(x)|^2 + eps^2),  grad+ = forward differences, K = nx*ny*nz;
 * loss float64 (host or device), dL_dvol float32 (may be NULL), eps > 0. */
int bp_tv(bp_ctx* ctx, const float* vol, const bp_vol_desc* vdesc, double eps, double* loss,
          float* dL_dvol, void* stream);

/* Allocation-free sharpness loss.  The paper has no counterpart: this is for
 * callers that cannot allocate device memory during the call -- code being
 * recorded into a CUDA graph (an allocation would break the stream capture),
 * hosts that give all device memory to their own pool at start-up, and
 * real-time loops that must not wait on the allocator.  It computes the loss
 * and gradient of bp_sharpness -- the gradient bit for bit, the loss up to
 * the order of its FP64 sums (fixed chunks of 4096 voxels here, a
 * grid-stride loop there) -- needs no context, allocates nothing (no
 * cudaMalloc/cudaFree, no allocating library routine) and keeps its per-chunk
 * FP64 partial sums in a fixed array inside the library: 256 KiB on every GPU
 * that loads the library, held until the process exits.
 *   vol, dL_dvol, loss  device memory of the current device (host pointers
 *                       are rejected with BP_ERR_INVALID_ARG); dL_dvol may
 *                       be NULL;
 *   limit               at most 512^3 = 134217728 voxels; larger volumes
 *                       return BP_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Calls
 * share the array: calls whose kernels may overlap on the GPU (other streams,
 * other host threads) race and give wrong results.  Every call overwrites
 * all partials it reads, so no state carries over.  Asynchronous on
 * `stream`.  Errors are reported by the return code only. */
int bp_sharpness_noalloc(const float* vol, const bp_vol_desc* vdesc, double* loss,
                         float* dL_dvol, void* stream);

/* Optimiser steps on theta float64 [V][6] in place (device or host).
 * Eq. 6: theta -= s0 * t^n * grad.  Adam: standard bias-corrected Adam with
 * iteration counter n >= 1 and moments m1, m2 ([V][6], caller-owned, start
 * at zero).  With gauge != 0 the per-parameter mean over views is removed
 * afterwards (a rigid motion common to all views only moves the volume and
 * is not identifiable by an image-quality loss). */
int bp_gd_step(bp_ctx* ctx, int nviews, double* theta, const double* grad, double s0, double t,
               int n, int gauge, void* stream);
int bp_adam_step(bp_ctx* ctx, int nviews, double* theta, const double* grad, double* m1,
                 double* m2, double lr, double beta1, double beta2, double eps, int n, int gauge,
                 void* stream);

/* Akima spline motion model (Sec. II-B.1): each of the six motion parameters
 * is an Akima spline through n_nodes node values at knots spread evenly over
 * the views (first knot at view 0, last at view nviews-1), and theta[j] is
 * the six splines at view j.  Akima's construction: secants between nodes,
 * two more secants per end by linear extrapolation, node slopes as the
 * |secant difference|-weighted mean of the two neighbouring secants (their
 * plain mean where both weights are 0), cubic Hermite pieces.
 *   nodes       float64 [n_nodes][6] (same parameter order as theta);
 *   theta       float64 [nviews][6] output;
 *   dL_dtheta   float64 [nviews][6]; dL_dnodes float64 [n_nodes][6] output
 *               = (d theta / d nodes)^T dL_dtheta, per parameter.
 * Requires 3 <= n_nodes <= 512 and nviews >= 2 (BP_ERR_INVALID_ARG or
 * BP_ERR_UNSUPPORTED otherwise).  FP64 throughout; arrays host or device.
 * The VJP sums in a fixed order (deterministic). */
int bp_akima_motion(bp_ctx* ctx, int n_nodes, int nviews, const double* nodes, double* theta,
                    void* stream);
int bp_akima_motion_vjp(bp_ctx* ctx, int n_nodes, int nviews, const double* nodes,
                        const double* dL_dtheta, double* dL_dnodes, void* stream);

/* FDK preprocessing of raw line integrals (the filtering of Sec. III; the
 * redundancy weights of a short scan):
 *   out[j][b][a] = tau * sum_k h[a-k] * w_j(k) * c(k,b) * raw[j][b][k],
 *   c(a,b) = SDD / sqrt(SDD^2 + x_a^2 + y_b^2)   cosine weight, x_a, y_b in mm
 *            from the principal point ((nu-1)/2, (nv-1)/2), pixel pitch `pitch`;
 *   h[n]   = -2 / (pi^2 tau^2 (4 n^2 - 1))      Shepp-Logan ramp, tau = pitch*SID/SDD;
 *   w_j(k) = Parker's weight of the ray (view j, column k) for a short scan
 *            of arc `arc` (rad, views spread evenly from the scan start,
 *            delta = (arc - pi)/2 in place of the maximum fan angle), or 1/2
 *            for a full scan (arc >= 2 pi).
 * A direct linear convolution along each row.  ext > 0 is the truncation
 * correction of Sec. IV-D: every weighted row is extended by ext pixels on
 * either side, falling linearly from its edge value to 0 (extension pixel
 * m = 1..ext holds edge * (1 - m/ext)), before the convolution; the paper
 * extends by 10 % of the width.  ext = 0: zero outside the row.
 *   raw, out  float32 [nviews][nv][nu], contiguous, host or device;
 *   limits    nu + 2 ext <= 8192; a short-scan arc must exceed pi + the full
 *             fan angle.
 * The tables are FP64 rounded to FP32; accumulation is FP32. */
int bp_fdk_filter(bp_ctx* ctx, const float* raw, int nviews, int nv, int nu, double pitch,
                  double sid, double sdd, double arc, int ext, float* out, void* stream);

/* ------------------------------------------------------------------ jobs
 * A motion-estimation job (Sec. II-C): everything one scan needs stays on the
 * device -- projections, gradient images, theta, optimiser state, volume and
 * loss history -- and motion_step() replays one captured CUDA graph per
 * iteration: compose (Eq. 1) -> backprojection (Eq. 3) -> sharpness loss ->
 * motion VJP (Eqs. 4-5) -> FP64 reduction and chain (Eq. 2) -> update
 * (Eq. 6 or Adam), followed by the view-mean gauge step. */

typedef enum { BP_OPT_GD = 0 /* Eq. 6 */, BP_OPT_ADAM = 1 } bp_optimizer;
typedef enum { BP_LOSS_SHARPNESS = 0 /* bp_sharpness */, BP_LOSS_TV = 1 /* bp_tv */ } bp_loss;

typedef struct {
  int optimizer;    /* bp_optimizer */
  double lr;        /* Adam step (translations, mm) or Eq. 6 s0 for translations */
  double lr_rot;    /* the same for rotations (rad) */
  double decay;     /* Eq. 6 t (GD only) */
  double beta1, beta2, eps;  /* Adam */
  int gauge;        /* remove the per-parameter view mean after each step */
  int loss;         /* bp_loss: the image-quality target minimised */
  double tv_eps;    /* eps of BP_LOSS_TV */
  int motion_nodes; /* 0: one free theta per view (6V parameters); 3..512: the
                       Akima spline motion model of Sec. II-B.1 (bp_akima_motion)
                       with this many nodes, and the optimiser works on the
                       6 N_n node values (gauge: mean over nodes removed) */
} bp_opt_desc;

typedef struct bp_job bp_job;

/* Create a job: copies proj (any location; stored compactly in its dtype), P,
 * view_weight and theta0 (NULL = zero motion; [V][6] per-view values, or
 * [N_n][6] node values when opt->motion_nodes > 0) to job-owned device memory and
 * precomputes the gradient images (CENTRAL).  max_iters bounds the loss
 * history.  Admission: if the job's device bytes (bp_job_bytes) would take
 * the context's live jobs beyond its HBM budget (bp_ctx_set_hbm_budget, or the
 * device's free memory when 0) it fails with BP_ERR_OOM and allocates
 * nothing. */
int bp_job_create(bp_ctx* ctx, const void* proj, const bp_proj_desc* pdesc, const double* P,
                  const double* view_weight, int weight, int deriv, const bp_vol_desc* vdesc,
                  const bp_opt_desc* opt, const double* theta0, int max_iters, bp_job** out);
/* Device bytes a job with these sizes would hold (no allocation). */
long long bp_job_bytes_for(const bp_proj_desc* pdesc, const bp_vol_desc* vdesc, int deriv,
                           int max_iters);
long long bp_job_bytes(const bp_job* job);
int bp_ctx_set_hbm_budget(bp_ctx* ctx, long long bytes);
/* Run n_iters iterations on `stream` (asynchronous; the replays wait for
 * the job's earlier work).  The first call captures the iteration graph on a
 * job-owned stream.  Jobs on different streams overlap on the device. */
int motion_step(bp_job* job, int n_iters, void* stream);
/* Wait for the job's queued iterations (not for other work on the device)
 * and copy theta (float64 [V][6]; with the spline model, the splines of the
 * current nodes at every view) and the loss history (float64
 * [max_iters], may be NULL) to host memory; *iters_done (may be NULL)
 * receives the number of iterations run. */
int bp_job_get_motion(const bp_job* job, double* theta_host, double* loss_history,
                      int* iters_done);
/* Copy the current spline node values (float64 [N_n][6]) of a job with the
 * Akima motion model to host memory (BP_ERR_INVALID_ARG for per-view jobs). */
int bp_job_get_nodes(const bp_job* job, double* nodes_host);
/* The job's current volume (float32, device pointer owned by the job). */
const float* bp_job_volume(const bp_job* job);
/* Waits for the job's queued iterations, then frees its memory with the
 * stream-ordered allocator (no device-wide synchronisation). */
void bp_job_destroy(bp_job* job);

/* Cancel a job: later motion_step calls return BP_ERR_CANCELLED and a batch
 * drops it at its next step; iterations already queued still run, and the
 * job's state stays readable (bp_job_get_motion) until bp_job_destroy.  The
 * paper has no counterpart (serving control). */
int bp_job_cancel(bp_job* job);
/* Wait for the job's queued iterations for at most timeout_ms milliseconds
 * (< 0: no limit), polling an event from the host; BP_ERR_TIMEOUT if they
 * are still running then (nothing is stopped; wait again or cancel).  The
 * paper has no counterpart (serving control). */
int bp_job_wait(const bp_job* job, double timeout_ms);
/* Iterations queued for the job so far (motion_step or batches), or -1. */
int bp_job_iterations_queued(const bp_job* job);

/* ---------------------------------------------------------------- batches
 * Several resident jobs advanced together (the serving form): compose
 * (Eq. 1), backprojection (Eq. 3), loss, FP64 reduction and chain (Eq. 2)
 * and update are each ONE launch whose blocks walk the work items (views,
 * tiles, loss chunks) of every member -- the backprojection a persistent
 * kernel -- so jobs of different volume and view counts share each kernel
 * and fill the GPU together; the motion VJP (Eqs. 4-5) runs each member's
 * own VJP kernel on a parallel branch of the same graph, so the members'
 * VJPs overlap.  The member table is a kernel parameter; each member set
 * gets one captured CUDA graph of the iteration (made at the first step
 * after the set changes; the graph of an earlier set is freed once its
 * queued replays have run).  Every item runs the per-job arithmetic: a
 * member's iterations are bit for bit those of motion_step.
 * Members must share dtype, weight, derivative mode, loss and optimiser,
 * use per-view motion (motion_nodes = 0) and have detector rows of a
 * multiple of 16 bytes; a job is a member of at most one batch and is not
 * advanced by motion_step while it is one.  The paper has no counterpart. */
typedef struct bp_batch bp_batch;
/* max_jobs: 1..32 members. */
int bp_batch_create(bp_ctx* ctx, int max_jobs, bp_batch** out);
/* Replace the member set (n_jobs = 0 empties it); takes effect at the next
 * step.  BP_ERR_INVALID_ARG / BP_ERR_UNSUPPORTED / BP_ERR_CANCELLED for a
 * member that breaks the rules above; the set is then unchanged. */
int bp_batch_set_jobs(bp_batch* batch, bp_job* const* jobs, int n_jobs);
/* Queue n_iters iterations of every member on `stream` (asynchronous; waits
 * for the members' earlier work; cancelled members are dropped first). */
int bp_batch_step(bp_batch* batch, int n_iters, void* stream);
/* Number of members, or -1. */
int bp_batch_size(const bp_batch* batch);
/* Waits for the batch's queued steps, then frees it (the jobs stay). */
void bp_batch_destroy(bp_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* BP_GB300_H */
