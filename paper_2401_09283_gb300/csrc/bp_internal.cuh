// Internal declarations of the bp_gb300 library (CUDA, sm_103a).
//
// Frames used by the kernels (all derived from the caller's inputs in FP64):
//   index frame  voxel coordinates relative to the volume centre,
//                q = (i - cx, j - cy, k - cz), c = (n-1)/2 per axis;
//   P'           = Phat * A, where A maps the index frame to world mm, so
//                (u, v, w) = P' (q, 1) with (u/w, v/w) in absolute pixels;
//   anchored     per (tile of voxels, view) the integer pixel (au, av)
//                nearest the tile centre's projection is subtracted:
//                rows R_u = P'_0 - au P'_2, R_v = P'_1 - av P'_2, R_w = P'_2,
//                and the tile centre qc is factored out, q = qc + dq.
//                The FP32 inner loops see only small numbers (|u/w| of a
//                few tens of pixels, |dq| of a few voxels), so detector
//                positions keep ~1e-6 px precision up to 1240-px detectors.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bpk {

// Volume-major tiling: a CTA owns TX x TY voxel columns of ZB voxels each.
constexpr int TX = 16;
constexpr int TY = 16;
constexpr int NT = TX * TY;   // threads per CTA
constexpr int VB = 32;        // views per FP64 set-up batch
constexpr int PSLOTS = 16;    // floats per (tile, view) partial record

// z-extent of the VJP tiles (the tiling of the per-tile partial records)
#ifndef BP_ZB_VJP
#define BP_ZB_VJP 16
#endif
constexpr int ZB_VJP = BP_ZB_VJP;

// Per view, written by compose_kernel.
struct ViewGeom {
  double P[12];   // P' = P T(theta) A   (index frame -> absolute pixels)
  double wgt;     // c_j * (FDK ? sid^2 : 1)
  double scale;   // per-view dequantisation scale (1 for float32 data)
};

// Per (tile, view), in shared memory.
struct TileView {
  float U0, V0, W0;   // anchored homogeneous coordinates at the tile centre
  float ru[3];        // d(u_rel)/d(dq)
  float rv[3];
  float rw[3];
  int au, av;         // anchor pixel
  float wgt;          // wgt * scale (FP32): weight of a stored sample
  float wgtd;         // wgt alone: weight of a dequantised sample (data VJP)
  int mode;           // MODE_*
  int fu0, fv0;       // detector footprint of the tile (first pixel), clipped
  int fw, fh;         // footprint size in pixels (0 when unbounded)
  int csafe;          // every tap pixel and its central-difference neighbours
                      // (one more pixel each side) lie inside the detector
  // Staged footprint in shared memory (staged != 0): detector rows
  // [sv0, sv0 + sh) and 16-byte chunks [sx0, sx0 + scpr * CH) at a fixed row
  // pitch, zero where they lie off the detector.  soff turns the
  // magic-number floor bits (bx, by) of a sample into its element index
  // by * pitch + bx + soff (mod 2^32); srpp rows are copied per warp pass and
  // smag = ceil(2^16 / scpr) divides a lane index by scpr.
  int sx0, sv0, sh, scpr, srpp, smag, soff, staged;
};

enum { MODE_SKIP = 0, MODE_INTERIOR = 1, MODE_EDGE = 2 };

struct VolInfo {
  int nx, ny, nz;
  int tiles_x, tiles_y, tiles_z;
  int zb;
  double cx, cy, cz;  // (n-1)/2
  double A[12];       // index frame -> world (3x4, last row implicit 0 0 0 1)
};

struct ProjInfo {
  int nu, nv, nviews;
  long long rs, vs;   // element strides
};

// ------------------------------------------------------------ launchers
// All launchers are asynchronous on `stream` and return cudaGetLastError().

cudaError_t launch_compose(const double* P, const double* theta, const double* view_weight,
                           const float* view_scale, int V, int fdk, double sid,
                           const VolInfo& vi, ViewGeom* geom, double* Phat, cudaStream_t s);

cudaError_t launch_forward(const void* proj, int dtype, const ProjInfo& pi, const ViewGeom* geom,
                           const VolInfo& vi, int fdk, float* vol, cudaStream_t s);
// Set the forward / motion-VJP kernels' shared-memory attributes on the
// current device (done by the first launch anyway; call before capturing a
// graph).
cudaError_t prepare_forward(int dtype, int fdk);
cudaError_t prepare_vjp(int dtype, int fdk, int exact);

cudaError_t launch_grad_images(const void* proj, int dtype, const ProjInfo& pi, float2* grad,
                               cudaStream_t s);

// dproj != NULL fuses the data VJP (same samples, contiguous [V][nv][nu]
// output zeroed by the caller) into the motion-VJP kernel.  blk (NULL or
// block_image_floats(pi) floats of scratch) is the block image of the staged
// CENTRAL scatter (per pixel, the 2x2 block it starts, 16 bytes); when
// vjp_uses_blocks() the launch zeroes it, runs the VJP and then a second
// kernel that adds it into dproj.
cudaError_t launch_vjp_motion(const float* dvol, const void* proj, int dtype, const ProjInfo& pi,
                              const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                              int fdk, int exact, float* partials, float* dproj, float* blk,
                              cudaStream_t s);
long long block_image_floats(const ProjInfo& pi);
bool vjp_uses_blocks(const void* proj, int dtype, const ProjInfo& pi, int exact);

cudaError_t launch_reduce_chain(const float* partials, int ntiles, const VolInfo& vi,
                                const double* P, const double* theta, int V, double* dL_dPhat,
                                double* dL_dtheta, cudaStream_t s);

// Data VJP alone; blk (NULL or block_image_floats(pi) floats) as above.
cudaError_t launch_vjp_proj(const float* dvol, const ProjInfo& pi, const ViewGeom* geom,
                            const VolInfo& vi, int fdk, float* dproj, float* blk, cudaStream_t s);

cudaError_t launch_sharpness(const float* vol, int nx, int ny, int nz, double* block_sums,
                             int max_blocks, double* loss, float* grad, cudaStream_t s);

cudaError_t launch_gd(int V, double* theta, const double* grad, double s0, double t, int n,
                      int gauge, cudaStream_t s);

cudaError_t launch_adam(int V, double* theta, const double* grad, double* m1, double* m2,
                        double lr, double b1, double b2, double eps, int n, int gauge,
                        cudaStream_t s);

int sharpness_blocks(long long nvox);

// Smoothed isotropic total variation and its gradient; iter == NULL writes
// *loss, otherwise loss[*iter] (a history, graph-replayable).
cudaError_t launch_tv(const float* vol, int nx, int ny, int nz, float eps, double* block_sums,
                      int max_blocks, double* loss, const int* iter, int hist_len, float* grad,
                      cudaStream_t s);

// Graph-replayable variants: the iteration number lives on the device.
cudaError_t launch_sharpness_hist(const float* vol, int nx, int ny, int nz, double* block_sums,
                                  int max_blocks, double* history, const int* iter, int hist_len,
                                  float* grad, cudaStream_t s);
cudaError_t launch_adam_dev(int V, double* theta, const double* grad, double* m1, double* m2,
                            double lr_t, double lr_r, double b1, double b2, double eps, int* iter,
                            int gauge, cudaStream_t s);
cudaError_t launch_gd_dev(int V, double* theta, const double* grad, double s0_t, double s0_r,
                          double t, int* iter, int gauge, cudaStream_t s);

// Akima spline motion model (bp_spline.cu): nodes [n][6] -> theta [V][6]
// and its VJP; n >= 3, V >= 2, n <= AKIMA_MAX_NODES.
constexpr int AKIMA_MAX_NODES = 512;  // VJP shared memory: 8 (8n + 2) bytes
cudaError_t launch_akima_eval(int n, int V, const double* nodes, double* theta, cudaStream_t s);
cudaError_t launch_akima_vjp(int n, int V, const double* nodes, const double* g, double* dnodes,
                             cudaStream_t s);

// FDK preprocessing (bp_fdk.cu): cosine and redundancy weights, optional
// truncation extension by `ext` pixels per side, Shepp-Logan ramp along rows.
// `tab` holds fdk_table_floats(V, nu, ext) floats of workspace; nu + 2 ext <=
// FDK_MAX_NU (shared memory of the convolution: fdk_smem_bytes(nu, ext)).
constexpr int FDK_MAX_NU = 8192;
size_t fdk_table_floats(int V, int nu, int ext);
size_t fdk_smem_bytes(int nu, int ext);
cudaError_t launch_fdk_filter(const float* raw, int V, int nv, int nu, int ext, double pitch,
                              double sid, double sdd, double arc, float* tab, float* out,
                              cudaStream_t s);

// ---------------------------------------------------------------- batches
// Several motion-estimation jobs advanced together: each stage of an
// iteration is one launch over the work items of every member job (views,
// tiles, (tile, view chunk) pairs, loss chunks).  The member table is a
// __grid_constant__ kernel parameter: the kernels read each job's sizes and
// pointers from read-only parameter space, as the per-job kernels read their
// arguments (from a table in shared or global memory the compiler must
// assume aliased, the VJP ran 26 % more instructions).  Members share dtype,
// weight, derivative mode, loss and optimiser (template or launch-uniform
// parameters).  At most BATCH_MAX_JOBS members (the table fits the 32 KB of
// kernel parameters).
constexpr int BATCH_MAX_JOBS = 32;

struct BatchJob {
  const void* proj;        // [V][nv][nu] compact, the batch's dtype
  const float2* grad;      // CENTRAL gradient images (NULL with BILINEAR_EXACT)
  const double* P;         // [V][12]
  const double* vw;        // [V] or NULL
  const float* scale;      // [V] or NULL
  double* theta;           // [V][6]
  double* gth;             // [V][6]
  double *m1, *m2;         // Adam moments
  ViewGeom* geom;
  float *vol, *dvol, *partials;
  double *blk, *hist;      // loss block sums, loss history
  int* iter;               // iterations done (device counter)
  ProjInfo pi;
  VolInfo vi;              // VJP tiling (zb = ZB_VJP)
  VolInfo vif;             // forward tiling
  double sid;
  double lr_t, lr_r, beta1, beta2, eps, decay;
  float tv_eps;
  int V, ntiles_f, ntiles_v, nblk, max_iters, gauge;
};

struct BatchTable {
  int njobs;
  int off_view[BATCH_MAX_JOBS + 1];  // prefix sums of V (compose, reduction)
  int off_fwd[BATCH_MAX_JOBS + 1];   // of forward tiles
  int off_loss[BATCH_MAX_JOBS + 1];  // of loss blocks
  BatchJob job[BATCH_MAX_JOBS];
};
static_assert(sizeof(BatchTable) <= 30000, "the member table must fit the kernel parameters");

// Index of the job whose range [off[j], off[j+1]) holds work item w.
// (i, j, k) of linear voxel index x in an [nz][ny][nx] volume: 32-bit
// division when the volume has fewer than 2^32 voxels (the 64-bit one costs
// several times more instructions).
__device__ __forceinline__ void voxel_ijk(long long x, int nx, int ny, long long nvox, int& i,
                                          int& j, int& k) {
  if (nvox <= 0xffffffffLL) {
    const unsigned ux = (unsigned)x, q = ux / (unsigned)nx;
    i = (int)(ux - q * (unsigned)nx);
    j = (int)(q % (unsigned)ny);
    k = (int)(q / (unsigned)ny);
  } else {
    const long long q = x / nx;
    i = (int)(x - q * nx);
    j = (int)(q % ny);
    k = (int)(q / ny);
  }
}

__host__ __device__ inline int batch_find(const int* off, int n, int w) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Forward tiling and VJP view chunk of a job (host side, for the table).
int forward_zb();

// Streams and events for running the members' VJP kernels as parallel
// branches of a stream capture: fork from the capturing stream, one stream
// per member, join back.
struct BatchBranches {
  int n = 0;  // streams and join events available
  cudaStream_t* streams = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t* joins = nullptr;
};

// One iteration of every member: compose -> forward -> loss -> VJP ->
// reduction and chain -> update.  Every stage but the VJP is one launch over
// the table's work items: the forward persistent (SMs x 4 CTAs taking tiles
// from *counter, which the compose launch resets), the small stages
// grid-stride loops.  The VJP runs each member's own VJP kernel on its own
// branch, so the members' kernels overlap: br must hold a stream and a join
// event per member (cudaErrorInvalidValue otherwise).
// loss: 0 sharpness, 1 TV; opt: 0 Eq. 6 step, 1 Adam.
cudaError_t prepare_batch(int dtype, int fdk, int exact);
cudaError_t launch_batch_iteration(const BatchTable& tab, unsigned* counter, int dtype, int fdk,
                                   int exact, int loss, int opt, int sms, cudaStream_t s,
                                   const BatchBranches* br);
cudaError_t launch_batch_forward(const BatchTable& tab, unsigned* counter, int dtype, int fdk,
                                 int sms, cudaStream_t s);
constexpr int BATCH_KERNELS = 6;  // launches per batched iteration besides the VJP

// Bounds-check word of debug builds (-DBP_BOUNDS_CHECK): op 0 reads the flag
// bits and the first failure, 1 reads and clears them, 2 records a synthetic
// failure first (self test of the reporting path).  cudaErrorNotSupported in
// release builds.
cudaError_t bounds_status(unsigned* flags, long long* first, int op, cudaStream_t s);

// Throughput probes (bp_probe.cu): kind 0 scalar FP32 FMA lane-ops/s, 1 packed
// f32x2 FMA lane-ops/s, 2 coalesced FP32 L2 atomic adds/s, 3 atomic adds/s in
// the data VJP's scattered 2 x 2 pattern.  scratch: scratch_words floats.
cudaError_t run_probe(int kind, float* scratch, long long scratch_words, int sms, double* result,
                      cudaStream_t s);

}  // namespace bpk
