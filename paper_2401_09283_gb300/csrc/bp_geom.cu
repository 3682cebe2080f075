// FP64 per-view kernels (motion composition of Eq. 1, the cross-tile
// reduction and chain rule of Eq. 2), the sharpness loss and the optimiser
// updates (Eq. 6 and Adam).  None of these is on the voxel-view hot loop;
// all are deterministic (fixed summation order, no atomics).
#include "bp_internal.cuh"

namespace bpk {

// ---------------------------------------------------------------- rigid motion

// R = Rz(rz) Ry(ry) Rx(rx) (row-major 3x3), or its derivative with respect
// to one angle when dax = 0, 1, 2 (x, y, z).
__device__ static void rot_zyx(const double* th, int dax, double R[9]) {
  double sx, cx, sy, cy, sz, cz;
  sincos(th[3], &sx, &cx);
  sincos(th[4], &sy, &cy);
  sincos(th[5], &sz, &cz);
  double X[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  double Y[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  double Z[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  if (dax == 0) {
    double D[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
    for (int e = 0; e < 9; ++e) X[e] = D[e];
  } else if (dax == 1) {
    double D[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
    for (int e = 0; e < 9; ++e) Y[e] = D[e];
  } else if (dax == 2) {
    double D[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
    for (int e = 0; e < 9; ++e) Z[e] = D[e];
  }
  double ZY[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      ZY[3 * r + c] = Z[3 * r] * Y[c] + Z[3 * r + 1] * Y[3 + c] + Z[3 * r + 2] * Y[6 + c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = ZY[3 * r] * X[c] + ZY[3 * r + 1] * X[3 + c] + ZY[3 * r + 2] * X[6 + c];
}

// M (3x4) = P (3x4) * [[R t],[0 1]] (rigid 4x4 given by R and t).
__device__ static void p_times_rigid(const double* P, const double R[9], const double t[3],
                                     double tw, double* M) {
  for (int r = 0; r < 3; ++r) {
    const double* p = P + 4 * r;
    for (int c = 0; c < 3; ++c) M[4 * r + c] = p[0] * R[c] + p[1] * R[3 + c] + p[2] * R[6 + c];
    M[4 * r + 3] = p[0] * t[0] + p[1] * t[1] + p[2] * t[2] + p[3] * tw;
  }
}

// View j: Phat = P T(theta) (Eq. 1), then P' = Phat A.
__device__ static void compose_view(const double* __restrict__ P, const double* __restrict__ theta,
                                    const double* __restrict__ vw, const float* __restrict__ vscale,
                                    int fdk, double sid, const VolInfo& vi,
                                    ViewGeom* __restrict__ geom, double* __restrict__ Phat, int j) {
  double Ph[12];
  if (theta) {
    double R[9];
    rot_zyx(theta + 6 * j, -1, R);
    p_times_rigid(P + 12 * j, R, theta + 6 * j, 1.0, Ph);
  } else {
    for (int e = 0; e < 12; ++e) Ph[e] = P[12 * j + e];
  }
  if (Phat)
    for (int e = 0; e < 12; ++e) Phat[12 * j + e] = Ph[e];
  if (!geom) return;
  ViewGeom g;
  for (int r = 0; r < 3; ++r) {
    const double* p = Ph + 4 * r;
    // A = [[sx 0 0 tx],[0 sy 0 ty],[0 0 sz tz],[0 0 0 1]]
    g.P[4 * r + 0] = p[0] * vi.A[0];
    g.P[4 * r + 1] = p[1] * vi.A[5];
    g.P[4 * r + 2] = p[2] * vi.A[10];
    g.P[4 * r + 3] = p[0] * vi.A[3] + p[1] * vi.A[7] + p[2] * vi.A[11] + p[3];
  }
  double c = vw ? vw[j] : 1.0;
  g.wgt = fdk ? c * sid * sid : c;
  g.scale = vscale ? (double)vscale[j] : 1.0;
  geom[j] = g;
}

// One thread per view.
__global__ void compose_kernel(const double* __restrict__ P, const double* __restrict__ theta,
                               const double* __restrict__ vw, const float* __restrict__ vscale,
                               int V, int fdk, double sid, VolInfo vi, ViewGeom* __restrict__ geom,
                               double* __restrict__ Phat) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= V) return;
  compose_view(P, theta, vw, vscale, fdk, sid, vi, geom, Phat, j);
}

cudaError_t launch_compose(const double* P, const double* theta, const double* view_weight,
                           const float* view_scale, int V, int fdk, double sid,
                           const VolInfo& vi, ViewGeom* geom, double* Phat, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  compose_kernel<<<(V + 127) / 128, 128, 0, s>>>(P, theta, view_weight, view_scale, V, fdk, sid,
                                                  vi, geom, Phat);
  return cudaGetLastError();
}

// ------------------------------------------------- cross-tile reduction + chain

// Block j: dL/dP' for view j as the FP64 sum over tiles of the tile records
// (each record is in its tile's anchored, centred frame and is mapped back to
// the index frame first), then dL/dPhat = dL/dP' A^T and
// dL/dtheta_m = < dL/dPhat , P dT/dtheta_m > (Eq. 2 through Eq. 1).
// All 256 threads of the block call it for view j.
__device__ static void reduce_chain_view(const float* __restrict__ partials, int ntiles,
                                         const VolInfo& vi, const double* __restrict__ P,
                                         const double* __restrict__ theta,
                                         double* __restrict__ dPhat, double* __restrict__ dth,
                                         int j) {
  __shared__ double red[12][256];
  const int tid = threadIdx.x;
  double acc[12];
  for (int e = 0; e < 12; ++e) acc[e] = 0.0;
  for (int c = tid; c < ntiles; c += blockDim.x) {
    const float* rec = partials + ((size_t)j * ntiles + c) * PSLOTS;
    int tx = c % vi.tiles_x;
    int ty = (c / vi.tiles_x) % vi.tiles_y;
    int tz = c / (vi.tiles_x * vi.tiles_y);
    double qc[3] = {tx * TX + 0.5 * (TX - 1) - vi.cx, ty * TY + 0.5 * (TY - 1) - vi.cy,
                    tz * vi.zb + 0.5 * (vi.zb - 1) - vi.cz};
    double G[12];
    for (int r = 0; r < 3; ++r) {
      double s = rec[4 * r + 3];
      for (int k = 0; k < 3; ++k) G[4 * r + k] = (double)rec[4 * r + k] + s * qc[k];
      G[4 * r + 3] = s;
    }
    double au = rec[12], av = rec[13];
    for (int k = 0; k < 4; ++k) G[8 + k] -= au * G[k] + av * G[4 + k];
    for (int e = 0; e < 12; ++e) acc[e] += G[e];
  }
  for (int e = 0; e < 12; ++e) red[e][tid] = acc[e];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int e = 0; e < 12; ++e) red[e][tid] += red[e][tid + w];
    __syncthreads();
  }
  if (tid != 0) return;
  double Gp[12], Gh[12];
  for (int e = 0; e < 12; ++e) Gp[e] = red[e][0];
  const double sxyz[3] = {vi.A[0], vi.A[5], vi.A[10]};
  const double txyz[3] = {vi.A[3], vi.A[7], vi.A[11]};
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) Gh[4 * r + c] = Gp[4 * r + c] * sxyz[c] + Gp[4 * r + 3] * txyz[c];
    Gh[4 * r + 3] = Gp[4 * r + 3];
  }
  if (dPhat)
    for (int e = 0; e < 12; ++e) dPhat[12 * j + e] = Gh[e];
  if (!dth) return;
  const double zero6[6] = {0, 0, 0, 0, 0, 0};
  const double* th = theta ? theta + 6 * j : zero6;
  const double* Pj = P + 12 * j;
  for (int m = 0; m < 6; ++m) {
    double J[12];
    if (m < 3) {
      // dT/dt_m: zero rotation block, unit vector in the translation column
      const double Rz0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      double t[3] = {0, 0, 0};
      t[m] = 1.0;
      p_times_rigid(Pj, Rz0, t, 0.0, J);
    } else {
      double dR[9];
      const double t0[3] = {0, 0, 0};
      rot_zyx(th, m - 3, dR);
      p_times_rigid(Pj, dR, t0, 0.0, J);
    }
    double s = 0.0;
    for (int e = 0; e < 12; ++e) s += Gh[e] * J[e];
    dth[6 * j + m] = s;
  }
}

__global__ void reduce_chain_kernel(const float* __restrict__ partials, int ntiles, VolInfo vi,
                                    const double* __restrict__ P, const double* __restrict__ theta,
                                    int V, double* __restrict__ dPhat, double* __restrict__ dth) {
  reduce_chain_view(partials, ntiles, vi, P, theta, dPhat, dth, blockIdx.x);
}

cudaError_t launch_reduce_chain(const float* partials, int ntiles, const VolInfo& vi,
                                const double* P, const double* theta, int V, double* dL_dPhat,
                                double* dL_dtheta, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  reduce_chain_kernel<<<V, 256, 0, s>>>(partials, ntiles, vi, P, theta, V, dL_dPhat, dL_dtheta);
  return cudaGetLastError();
}

// --------------------------------------------------------------- sharpness loss

constexpr int SH_THREADS = 256;

int sharpness_blocks(long long nvox) {
  long long b = (nvox + SH_THREADS - 1) / SH_THREADS;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

// L = -(1/K) sum_pairs (I[y]-I[x])^2 over forward neighbours y = x + e_a
// inside the volume; dL/dI[x] = (2/K) sum over the valid neighbours n of x
// (I[n] - I[x]).  Per-block FP64 partial sums in a fixed order.
// Block b of nb (grid-stride partition of the voxels over nb blocks of
// SH_THREADS threads); all threads of the block call it.
__device__ static void sharpness_block(const float* __restrict__ vol, int nx, int ny, int nz,
                                       double* __restrict__ block_sums, float* __restrict__ grad,
                                       int b, int nb) {
  __shared__ double red[SH_THREADS];
  const long long nvox = (long long)nx * ny * nz;
  const double K = (double)nvox;
  const float g2 = (float)(2.0 / K);
  double acc = 0.0;
  const long long nxy = (long long)nx * ny;
  for (long long x = b * (long long)SH_THREADS + threadIdx.x; x < nvox;
       x += (long long)nb * SH_THREADS) {
    int i, j, k;
    voxel_ijk(x, nx, ny, nvox, i, j, k);
    float c = vol[x];
    float gsum = 0.0f;
    // the voxel's squared forward differences summed in FP32 (x, y, z order),
    // accumulated in FP64: one FP64 add per voxel (FP64 is slow on GB300)
    float q = 0.0f;
    if (i + 1 < nx) {
      float d = vol[x + 1] - c;
      q = d * d;
      gsum += d;
    }
    if (j + 1 < ny) {
      float d = vol[x + nx] - c;
      q = fmaf(d, d, q);
      gsum += d;
    }
    if (k + 1 < nz) {
      float d = vol[x + nxy] - c;
      q = fmaf(d, d, q);
      gsum += d;
    }
    acc += (double)q;
    if (grad) {
      if (i > 0) gsum += vol[x - 1] - c;
      if (j > 0) gsum += vol[x - nx] - c;
      if (k > 0) gsum += vol[x - nxy] - c;
      grad[x] = g2 * gsum;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SH_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[b] = red[0];
}

__global__ void sharpness_kernel(const float* __restrict__ vol, int nx, int ny, int nz,
                                 double* __restrict__ block_sums, float* __restrict__ grad) {
  sharpness_block(vol, nx, ny, nz, block_sums, grad, blockIdx.x, gridDim.x);
}

__global__ void sharpness_finish_kernel(const double* __restrict__ block_sums, int nb, double K,
                                        double* __restrict__ loss) {
  __shared__ double red[SH_THREADS];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += block_sums[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SH_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = -red[0] / K;
}

cudaError_t launch_sharpness(const float* vol, int nx, int ny, int nz, double* block_sums,
                             int max_blocks, double* loss, float* grad, cudaStream_t s) {
  long long nvox = (long long)nx * ny * nz;
  int nb = sharpness_blocks(nvox);
  if (nb > max_blocks) nb = max_blocks;
  sharpness_kernel<<<nb, SH_THREADS, 0, s>>>(vol, nx, ny, nz, block_sums, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sharpness_finish_kernel<<<1, SH_THREADS, 0, s>>>(block_sums, nb, (double)nvox, loss);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ optimisers

// Subtract the per-parameter mean over views (fixed-order sums).
__device__ static void remove_mean(int V, double* theta) {
  __shared__ double red[256];
  __shared__ double mean;
  for (int m = 0; m < 6; ++m) {
    double acc = 0.0;
    for (int j = threadIdx.x; j < V; j += blockDim.x) acc += theta[6 * j + m];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) mean = red[0] / V;
    __syncthreads();
    for (int j = threadIdx.x; j < V; j += blockDim.x) theta[6 * j + m] -= mean;
    __syncthreads();
  }
}

__global__ void gd_kernel(int V, double* theta, const double* grad, double step, int gauge) {
  for (int e = threadIdx.x; e < 6 * V; e += blockDim.x) theta[e] -= step * grad[e];
  __syncthreads();
  if (gauge) remove_mean(V, theta);
}

__global__ void adam_kernel(int V, double* theta, const double* grad, double* m1, double* m2,
                            double lr, double b1, double b2, double eps, double c1, double c2,
                            int gauge) {
  for (int e = threadIdx.x; e < 6 * V; e += blockDim.x) {
    double g = grad[e];
    double a = b1 * m1[e] + (1.0 - b1) * g;
    double b = b2 * m2[e] + (1.0 - b2) * g * g;
    m1[e] = a;
    m2[e] = b;
    theta[e] -= lr * (a / c1) / (sqrt(b / c2) + eps);
  }
  __syncthreads();
  if (gauge) remove_mean(V, theta);
}

cudaError_t launch_gd(int V, double* theta, const double* grad, double s0, double t, int n,
                      int gauge, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  gd_kernel<<<1, 256, 0, s>>>(V, theta, grad, s0 * pow(t, (double)n), gauge);
  return cudaGetLastError();
}

cudaError_t launch_adam(int V, double* theta, const double* grad, double* m1, double* m2,
                        double lr, double b1, double b2, double eps, int n, int gauge,
                        cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  double c1 = 1.0 - pow(b1, (double)n), c2 = 1.0 - pow(b2, (double)n);
  adam_kernel<<<1, 256, 0, s>>>(V, theta, grad, m1, m2, lr, b1, b2, eps, c1, c2, gauge);
  return cudaGetLastError();
}

// ------------------------------------------- graph-replayable (device counter)

// The job loop replays one captured CUDA graph per iteration, so iteration
// numbers live on the device: the loss goes to history[*iter], the update
// reads *iter and advances it.

// Fixed-order sum of nb block sums -> -sum/K at history[*iter] (TV: +sum/K,
// sign = +1).  All SH_THREADS threads of the block call it.
__device__ static void loss_finish_hist(const double* __restrict__ block_sums, int nb, double K,
                                        double sign, double* __restrict__ history,
                                        const int* __restrict__ iter, int hist_len) {
  __shared__ double red[SH_THREADS];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += block_sums[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SH_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int it = *iter;
    if (it >= 0 && it < hist_len) history[it] = sign * red[0] / K;
  }
}

__global__ void sharpness_finish_hist_kernel(const double* __restrict__ block_sums, int nb,
                                             double K, double* __restrict__ history,
                                             const int* __restrict__ iter, int hist_len) {
  loss_finish_hist(block_sums, nb, K, -1.0, history, iter, hist_len);
}

cudaError_t launch_sharpness_hist(const float* vol, int nx, int ny, int nz, double* block_sums,
                                  int max_blocks, double* history, const int* iter, int hist_len,
                                  float* grad, cudaStream_t s) {
  long long nvox = (long long)nx * ny * nz;
  int nb = sharpness_blocks(nvox);
  if (nb > max_blocks) nb = max_blocks;
  sharpness_kernel<<<nb, SH_THREADS, 0, s>>>(vol, nx, ny, nz, block_sums, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sharpness_finish_hist_kernel<<<1, SH_THREADS, 0, s>>>(block_sums, nb, (double)nvox, history, iter,
                                                         hist_len);
  return cudaGetLastError();
}

// Adam with separate step sizes for translations (mm) and rotations (rad);
// n = *iter + 1.
__device__ static void adam_dev_body(int V, double* theta, const double* grad, double* m1,
                                     double* m2, double lr_t, double lr_r, double b1, double b2,
                                     double eps, int* iter, int gauge) {
  const int n = *iter + 1;
  const double c1 = 1.0 - pow(b1, (double)n), c2 = 1.0 - pow(b2, (double)n);
  for (int e = threadIdx.x; e < 6 * V; e += blockDim.x) {
    const double g = grad[e];
    const double a = b1 * m1[e] + (1.0 - b1) * g;
    const double b = b2 * m2[e] + (1.0 - b2) * g * g;
    m1[e] = a;
    m2[e] = b;
    const double lr = (e % 6) < 3 ? lr_t : lr_r;
    theta[e] -= lr * (a / c1) / (sqrt(b / c2) + eps);
  }
  __syncthreads();
  if (gauge) remove_mean(V, theta);
  if (threadIdx.x == 0) *iter = n;
}

__global__ void adam_dev_kernel(int V, double* theta, const double* grad, double* m1, double* m2,
                                double lr_t, double lr_r, double b1, double b2, double eps,
                                int* iter, int gauge) {
  adam_dev_body(V, theta, grad, m1, m2, lr_t, lr_r, b1, b2, eps, iter, gauge);
}

// Eq. 6 with step s0 * t^n (n = *iter, starting at 0), separate s0 for
// translations and rotations.
__device__ static void gd_dev_body(int V, double* theta, const double* grad, double s0_t,
                                   double s0_r, double t, int* iter, int gauge) {
  const int n = *iter;
  const double f = pow(t, (double)n);
  for (int e = threadIdx.x; e < 6 * V; e += blockDim.x)
    theta[e] -= ((e % 6) < 3 ? s0_t : s0_r) * f * grad[e];
  __syncthreads();
  if (gauge) remove_mean(V, theta);
  if (threadIdx.x == 0) *iter = n + 1;
}

__global__ void gd_dev_kernel(int V, double* theta, const double* grad, double s0_t, double s0_r,
                              double t, int* iter, int gauge) {
  gd_dev_body(V, theta, grad, s0_t, s0_r, t, iter, gauge);
}

cudaError_t launch_adam_dev(int V, double* theta, const double* grad, double* m1, double* m2,
                            double lr_t, double lr_r, double b1, double b2, double eps, int* iter,
                            int gauge, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  adam_dev_kernel<<<1, 256, 0, s>>>(V, theta, grad, m1, m2, lr_t, lr_r, b1, b2, eps, iter, gauge);
  return cudaGetLastError();
}

cudaError_t launch_gd_dev(int V, double* theta, const double* grad, double s0_t, double s0_r,
                          double t, int* iter, int gauge, cudaStream_t s) {
  if (V <= 0) return cudaSuccess;
  gd_dev_kernel<<<1, 256, 0, s>>>(V, theta, grad, s0_t, s0_r, t, iter, gauge);
  return cudaGetLastError();
}

// ------------------------------------------------------------ total variation

// Smoothed isotropic TV, L = (1/K) sum over voxels x with all three forward
// neighbours inside of n(x) = sqrt(|grad+ I(x)|^2 + eps^2).  Gather form of
// the gradient: voxel y collects -(gx+gy+gz)/n from itself and g_a/n from
// y - e_a for the axes whose neighbour is an interior voxel.
__device__ __forceinline__ bool tv_interior(int i, int j, int k, int nx, int ny, int nz) {
  return i >= 0 && j >= 0 && k >= 0 && i + 1 < nx && j + 1 < ny && k + 1 < nz;
}

__device__ __forceinline__ void tv_terms(const float* vol, long long x, long long nx,
                                         long long nxy, float eps2, float& gx, float& gy,
                                         float& gz, float& inv_n, double& n) {
  const float c = vol[x];
  gx = vol[x + 1] - c;
  gy = vol[x + nx] - c;
  gz = vol[x + nxy] - c;
  // FP32 norm (GB300's FP64 square root and division are far slower than
  // the whole memory-bound pass); the loss sums the norms in FP64
  const float nf = sqrtf(fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, eps2))));
  inv_n = 1.0f / nf;
  n = (double)nf;
}

// Block b of nb, like sharpness_block.
__device__ static void tv_block(const float* __restrict__ vol, int nx, int ny, int nz, float eps,
                                double* __restrict__ block_sums, float* __restrict__ grad, int b,
                                int nb) {
  __shared__ double red[SH_THREADS];
  const long long nvox = (long long)nx * ny * nz;
  const long long nxy = (long long)nx * ny;
  const float invK = (float)(1.0 / (double)nvox);
  const float eps2 = eps * eps;
  double acc = 0.0;
  for (long long x = b * (long long)SH_THREADS + threadIdx.x; x < nvox;
       x += (long long)nb * SH_THREADS) {
    int i, j, k;
    voxel_ijk(x, nx, ny, nvox, i, j, k);
    float gsum = 0.0f, gx, gy, gz, in;
    double n;
    if (tv_interior(i, j, k, nx, ny, nz)) {
      tv_terms(vol, x, nx, nxy, eps2, gx, gy, gz, in, n);
      acc += n;
      gsum -= (gx + gy + gz) * in;
    }
    if (grad) {
      if (tv_interior(i - 1, j, k, nx, ny, nz)) {
        tv_terms(vol, x - 1, nx, nxy, eps2, gx, gy, gz, in, n);
        gsum += gx * in;
      }
      if (tv_interior(i, j - 1, k, nx, ny, nz)) {
        tv_terms(vol, x - nx, nx, nxy, eps2, gx, gy, gz, in, n);
        gsum += gy * in;
      }
      if (tv_interior(i, j, k - 1, nx, ny, nz)) {
        tv_terms(vol, x - nxy, nx, nxy, eps2, gx, gy, gz, in, n);
        gsum += gz * in;
      }
      grad[x] = gsum * invK;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SH_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[b] = red[0];
}

__global__ void tv_kernel(const float* __restrict__ vol, int nx, int ny, int nz, float eps,
                          double* __restrict__ block_sums, float* __restrict__ grad) {
  tv_block(vol, nx, ny, nz, eps, block_sums, grad, blockIdx.x, gridDim.x);
}

// loss = +sum/K (TV is minimised as is); with a history, at history[*iter].
__global__ void tv_finish_kernel(const double* __restrict__ block_sums, int nb, double K,
                                 double* __restrict__ loss, const int* __restrict__ iter,
                                 int hist_len) {
  __shared__ double red[SH_THREADS];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += block_sums[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = SH_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!iter) {
      *loss = red[0] / K;
    } else {
      const int it = *iter;
      if (it >= 0 && it < hist_len) loss[it] = red[0] / K;
    }
  }
}

cudaError_t launch_tv(const float* vol, int nx, int ny, int nz, float eps, double* block_sums,
                      int max_blocks, double* loss, const int* iter, int hist_len, float* grad,
                      cudaStream_t s) {
  long long nvox = (long long)nx * ny * nz;
  int nb = sharpness_blocks(nvox);
  if (nb > max_blocks) nb = max_blocks;
  tv_kernel<<<nb, SH_THREADS, 0, s>>>(vol, nx, ny, nz, eps, block_sums, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tv_finish_kernel<<<1, SH_THREADS, 0, s>>>(block_sums, nb, (double)nvox, loss, iter, hist_len);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- batches
// The per-job kernels above, as launches over the work items of every member
// of a batch table (a __grid_constant__ parameter; grid-stride loops, so any
// grid size covers any member set).  Each item runs exactly the per-job
// arithmetic: a job gives bit for bit the same iteration in a batch as alone.

__global__ void batch_compose_kernel(const __grid_constant__ BatchTable t, int fdk,
                                     unsigned* counter) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0u;  // the forward's work counter
  const int n = t.njobs, total = t.off_view[n];
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < total; w += gridDim.x * blockDim.x) {
    const int j = batch_find(t.off_view, n, w);
    const BatchJob& J = t.job[j];
    compose_view(J.P, J.theta, J.vw, J.scale, fdk, J.sid, J.vi, J.geom, nullptr, w - t.off_view[j]);
  }
}

template <int LOSS>
__global__ void batch_loss_kernel(const __grid_constant__ BatchTable t) {
  const int n = t.njobs, total = t.off_loss[n];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int j = batch_find(t.off_loss, n, w);
    const BatchJob& J = t.job[j];
    const int b = w - t.off_loss[j];
    if (LOSS == 1)
      tv_block(J.vol, J.vi.nx, J.vi.ny, J.vi.nz, J.tv_eps, J.blk, J.dvol, b, J.nblk);
    else
      sharpness_block(J.vol, J.vi.nx, J.vi.ny, J.vi.nz, J.blk, J.dvol, b, J.nblk);
    __syncthreads();
  }
}

template <int LOSS>
__global__ void batch_loss_finish_kernel(const __grid_constant__ BatchTable t) {
  for (int j = blockIdx.x; j < t.njobs; j += gridDim.x) {
    const BatchJob& J = t.job[j];
    const double K = (double)J.vi.nx * J.vi.ny * J.vi.nz;
    loss_finish_hist(J.blk, J.nblk, K, LOSS == 1 ? 1.0 : -1.0, J.hist, J.iter, J.max_iters);
    __syncthreads();
  }
}

__global__ void batch_reduce_kernel(const __grid_constant__ BatchTable t) {
  const int n = t.njobs, total = t.off_view[n];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int j = batch_find(t.off_view, n, w);
    const BatchJob& J = t.job[j];
    reduce_chain_view(J.partials, J.ntiles_v, J.vi, J.P, J.theta, nullptr, J.gth,
                      w - t.off_view[j]);
    __syncthreads();
  }
}

template <int OPT>
__global__ void batch_opt_kernel(const __grid_constant__ BatchTable t) {
  for (int j = blockIdx.x; j < t.njobs; j += gridDim.x) {
    const BatchJob& J = t.job[j];
    if (OPT == 1)
      adam_dev_body(J.V, J.theta, J.gth, J.m1, J.m2, J.lr_t, J.lr_r, J.beta1, J.beta2, J.eps,
                    J.iter, J.gauge);
    else
      gd_dev_body(J.V, J.theta, J.gth, J.lr_t, J.lr_r, J.decay, J.iter, J.gauge);
    __syncthreads();
  }
}

cudaError_t launch_batch_iteration(const BatchTable& tab, unsigned* counter, int dtype, int fdk,
                                   int exact, int loss, int opt, int sms, cudaStream_t s,
                                   const BatchBranches* br) {
  batch_compose_kernel<<<sms, 128, 0, s>>>(tab, fdk, counter);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_batch_forward(tab, counter, dtype, fdk, sms, s);
  if (e != cudaSuccess) return e;
  const int jb = tab.njobs > 0 ? tab.njobs : 1;
  if (loss == 1) {
    batch_loss_kernel<1><<<sms * 8, SH_THREADS, 0, s>>>(tab);
    batch_loss_finish_kernel<1><<<jb, SH_THREADS, 0, s>>>(tab);
  } else {
    batch_loss_kernel<0><<<sms * 8, SH_THREADS, 0, s>>>(tab);
    batch_loss_finish_kernel<0><<<jb, SH_THREADS, 0, s>>>(tab);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tab.njobs > 0) {
    // each member's VJP kernel (the per-job launch, with its own constant
    // parameters) on a branch of its own
    if (!br || br->n < tab.njobs) return cudaErrorInvalidValue;
    e = cudaEventRecord(br->fork, s);
    for (int m = 0; m < tab.njobs && e == cudaSuccess; ++m) {
      const BatchJob& J = tab.job[m];
      e = cudaStreamWaitEvent(br->streams[m], br->fork, 0);
      if (e == cudaSuccess)
        e = launch_vjp_motion(J.dvol, J.proj, dtype, J.pi, J.grad, J.geom, J.vi, fdk, exact,
                              J.partials, nullptr, nullptr, br->streams[m]);
      if (e == cudaSuccess) e = cudaEventRecord(br->joins[m], br->streams[m]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, br->joins[m], 0);
    }
  }
  if (e != cudaSuccess) return e;
  batch_reduce_kernel<<<sms * 8, 256, 0, s>>>(tab);
  if (opt == 1)
    batch_opt_kernel<1><<<jb, 256, 0, s>>>(tab);
  else
    batch_opt_kernel<0><<<jb, 256, 0, s>>>(tab);
  return cudaGetLastError();
}

}  // namespace bpk
