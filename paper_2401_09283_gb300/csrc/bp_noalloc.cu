// Allocation-free variant of the sharpness loss (bp_sharpness_noalloc).
//
// Some callers cannot allocate device memory while they run: code that is
// being recorded into a CUDA graph (an allocation during stream capture
// breaks the capture), hosts that hand all device memory to their own pool at
// start-up and forbid further cudaMalloc calls, and real-time loops that must
// not block on the allocator.  For them this file keeps the per-chunk partial
// sums of the loss in a fixed device array that the library owns, so the call
// needs only the caller's input and output buffers.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it (NA_MAX_CHUNKS doubles = 256 KiB per GPU).  Every call shares it:
// two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and give wrong results.  Each call
// writes every slot it later reads, so nothing needs clearing between calls.
#include <mutex>

#include "bp_gb300.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;
constexpr long long NA_CHUNK = (long long)NA_THREADS * NA_PER_THREAD;  // voxels per block
constexpr int NA_MAX_CHUNKS = 32768;                                   // 512^3 voxels at most
constexpr int NA_MAX_DEVICES = 64;

// Scratch: one FP64 partial sum per chunk of NA_CHUNK voxels.
static __device__ __align__(256) double g_sharp_partials[NA_MAX_CHUNKS];

// Host-side cache of the array's device address, one per device.  In host
// code the name g_sharp_partials is only a stand-in: its address must come
// from cudaGetSymbolAddress with the device current.
void* g_addr[NA_MAX_DEVICES] = {};
std::mutex g_mu;

// Block b sums the squared forward differences of voxels [b*NA_CHUNK,
// (b+1)*NA_CHUNK) into partials[b] and writes dL/dI of those voxels:
// L = -(1/K) sum_pairs (I[y] - I[x])^2, dL/dI[x] = (2/K) sum_n (I[n] - I[x]).
__global__ void sharp_chunk_kernel(const float* __restrict__ vol, int nx, int ny, int nz,
                                   double* __restrict__ partials, float* __restrict__ grad) {
  __shared__ double red[NA_THREADS];
  const long long nvox = (long long)nx * ny * nz;
  const long long nxy = (long long)nx * ny;
  const float g2 = (float)(2.0 / (double)nvox);
  double acc = 0.0;
  const long long base = (long long)blockIdx.x * NA_CHUNK;
  for (int r = 0; r < NA_PER_THREAD; ++r) {
    const long long x = base + (long long)r * NA_THREADS + threadIdx.x;
    if (x >= nvox) break;
    // nvox <= 512^3 < 2^32: 32-bit index arithmetic
    const unsigned ux = (unsigned)x, qx = ux / (unsigned)nx;
    const int i = (int)(ux - qx * (unsigned)nx), j = (int)(qx % (unsigned)ny),
              k = (int)(qx / (unsigned)ny);
    const float c = vol[x];
    float gsum = 0.0f;
    // the voxel's squared forward differences summed in FP32 (x, y, z order),
    // accumulated in FP64 -- the per-voxel arithmetic of bp_sharpness
    float q = 0.0f;
    if (i + 1 < nx) {
      const float d = vol[x + 1] - c;
      q = d * d;
      gsum += d;
    }
    if (j + 1 < ny) {
      const float d = vol[x + nx] - c;
      q = fmaf(d, d, q);
      gsum += d;
    }
    if (k + 1 < nz) {
      const float d = vol[x + nxy] - c;
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
  for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// One block: fixed-order sum of the chunk partials -> loss.
__global__ void sharp_chunk_finish_kernel(const double* __restrict__ partials, int nb, double K,
                                          double* __restrict__ loss) {
  __shared__ double red[NA_THREADS];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += NA_THREADS) acc += partials[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = -red[0] / K;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int bp_sharpness_noalloc(const float* vol, const bp_vol_desc* vdesc, double* loss,
                                    float* dL_dvol, void* stream) {
  if (!vdesc || !loss) return BP_ERR_INVALID_ARG;
  if (vdesc->nx < 0 || vdesc->ny < 0 || vdesc->nz < 0) return BP_ERR_INVALID_ARG;
  const long long nvox = (long long)vdesc->nx * vdesc->ny * vdesc->nz;
  const long long nchunks = (nvox + NA_CHUNK - 1) / NA_CHUNK;
  if (nchunks > NA_MAX_CHUNKS) return BP_ERR_UNSUPPORTED;  // more than 512^3 voxels
  if (!on_device(loss) || (nvox > 0 && (!vol || !on_device(vol))) ||
      (dL_dvol && !on_device(dL_dvol)))
    return BP_ERR_INVALID_ARG;  // device memory only: host data would need staging buffers
  cudaStream_t s = (cudaStream_t)stream;
  if (nvox == 0) {
    // memset of caller memory allocates nothing
    return cudaMemsetAsync(loss, 0, sizeof(double), s) == cudaSuccess ? BP_OK : BP_ERR_CUDA;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BP_ERR_CUDA;
  }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return BP_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  {
    // first call on this device: look up the array's device address (with
    // this device current); later calls reuse it
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_sharp_partials);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return BP_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  sharp_chunk_kernel<<<(int)nchunks, NA_THREADS, 0, s>>>(vol, vdesc->nx, vdesc->ny, vdesc->nz,
                                                          (double*)scratch, dL_dvol);
  if (cudaGetLastError() != cudaSuccess) return BP_ERR_CUDA;
  sharp_chunk_finish_kernel<<<1, NA_THREADS, 0, s>>>((const double*)scratch, (int)nchunks,
                                                      (double)nvox, loss);
  if (cudaGetLastError() != cudaSuccess) return BP_ERR_CUDA;
  return BP_OK;
}
