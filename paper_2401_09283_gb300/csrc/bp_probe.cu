// Throughput probes behind the roofline denominators: FP32 FMA lane
// operations per second with scalar FFMA and with packed f32x2 FMA (each
// packed instruction counted as two lane operations), and FP32 atomic adds
// per second in L2 (scalar reductions, coalesced and in the scattered pattern
// of the data VJP).  Timed with CUDA events; the paper has no counterpart.
#include "bp_internal.cuh"

namespace bpk {

constexpr int PROBE_ITERS = 4096;

__global__ void __launch_bounds__(256) probe_ffma_kernel(float* out, float a, float b) {
  float x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
        x6 = x0 + 6, x7 = x0 + 7;
#pragma unroll 16
  for (int i = 0; i < PROBE_ITERS; ++i) {
    x0 = fmaf(x0, a, b);
    x1 = fmaf(x1, a, b);
    x2 = fmaf(x2, a, b);
    x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b);
    x5 = fmaf(x5, a, b);
    x6 = fmaf(x6, a, b);
    x7 = fmaf(x7, a, b);
  }
  const float s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_ffma2_kernel(float* out, float a, float b) {
  unsigned long long x[8], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float lo = threadIdx.x + 2 * k, hi = lo + 1;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
  }
#pragma unroll 16
  for (int i = 0; i < PROBE_ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == 1.2345f) out[blockIdx.x] = s;
}

// Every thread adds to `per_thread` addresses; coalesced: lane l of a warp
// to consecutive words; scattered: the 2 x 2 taps of samples ~2.6 px apart
// on a 616-wide image (the data VJP's pattern).
template <bool SCATTER>
__global__ void __launch_bounds__(256) probe_red_kernel(float* buf, long long words, int per_thread) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    long long a;
    if (SCATTER) {
      const int lane = threadIdx.x & 31, q = k & 3;
      const long long s = (t >> 5) * 97 + (long long)(k >> 2) * 131;  // a sample per (warp, k/4)
      const long long row = (s * 3) % 478, col = (long long)(lane * 2.6f) + (s % 400);
      a = (row + (q >> 1)) * 616 + col + (q & 1) + ((s / 478) % 64) * 616 * 480;
    } else {
      a = (t + (long long)k * gridDim.x * blockDim.x) % words;
    }
    atomicAdd(buf + (a % words), 1.0f);
  }
}

cudaError_t run_probe(int kind, float* scratch, long long scratch_words, int sms, double* result,
                      cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8, per = 64;
  double ops = 0.0;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
    cudaEventRecord(e0, s);
    if (kind == 0) {
      probe_ffma_kernel<<<blocks, 256, 0, s>>>(scratch, 0.999f, 0.001f);
      ops = (double)blocks * 256 * PROBE_ITERS * 8;
    } else if (kind == 1) {
      probe_ffma2_kernel<<<blocks, 256, 0, s>>>(scratch, 0.999f, 0.001f);
      ops = (double)blocks * 256 * PROBE_ITERS * 16;
    } else {
      const int rb = sms * 64;
      if (kind == 2)
        probe_red_kernel<false><<<rb, 256, 0, s>>>(scratch, scratch_words, per);
      else
        probe_red_kernel<true><<<rb, 256, 0, s>>>(scratch, scratch_words, per);
      ops = (double)rb * 256 * per;
    }
    e = cudaGetLastError();
    cudaEventRecord(e1, s);
  }
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) *result = ops / (ms * 1e-3);
  return e;
}

}  // namespace bpk
