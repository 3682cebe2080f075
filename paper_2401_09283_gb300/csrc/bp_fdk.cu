// FDK preprocessing of raw line integrals (the filtering of Sec. III; the
// short-scan weights that the 200-degree arcs need): per pixel the cosine
// weight SDD / sqrt(SDD^2 + x^2 + y^2) and the redundancy weight of its ray
// (Parker's, generalised to over-scan by delta = (arc - pi)/2 in place of the
// maximum fan angle; 1/2 for a full scan), then along every detector row the
// linear convolution with the Shepp-Logan ramp h[n] = -2 / (pi^2 tau^2
// (4 n^2 - 1)), tau = pitch * SID / SDD, times tau.
//
// The ramp and the per-(view, column) redundancy weights are tabulated in
// FP64 and rounded to FP32; the convolution is a direct O(nu^2) sum in FP32,
// four detector rows per CTA so that one broadcast float4 load feeds four
// FMAs per tap.  With ext > 0 (truncation correction, Sec. IV-D) every
// weighted row is extended by ext pixels per side falling linearly from its
// edge value to 0 (extension pixel m = 1..ext holds edge * (1 - m/ext)) and
// the measured nu pixels of the filtered, extended row are kept.
#include "bp_internal.cuh"

namespace bpk {

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ double parker_w(double beta, double gamma, double arc) {
  const double delta = 0.5 * (arc - kPi);
  double w = 1.0;
  if (beta < 2.0 * delta + 2.0 * gamma) {
    const double s = sin(0.25 * kPi * beta / (delta + gamma));
    w = s * s;
  } else if (beta > kPi + 2.0 * gamma) {
    const double s = sin(0.25 * kPi * (kPi + 2.0 * delta - beta) / (delta - gamma));
    w = s * s;
  }
  return fmin(fmax(w, 0.0), 1.0);
}

// h[m + ne - 1] for |m| < ne = nu + 2 ext, then the redundancy weight of
// (view j, column a) at [2 ne - 1 + j nu + a].
__global__ void fdk_tables_kernel(int V, int nu, int ext, double pitch, double sid, double sdd,
                                  double arc, float* __restrict__ tab) {
  const double tau = pitch * sid / sdd;
  const bool full = arc >= 2.0 * kPi - 1e-12;
  const double dbeta = full ? arc / V : (V > 1 ? arc / (V - 1) : 0.0);
  const int ne = nu + 2 * ext;
  const long long nh = 2LL * ne - 1, n = nh + (long long)V * nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nh) {
      const double m = (double)(e - (ne - 1));
      tab[e] = (float)(-2.0 / (kPi * kPi * tau * tau * (4.0 * m * m - 1.0)));
    } else {
      const long long q = e - nh;
      const int j = (int)(q / nu), a = (int)(q % nu);
      const double x = (a - 0.5 * (nu - 1)) * pitch;
      tab[e] = full ? 0.5f : (float)parker_w(j * dbeta, atan(x / sdd), arc);
    }
  }
}

constexpr int ROWS = 4;

// grid (ceil(nv / ROWS), V); dynamic shared memory: ne = nu + 2 ext float4
// (the four weighted, extended rows interleaved) + (2 ne - 1) floats (the ramp).
__global__ void __launch_bounds__(256) fdk_conv_kernel(const float* __restrict__ raw, int nu,
                                                       int nv, int ext, double pitch, double sdd,
                                                       float tau, const float* __restrict__ tab,
                                                       float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ne = nu + 2 * ext;
  float4* ext_rows = reinterpret_cast<float4*>(smem);
  float4* rows = ext_rows + ext;  // rows[k], k = -ext .. nu + ext - 1
  float* h = reinterpret_cast<float*>(smem + sizeof(float4) * (size_t)ne);
  const int j = blockIdx.y, b0 = blockIdx.x * ROWS;
  const float* park = tab + (2 * ne - 1) + (size_t)j * nu;
  for (int e = threadIdx.x; e < 2 * ne - 1; e += blockDim.x) h[e] = tab[e];
  for (int k = threadIdx.x; k < nu; k += blockDim.x) {
    const double x = (k - 0.5 * (nu - 1)) * pitch;
    float v[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int b = b0 + r;
      v[r] = 0.0f;
      if (b < nv) {
        const double y = (b - 0.5 * (nv - 1)) * pitch;
        const double c = sdd / sqrt(sdd * sdd + x * x + y * y);
        v[r] = (float)(c * (double)park[k]) * raw[((size_t)j * nv + b) * nu + k];
      }
    }
    rows[k] = make_float4(v[0], v[1], v[2], v[3]);
  }
  __syncthreads();
  for (int m = 1 + threadIdx.x; m <= ext; m += blockDim.x) {  // linear fall-off to 0
    const float f = 1.0f - (float)m / (float)ext;
    const float4 l = rows[0], r = rows[nu - 1];
    rows[-m] = make_float4(l.x * f, l.y * f, l.z * f, l.w * f);
    rows[nu - 1 + m] = make_float4(r.x * f, r.y * f, r.z * f, r.w * f);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < nu; a += blockDim.x) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const float* ha = h + a + ext + ne - 1;  // ha[-k'] = h[(a + ext) - k'], k' = k + ext
#pragma unroll 4
    for (int kk = 0; kk < ne; ++kk) {
      const int k = kk - ext;
      const float4 p = rows[k];
      const float w = ha[-kk];
      s0 = fmaf(w, p.x, s0);
      s1 = fmaf(w, p.y, s1);
      s2 = fmaf(w, p.z, s2);
      s3 = fmaf(w, p.w, s3);
    }
    const float s[ROWS] = {s0, s1, s2, s3};
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
      if (b0 + r < nv) out[((size_t)j * nv + b0 + r) * nu + a] = tau * s[r];
  }
}

}  // namespace

size_t fdk_table_floats(int V, int nu, int ext) {
  return (size_t)(2 * (nu + 2 * ext) - 1) + (size_t)V * nu;
}

size_t fdk_smem_bytes(int nu, int ext) {
  const size_t ne = (size_t)nu + 2 * (size_t)ext;
  return sizeof(float) * (4 * ne + 2 * ne - 1);
}

cudaError_t launch_fdk_filter(const float* raw, int V, int nv, int nu, int ext, double pitch,
                              double sid, double sdd, double arc, float* tab, float* out,
                              cudaStream_t s) {
  if (V == 0 || nv == 0) return cudaSuccess;
  const long long n = (long long)fdk_table_floats(V, nu, ext);
  long long nb = (n + 255) / 256;
  if (nb > 152 * 16) nb = 152 * 16;
  fdk_tables_kernel<<<(int)nb, 256, 0, s>>>(V, nu, ext, pitch, sid, sdd, arc, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = fdk_smem_bytes(nu, ext);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(fdk_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((nv + ROWS - 1) / ROWS, V);
  fdk_conv_kernel<<<grid, 256, smem, s>>>(raw, nu, nv, ext, pitch, sdd,
                                          (float)(pitch * sid / sdd), tab, out);
  return cudaGetLastError();
}

}  // namespace bpk
