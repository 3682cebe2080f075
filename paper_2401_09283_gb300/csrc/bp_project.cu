// Voxel-driven kernels of the backprojection (Eq. 3) and its vector-Jacobian
// products (Eqs. 4-5) for sm_103a.
//
// Work decomposition: a CTA of 256 threads owns a 16 x 16 x ZB box of voxels
// (one z-column of ZB voxels per thread, warps of 8 x 4 columns) and loops
// over all views.  For each batch of 32 views one thread per view computes,
// in FP64, the anchored per-tile view record (TileView): the integer pixel
// nearest the projection of the tile centre, the anchored rows and the
// classification of the whole box as entirely off the detector (SKIP),
// entirely inside it (INTERIOR: no bounds checks) or crossing an edge (EDGE:
// clamped coordinates and checked taps).  The inner loops are plain FP32:
// three FMAs for (u, v, w), one MUFU reciprocal, floor via a round-down add
// of 1.5*2^23, bilinear interpolation with FP32 lerps (hardware texture
// filtering is not used: its weights are 8-bit fixed point).
#include "bp_internal.cuh"

namespace bpk {

constexpr float MAGIC = 12582912.0f;   // 1.5 * 2^23
constexpr int MAGIC_BITS = 0x4B400000;

template <typename T>
__device__ __forceinline__ float ldv(const T* p);
template <>
__device__ __forceinline__ float ldv<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ldv<__half>(const __half* p) {
  return __half2float(__ldg(p));
}
template <>
__device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ------------------------------------------------------------ tile set-up

// FP64 set-up of one (tile, view) record.  qc: tile centre in the index
// frame; half: half-extent of the box of voxel centres.
__device__ void setup_tile_view(TileView& t, const ViewGeom& g, const double qc[3],
                                const double half[3], int nu, int nv, bool with_scale) {
  const double* M = g.P;
  double uc = fma(M[0], qc[0], fma(M[1], qc[1], fma(M[2], qc[2], M[3])));
  double vc = fma(M[4], qc[0], fma(M[5], qc[1], fma(M[6], qc[2], M[7])));
  double wc = fma(M[8], qc[0], fma(M[9], qc[1], fma(M[10], qc[2], M[11])));
  int au = 0, av = 0;
  if (wc > 0.0) {
    double a = floor(uc / wc), b = floor(vc / wc);
    a = fmin(fmax(a, -1048576.0), 1048576.0);
    b = fmin(fmax(b, -1048576.0), 1048576.0);
    au = (int)a;
    av = (int)b;
  }
  double Ru[4], Rv[4], Rw[4];
  for (int k = 0; k < 4; ++k) {
    Ru[k] = M[k] - au * M[8 + k];
    Rv[k] = M[4 + k] - av * M[8 + k];
    Rw[k] = M[8 + k];
  }
  double U0 = fma(Ru[0], qc[0], fma(Ru[1], qc[1], fma(Ru[2], qc[2], Ru[3])));
  double V0 = fma(Rv[0], qc[0], fma(Rv[1], qc[1], fma(Rv[2], qc[2], Rv[3])));
  double W0 = wc;
  t.U0 = (float)U0;
  t.V0 = (float)V0;
  t.W0 = (float)W0;
  for (int k = 0; k < 3; ++k) {
    t.ru[k] = (float)Ru[k];
    t.rv[k] = (float)Rv[k];
    t.rw[k] = (float)Rw[k];
  }
  t.au = au;
  t.av = av;
  t.wgt = (float)(with_scale ? g.wgt * g.scale : g.wgt);
  // classify the box by its 8 corners (u/w and v/w are linear-fractional, so
  // their extremes over a box with w > 0 are at the corners)
  int npos = 0;
  double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
  for (int c = 0; c < 8; ++c) {
    double d0 = (c & 1) ? half[0] : -half[0];
    double d1 = (c & 2) ? half[1] : -half[1];
    double d2 = (c & 4) ? half[2] : -half[2];
    double w = W0 + Rw[0] * d0 + Rw[1] * d1 + Rw[2] * d2;
    if (!(w > 0.0)) continue;
    ++npos;
    double u = (U0 + Ru[0] * d0 + Ru[1] * d1 + Ru[2] * d2) / w + au;
    double v = (V0 + Rv[0] * d0 + Rv[1] * d1 + Rv[2] * d2) / w + av;
    umin = fmin(umin, u);
    umax = fmax(umax, u);
    vmin = fmin(vmin, v);
    vmax = fmax(vmax, v);
  }
  const double m = 0.01;  // >> the FP32 coordinate error of the inner loops
  if (npos == 0) {
    t.mode = MODE_SKIP;
  } else if (npos < 8) {
    t.mode = MODE_EDGE;
  } else if (umax <= -1.0 - m || umin >= nu + m || vmax <= -1.0 - m || vmin >= nv + m) {
    t.mode = MODE_SKIP;
  } else if (umin >= m && umax <= nu - 1 - m && vmin >= m && vmax <= nv - 1 - m) {
    t.mode = MODE_INTERIOR;
  } else {
    t.mode = MODE_EDGE;
  }
}

// Detector position of one voxel in the anchored frame.
struct Sample {
  float rwi;     // 1/w
  float x, y;    // u/w - au, v/w - av (clamped in EDGE mode)
  float tu, tv;  // fractional parts
  int iu, iv;    // absolute floor pixel
  bool ok;       // w > 0
};

template <bool EDGE>
__device__ __forceinline__ Sample locate(float u, float v, float w, const TileView& t, int nu,
                                         int nv) {
  Sample s;
  s.ok = true;
  if (EDGE) s.ok = w > 1e-20f;  // a voxel at (or behind) the source plane contributes nothing
  s.rwi = rcp_approx(w);
  float x = u * s.rwi, y = v * s.rwi;
  if (EDGE) {
    // Clamp far-off coordinates into (-2, -1) or (n, n+1): all four taps are
    // then outside the detector, so value and derivatives are 0 there (a
    // clamp to exactly -1 would sit on the kink of the zero-padded
    // interpolant, where the exact derivative is d[0], not 0).
    x = fminf(fmaxf(x, -1.5f - (float)t.au), (float)nu + 0.5f - (float)t.au);
    y = fminf(fmaxf(y, -1.5f - (float)t.av), (float)nv + 0.5f - (float)t.av);
  }
  float rx = __fadd_rd(x, MAGIC), ry = __fadd_rd(y, MAGIC);
  s.tu = x - (rx - MAGIC);
  s.tv = y - (ry - MAGIC);
  s.iu = __float_as_int(rx) - MAGIC_BITS + t.au;
  s.iv = __float_as_int(ry) - MAGIC_BITS + t.av;
  s.x = x;
  s.y = y;
  return s;
}

// Four taps of a [nv][rs] image at (iu..iu+1, iv..iv+1), zero outside.
template <bool EDGE, typename T>
__device__ __forceinline__ void taps(const T* img, long long rs, int nu, int nv, const Sample& s,
                                     float& d00, float& d10, float& d01, float& d11) {
  if (!EDGE) {
    const T* p = img + (long long)s.iv * rs + s.iu;
    d00 = ldv(p);
    d10 = ldv(p + 1);
    d01 = ldv(p + rs);
    d11 = ldv(p + rs + 1);
  } else {
    bool u0 = (unsigned)s.iu < (unsigned)nu, u1 = (unsigned)(s.iu + 1) < (unsigned)nu;
    bool v0 = (unsigned)s.iv < (unsigned)nv, v1 = (unsigned)(s.iv + 1) < (unsigned)nv;
    const T* p = img + (long long)s.iv * rs + s.iu;
    d00 = (u0 && v0 && s.ok) ? ldv(p) : 0.0f;
    d10 = (u1 && v0 && s.ok) ? ldv(p + 1) : 0.0f;
    d01 = (u0 && v1 && s.ok) ? ldv(p + rs) : 0.0f;
    d11 = (u1 && v1 && s.ok) ? ldv(p + rs + 1) : 0.0f;
  }
}

__device__ __forceinline__ float bilerp(float tu, float tv, float d00, float d10, float d01,
                                        float d11) {
  float top = fmaf(tu, d10 - d00, d00);
  float bot = fmaf(tu, d11 - d01, d01);
  return fmaf(tv, bot - top, top);
}

struct TileIdx {
  int tx, ty, tz, lx, ly;
  float dx, dy;
  double qc[3], half[3];
};

template <int ZB>
__device__ __forceinline__ TileIdx tile_index(const VolInfo& vi) {
  TileIdx ti;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ti.lx = (warp & 1) * 8 + (lane & 7);
  ti.ly = (warp >> 1) * 4 + (lane >> 3);
  const int tile = blockIdx.x;
  ti.tx = tile % vi.tiles_x;
  ti.ty = (tile / vi.tiles_x) % vi.tiles_y;
  ti.tz = tile / (vi.tiles_x * vi.tiles_y);
  ti.dx = ti.lx - 0.5f * (TX - 1);
  ti.dy = ti.ly - 0.5f * (TY - 1);
  ti.qc[0] = ti.tx * TX + 0.5 * (TX - 1) - vi.cx;
  ti.qc[1] = ti.ty * TY + 0.5 * (TY - 1) - vi.cy;
  ti.qc[2] = ti.tz * ZB + 0.5 * (ZB - 1) - vi.cz;
  ti.half[0] = 0.5 * (TX - 1);
  ti.half[1] = 0.5 * (TY - 1);
  ti.half[2] = 0.5 * (ZB - 1);
  return ti;
}

// ------------------------------------------------------------------ forward

template <int ZB, typename T, bool FDK, bool EDGE>
__device__ __forceinline__ void forward_view(const T* img, long long rs, int nu, int nv,
                                             const TileView& t, float dx, float dy,
                                             float (&acc)[ZB]) {
  float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    const float dz = k - 0.5f * (ZB - 1);
    Sample s = locate<EDGE>(fmaf(dz, t.ru[2], u0), fmaf(dz, t.rv[2], v0), fmaf(dz, t.rw[2], w0),
                            t, nu, nv);
    if (EDGE && !s.ok) continue;
    float d00, d10, d01, d11;
    taps<EDGE>(img, rs, nu, nv, s, d00, d10, d01, d11);
    float val = bilerp(s.tu, s.tv, d00, d10, d01, d11);
    float wv = FDK ? s.rwi * (s.rwi * t.wgt) : t.wgt;
    acc[k] = fmaf(val, wv, acc[k]);
  }
}

template <int ZB, typename T, bool FDK>
__global__ void __launch_bounds__(NT, 2)
    forward_kernel(const T* __restrict__ proj, ProjInfo pi, const ViewGeom* __restrict__ geom,
                   VolInfo vi, float* __restrict__ vol) {
  __shared__ TileView tvs[VB];
  const TileIdx ti = tile_index<ZB>(vi);
  float acc[ZB];
#pragma unroll
  for (int k = 0; k < ZB; ++k) acc[k] = 0.0f;
  for (int j0 = 0; j0 < pi.nviews; j0 += VB) {
    const int nb = min(VB, pi.nviews - j0);
    __syncthreads();
    if (threadIdx.x < nb)
      setup_tile_view(tvs[threadIdx.x], geom[j0 + threadIdx.x], ti.qc, ti.half, pi.nu, pi.nv,
                      true);
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      const TileView t = tvs[b];
      if (t.mode == MODE_SKIP) continue;
      const T* img = proj + (long long)(j0 + b) * pi.vs;
      if (t.mode == MODE_INTERIOR)
        forward_view<ZB, T, FDK, false>(img, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, acc);
      else
        forward_view<ZB, T, FDK, true>(img, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, acc);
    }
  }
  const int i = ti.tx * TX + ti.lx, j = ti.ty * TY + ti.ly;
  if (i < vi.nx && j < vi.ny) {
#pragma unroll
    for (int k = 0; k < ZB; ++k) {
      const int z = ti.tz * ZB + k;
      if (z < vi.nz) vol[((long long)z * vi.ny + j) * vi.nx + i] = acc[k];
    }
  }
}

constexpr int ZB_FWD = 16;
constexpr int ZB_VJP = 16;

template <typename T, bool FDK>
static void forward_dispatch(const void* proj, const ProjInfo& pi, const ViewGeom* geom,
                             const VolInfo& vi, float* vol, cudaStream_t s) {
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  forward_kernel<ZB_FWD, T, FDK><<<ntiles, NT, 0, s>>>((const T*)proj, pi, geom, vi, vol);
}

cudaError_t launch_forward(const void* proj, int dtype, const ProjInfo& pi, const ViewGeom* geom,
                           const VolInfo& vi, int fdk, float* vol, cudaStream_t s) {
  if (vi.zb != ZB_FWD) return cudaErrorInvalidValue;
  if (dtype == 0) {
    fdk ? forward_dispatch<float, true>(proj, pi, geom, vi, vol, s)
        : forward_dispatch<float, false>(proj, pi, geom, vi, vol, s);
  } else if (dtype == 1) {
    fdk ? forward_dispatch<__half, true>(proj, pi, geom, vi, vol, s)
        : forward_dispatch<__half, false>(proj, pi, geom, vi, vol, s);
  } else {
    fdk ? forward_dispatch<__nv_bfloat16, true>(proj, pi, geom, vi, vol, s)
        : forward_dispatch<__nv_bfloat16, false>(proj, pi, geom, vi, vol, s);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------- gradient images

// g_u, g_v of one view in value per pixel: (d[+1] - d[-1]) / 2 inside,
// one-sided first differences on the two edge pixels (Sec. II-B.2), in
// stored units (the per-view dequantisation scale is applied with the view
// weight); output contiguous [V][nv][nu] float2.
template <typename T>
__global__ void grad_images_kernel(const T* __restrict__ proj, ProjInfo pi,
                                   float2* __restrict__ grad) {
  const long long n = (long long)pi.nviews * pi.nv * pi.nu;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e % pi.nu);
    const int b = (int)((e / pi.nu) % pi.nv);
    const int j = (int)(e / ((long long)pi.nu * pi.nv));
    const T* row = proj + (long long)j * pi.vs + (long long)b * pi.rs;
    float gu = 0.0f, gv = 0.0f;
    if (pi.nu >= 2) {
      if (a == 0) gu = ldv(row + 1) - ldv(row);
      else if (a == pi.nu - 1) gu = ldv(row + a) - ldv(row + a - 1);
      else gu = 0.5f * (ldv(row + a + 1) - ldv(row + a - 1));
    }
    if (pi.nv >= 2) {
      if (b == 0) gv = ldv(row + pi.rs + a) - ldv(row + a);
      else if (b == pi.nv - 1) gv = ldv(row + a) - ldv(row - pi.rs + a);
      else gv = 0.5f * (ldv(row + pi.rs + a) - ldv(row - pi.rs + a));
    }
    grad[e] = make_float2(gu, gv);
  }
}

cudaError_t launch_grad_images(const void* proj, int dtype, const ProjInfo& pi, float2* grad,
                               cudaStream_t s) {
  const long long n = (long long)pi.nviews * pi.nv * pi.nu;
  if (n == 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 64) nb = 152 * 64;
  if (dtype == 0)
    grad_images_kernel<float><<<(int)nb, 256, 0, s>>>((const float*)proj, pi, grad);
  else if (dtype == 1)
    grad_images_kernel<__half><<<(int)nb, 256, 0, s>>>((const __half*)proj, pi, grad);
  else
    grad_images_kernel<__nv_bfloat16>
        <<<(int)nb, 256, 0, s>>>((const __nv_bfloat16*)proj, pi, grad);
  return cudaGetLastError();
}

// ------------------------------------------------------- VJP w.r.t. Phat

// Sum of 16 per-lane values over the warp, scattered: lane l ends with the
// total of slot 8*b4 + 4*b3 + 2*b2 + b1 (b_i = bit i of l); lanes 2s and 2s+1
// hold the same slot.
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const bool hi = lane & 16;
    float send = hi ? v[s] : v[s + 8];
    float keep = hi ? v[s + 8] : v[s];
    v[s] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const bool hi = lane & 8;
    float send = hi ? v[s] : v[s + 4];
    float keep = hi ? v[s + 4] : v[s];
    v[s] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const bool hi = lane & 4;
    float send = hi ? v[s] : v[s + 2];
    float keep = hi ? v[s + 2] : v[s];
    v[s] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    float send = hi ? v[0] : v[1];
    float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

__device__ __forceinline__ int scatter_slot(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Per voxel-view, with s = delta * c * omega and r = 1/w, the derivative of
// the weighted sample with respect to (u_rel, v_rel, w) (Eq. 4 in the
// anchored frame): a = s*r*(g_u, g_v, -(g_u x + g_v y)) and, with FDK, the
// derivative of omega = wgt r^2 adds -2 s r val to the w component.  The
// 3x4 outer product with (dq, 1) is accumulated as S_r = sum a_r and
// Z_r = sum a_r dz along the thread's column; dx, dy are constant per thread.
template <int ZB, typename T, bool FDK, bool EXACT, bool EDGE>
__device__ __forceinline__ void vjp_view(const T* img, const float2* gimg, long long rs, int nu,
                                         int nv, const TileView& t, float dx, float dy,
                                         const float (&delta)[ZB], float (&S)[3], float (&Z)[3]) {
  float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    const float dz = k - 0.5f * (ZB - 1);
    Sample s = locate<EDGE>(fmaf(dz, t.ru[2], u0), fmaf(dz, t.rv[2], v0), fmaf(dz, t.rw[2], w0),
                            t, nu, nv);
    if (EDGE && !s.ok) continue;
    float gu, gv, val = 0.0f;
    if (EXACT) {
      float d00, d10, d01, d11;
      taps<EDGE>(img, rs, nu, nv, s, d00, d10, d01, d11);
      const float a = d10 - d00, b = d11 - d01;
      gu = fmaf(s.tv, b - a, a);
      const float c = d01 - d00, d = d11 - d10;
      gv = fmaf(s.tu, d - c, c);
      if (FDK) val = bilerp(s.tu, s.tv, d00, d10, d01, d11);
    } else {
      float2 g00, g10, g01, g11;
      const float2 z2 = make_float2(0.0f, 0.0f);
      if (!EDGE) {
        const float2* p = gimg + (long long)s.iv * nu + s.iu;
        g00 = __ldg(p);
        g10 = __ldg(p + 1);
        g01 = __ldg(p + nu);
        g11 = __ldg(p + nu + 1);
      } else {
        bool uu0 = (unsigned)s.iu < (unsigned)nu, uu1 = (unsigned)(s.iu + 1) < (unsigned)nu;
        bool vv0 = (unsigned)s.iv < (unsigned)nv, vv1 = (unsigned)(s.iv + 1) < (unsigned)nv;
        const float2* p = gimg + (long long)s.iv * nu + s.iu;
        g00 = (uu0 && vv0 && s.ok) ? __ldg(p) : z2;
        g10 = (uu1 && vv0 && s.ok) ? __ldg(p + 1) : z2;
        g01 = (uu0 && vv1 && s.ok) ? __ldg(p + nu) : z2;
        g11 = (uu1 && vv1 && s.ok) ? __ldg(p + nu + 1) : z2;
      }
      gu = bilerp(s.tu, s.tv, g00.x, g10.x, g01.x, g11.x);
      gv = bilerp(s.tu, s.tv, g00.y, g10.y, g01.y, g11.y);
      if (FDK) {
        float d00, d10, d01, d11;
        taps<EDGE>(img, rs, nu, nv, s, d00, d10, d01, d11);
        val = bilerp(s.tu, s.tv, d00, d10, d01, d11);
      }
    }
    float sd = delta[k] * (FDK ? s.rwi * (s.rwi * t.wgt) : t.wgt);
    const float sr = sd * s.rwi;
    const float a0 = gu * sr, a1 = gv * sr;
    float a2 = -fmaf(a0, s.x, a1 * s.y);
    if (FDK) a2 = fmaf(-2.0f * sr, val, a2);
    S[0] += a0;
    S[1] += a1;
    S[2] += a2;
    Z[0] = fmaf(a0, dz, Z[0]);
    Z[1] = fmaf(a1, dz, Z[1]);
    Z[2] = fmaf(a2, dz, Z[2]);
  }
}

template <int ZB, typename T, bool FDK, bool EXACT>
__global__ void __launch_bounds__(NT, 2)
    vjp_motion_kernel(const float* __restrict__ dvol, const T* __restrict__ proj, ProjInfo pi,
                      const float2* __restrict__ grad, const ViewGeom* __restrict__ geom,
                      VolInfo vi, float* __restrict__ partials) {
  __shared__ TileView tvs[VB];
  __shared__ float red[NT / 32][VB][12];
  const TileIdx ti = tile_index<ZB>(vi);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const int i = ti.tx * TX + ti.lx, j = ti.ty * TY + ti.ly;
  float delta[ZB];
  bool nz = false;
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    const int z = ti.tz * ZB + k;
    delta[k] = (i < vi.nx && j < vi.ny && z < vi.nz)
                   ? __ldg(dvol + ((long long)z * vi.ny + j) * vi.nx + i)
                   : 0.0f;
    nz |= delta[k] != 0.0f;
  }
  const bool any = __syncthreads_or(nz);
  for (int j0 = 0; j0 < pi.nviews; j0 += VB) {
    const int nb = min(VB, pi.nviews - j0);
    __syncthreads();
    if (threadIdx.x < nb)
      setup_tile_view(tvs[threadIdx.x], geom[j0 + threadIdx.x], ti.qc, ti.half, pi.nu, pi.nv,
                      true);
    __syncthreads();
    if (any) {
      for (int b = 0; b < nb; ++b) {
        const TileView t = tvs[b];
        if (t.mode == MODE_SKIP) continue;
        const T* img = proj + (long long)(j0 + b) * pi.vs;
        const float2* gimg = EXACT ? nullptr : grad + (long long)(j0 + b) * pi.nv * pi.nu;
        float S[3] = {0.0f, 0.0f, 0.0f}, Z[3] = {0.0f, 0.0f, 0.0f};
        if (t.mode == MODE_INTERIOR)
          vjp_view<ZB, T, FDK, EXACT, false>(img, gimg, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy,
                                             delta, S, Z);
        else
          vjp_view<ZB, T, FDK, EXACT, true>(img, gimg, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy,
                                            delta, S, Z);
        float v[16];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          v[4 * r + 0] = ti.dx * S[r];
          v[4 * r + 1] = ti.dy * S[r];
          v[4 * r + 2] = Z[r];
          v[4 * r + 3] = S[r];
        }
        v[12] = v[13] = v[14] = v[15] = 0.0f;
        const float tot = warp_reduce_scatter16(v, lane);
        const int slot = scatter_slot(lane);
        if (!(lane & 1) && slot < 12) red[warp][b][slot] = tot;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * PSLOTS; e += NT) {
      const int b = e / PSLOTS, slot = e % PSLOTS;
      float val = 0.0f;
      if (slot < 12) {
        if (any && tvs[b].mode != MODE_SKIP)
          for (int w = 0; w < NT / 32; ++w) val += red[w][b][slot];
      } else if (slot == 12) {
        val = (float)tvs[b].au;
      } else if (slot == 13) {
        val = (float)tvs[b].av;
      }
      partials[((long long)(j0 + b) * ntiles + blockIdx.x) * PSLOTS + slot] = val;
    }
  }
}

template <typename T, bool FDK, bool EXACT>
static void vjp_dispatch(const float* dvol, const void* proj, const ProjInfo& pi,
                         const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                         float* partials, cudaStream_t s) {
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  vjp_motion_kernel<ZB_VJP, T, FDK, EXACT>
      <<<ntiles, NT, 0, s>>>(dvol, (const T*)proj, pi, grad, geom, vi, partials);
}

template <typename T>
static void vjp_dispatch_t(int fdk, int exact, const float* dvol, const void* proj,
                           const ProjInfo& pi, const float2* grad, const ViewGeom* geom,
                           const VolInfo& vi, float* partials, cudaStream_t s) {
  if (fdk) {
    exact ? vjp_dispatch<T, true, true>(dvol, proj, pi, grad, geom, vi, partials, s)
          : vjp_dispatch<T, true, false>(dvol, proj, pi, grad, geom, vi, partials, s);
  } else {
    exact ? vjp_dispatch<T, false, true>(dvol, proj, pi, grad, geom, vi, partials, s)
          : vjp_dispatch<T, false, false>(dvol, proj, pi, grad, geom, vi, partials, s);
  }
}

cudaError_t launch_vjp_motion(const float* dvol, const void* proj, int dtype, const ProjInfo& pi,
                              const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                              int fdk, int exact, float* partials, cudaStream_t s) {
  if (vi.zb != ZB_VJP) return cudaErrorInvalidValue;
  if (dtype == 0)
    vjp_dispatch_t<float>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials, s);
  else if (dtype == 1)
    vjp_dispatch_t<__half>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials, s);
  else
    vjp_dispatch_t<__nv_bfloat16>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials, s);
  return cudaGetLastError();
}

// ------------------------------------------------- VJP w.r.t. the data

// Adjoint of Eq. 3 in d_j: every voxel-view scatters s = delta * c * omega
// times its four bilinear weights into a contiguous [V][nv][nu] FP32 image
// (global FP32 atomics; the caller zeroes the output first).
template <int ZB, bool FDK, bool EDGE>
__device__ __forceinline__ void proj_view(float* out, int nu, int nv, const TileView& t,
                                          float dx, float dy, const float (&delta)[ZB]) {
  float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    if (delta[k] == 0.0f) continue;
    const float dz = k - 0.5f * (ZB - 1);
    Sample s = locate<EDGE>(fmaf(dz, t.ru[2], u0), fmaf(dz, t.rv[2], v0), fmaf(dz, t.rw[2], w0),
                            t, nu, nv);
    if (EDGE && !s.ok) continue;
    const float sd = delta[k] * (FDK ? s.rwi * (s.rwi * t.wgt) : t.wgt);
    const float b1 = sd * s.tv, b0 = sd - b1;
    const float w11 = b1 * s.tu, w01 = b1 - w11, w10 = b0 * s.tu, w00 = b0 - w10;
    float* p = out + (long long)s.iv * nu + s.iu;
    if (!EDGE) {
      atomicAdd(p, w00);
      atomicAdd(p + 1, w10);
      atomicAdd(p + nu, w01);
      atomicAdd(p + nu + 1, w11);
    } else {
      bool uu0 = (unsigned)s.iu < (unsigned)nu, uu1 = (unsigned)(s.iu + 1) < (unsigned)nu;
      bool vv0 = (unsigned)s.iv < (unsigned)nv, vv1 = (unsigned)(s.iv + 1) < (unsigned)nv;
      if (uu0 && vv0) atomicAdd(p, w00);
      if (uu1 && vv0) atomicAdd(p + 1, w10);
      if (uu0 && vv1) atomicAdd(p + nu, w01);
      if (uu1 && vv1) atomicAdd(p + nu + 1, w11);
    }
  }
}

template <int ZB, bool FDK>
__global__ void __launch_bounds__(NT, 2)
    vjp_proj_kernel(const float* __restrict__ dvol, ProjInfo pi, const ViewGeom* __restrict__ geom,
                    VolInfo vi, float* __restrict__ dproj) {
  __shared__ TileView tvs[VB];
  const TileIdx ti = tile_index<ZB>(vi);
  const int i = ti.tx * TX + ti.lx, j = ti.ty * TY + ti.ly;
  float delta[ZB];
  bool nz = false;
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    const int z = ti.tz * ZB + k;
    delta[k] = (i < vi.nx && j < vi.ny && z < vi.nz)
                   ? __ldg(dvol + ((long long)z * vi.ny + j) * vi.nx + i)
                   : 0.0f;
    nz |= delta[k] != 0.0f;
  }
  if (!__syncthreads_or(nz)) return;
  for (int j0 = 0; j0 < pi.nviews; j0 += VB) {
    const int nb = min(VB, pi.nviews - j0);
    __syncthreads();
    if (threadIdx.x < nb)
      setup_tile_view(tvs[threadIdx.x], geom[j0 + threadIdx.x], ti.qc, ti.half, pi.nu, pi.nv,
                      false);
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      const TileView t = tvs[b];
      if (t.mode == MODE_SKIP) continue;
      float* out = dproj + (long long)(j0 + b) * pi.nv * pi.nu;
      if (t.mode == MODE_INTERIOR)
        proj_view<ZB, FDK, false>(out, pi.nu, pi.nv, t, ti.dx, ti.dy, delta);
      else
        proj_view<ZB, FDK, true>(out, pi.nu, pi.nv, t, ti.dx, ti.dy, delta);
    }
  }
}

cudaError_t launch_vjp_proj(const float* dvol, const ProjInfo& pi, const ViewGeom* geom,
                            const VolInfo& vi, int fdk, float* dproj, cudaStream_t s) {
  if (vi.zb != ZB_VJP) return cudaErrorInvalidValue;
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  if (fdk)
    vjp_proj_kernel<ZB_VJP, true><<<ntiles, NT, 0, s>>>(dvol, pi, geom, vi, dproj);
  else
    vjp_proj_kernel<ZB_VJP, false><<<ntiles, NT, 0, s>>>(dvol, pi, geom, vi, dproj);
  return cudaGetLastError();
}

}  // namespace bpk
