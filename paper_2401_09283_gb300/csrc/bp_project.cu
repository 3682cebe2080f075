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

// CTAs per SM the register budget is sized for (256 threads each).
#ifndef BP_FWD_MINB
#define BP_FWD_MINB 4
#endif
#ifndef BP_VJP_MINB
#define BP_VJP_MINB 3
#endif
constexpr int FWD_MINB = BP_FWD_MINB;
constexpr int VJP_MINB = BP_VJP_MINB;

constexpr float MAGIC = 12582912.0f;   // 1.5 * 2^23
constexpr int MAGIC_BITS = 0x4B400000;

// Footprint staging buffers: fixed row pitch (so tap offsets are
// immediates), rows of 21 16-byte chunks, 64 rows.  (A pitch of 80 floats,
// which a simulation of the c2 tap positions gave 3 % fewer bank-conflict
// wavefronts, measured the same: c2 step 19.448 against 19.445 ms.)
#ifndef BP_STAGE_PITCH_BYTES
#define BP_STAGE_PITCH_BYTES 336
#endif
constexpr int STAGE_PITCH_BYTES = BP_STAGE_PITCH_BYTES;
constexpr int STAGE_ROWS = 64;
constexpr int STAGE_BYTES = STAGE_PITCH_BYTES * STAGE_ROWS;
template <typename T>
struct StageGeom {
  static constexpr int CH = 16 / (int)sizeof(T);                // elements per chunk
  static constexpr int P = STAGE_PITCH_BYTES / (int)sizeof(T);  // row pitch in elements
};
// FP16/BF16 data staged with conversion: raw rows of 16-byte chunks (8
// pixels) at a pitch of CONV_P elements are converted into an FP32 buffer of
// the same pitch (in floats), which the sample loops read like FP32 data.
constexpr int CONV_P = 88;
struct ConvGeom {
  static constexpr int CH = 8;
  static constexpr int P = CONV_P;
};
constexpr int CONV_F_BYTES = CONV_P * STAGE_ROWS * 4;  // FP32 buffer
constexpr int CONV_R_BYTES = CONV_P * STAGE_ROWS * 2;  // raw buffer

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

// Packed FP32 pairs (Blackwell f32x2 instructions): two voxels' values in
// one 64-bit register, one instruction per pair.  Each element is rounded
// exactly like the scalar instruction, so packed and scalar code give
// identical results; the packing halves the issue slots of the FP32 work.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void up2(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 add2_rd(f2 a, f2 b) {  // rounded toward -inf
  f2 r;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// ------------------------------------------------------------ bounds check
// Debug builds (-DBP_BOUNDS_CHECK) check every staged, gathered and
// scattered index against the range it must lie in.  A failed check sets a
// bit in a device flag word, records the first failure, and redirects the
// access to a safe in-range position (the result is then wrong but nothing
// outside the buffers is touched); the host reads the word through
// bp_bounds_check.  Release builds compile the checks out.
enum { BC_STAGED_TAP = 0, BC_GLOBAL_TAP = 1, BC_SCATTER = 2, BC_STAGE_DST = 3, BC_SELFTEST = 7 };
#ifdef BP_BOUNDS_CHECK
__device__ unsigned int g_bc_flags;
__device__ unsigned long long g_bc_first;
__device__ __noinline__ void bc_fail(unsigned code, int a, int b) {
  atomicOr(&g_bc_flags, 1u << code);
  const unsigned long long rec = (1ull << 63) | ((unsigned long long)code << 56) |
                                 ((unsigned long long)(a & 0x0fffffff) << 28) |
                                 (unsigned long long)(b & 0x0fffffff);
  atomicCAS(&g_bc_first, 0ull, rec);
}
__global__ void bc_selftest_kernel() { bc_fail(BC_SELFTEST, 7, 9); }
#endif

cudaError_t bounds_status(unsigned* flags, long long* first, int op, cudaStream_t s) {
#ifdef BP_BOUNDS_CHECK
  if (op == 2) {
    bc_selftest_kernel<<<1, 1, 0, s>>>();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  unsigned long long f = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(flags, g_bc_flags, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, g_bc_first, sizeof(f));
  *first = (long long)(f & ~(1ull << 63)) | (f ? 0 : -1LL);
  if (e == cudaSuccess && op == 1) {
    const unsigned z = 0;
    const unsigned long long z64 = 0;
    e = cudaMemcpyToSymbol(g_bc_flags, &z, sizeof(z));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bc_first, &z64, sizeof(z64));
  }
  return e;
#else
  (void)flags;
  (void)first;
  (void)op;
  (void)s;
  return cudaErrorNotSupported;
#endif
}

// Unchecked global gathers and scatters (INTERIOR tiles) need both tap
// columns and rows on the detector.
__device__ __forceinline__ void bc_interior(int code, int& iu, int& iv, int nu, int nv) {
#ifdef BP_BOUNDS_CHECK
  if (!((unsigned)iu < (unsigned)(nu - 1) && (unsigned)iv < (unsigned)(nv - 1))) {
    bc_fail(code, iu, iv);
    iu = 0;
    iv = 0;
  }
#else
  (void)code;
  (void)iu;
  (void)iv;
  (void)nu;
  (void)nv;
#endif
}

// ------------------------------------------------------------ tile set-up

struct TileIdx {
  int tx, ty, tz, lx, ly;
  float dx, dy;
  double qc[3];
  float half[3];
};

template <int ZB>
__device__ __forceinline__ TileIdx tile_index(const VolInfo& vi, int tile) {
  TileIdx ti;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  ti.lx = (warp & 1) * 8 + (lane & 7);
  ti.ly = (warp >> 1) * 4 + (lane >> 3);
  ti.tx = tile % vi.tiles_x;
  ti.ty = (tile / vi.tiles_x) % vi.tiles_y;
  ti.tz = tile / (vi.tiles_x * vi.tiles_y);
  ti.dx = ti.lx - 0.5f * (TX - 1);
  ti.dy = ti.ly - 0.5f * (TY - 1);
  ti.qc[0] = ti.tx * TX + 0.5 * (TX - 1) - vi.cx;
  ti.qc[1] = ti.ty * TY + 0.5 * (TY - 1) - vi.cy;
  ti.qc[2] = ti.tz * ZB + 0.5 * (ZB - 1) - vi.cz;
  ti.half[0] = 0.5f * (TX - 1);
  ti.half[1] = 0.5f * (TY - 1);
  ti.half[2] = 0.5f * (ZB - 1);
  return ti;
}

// Cooperative set-up of the records of views j0 .. j0+nb-1 (nb <= 32) for
// this CTA's box; every thread of the CTA must call it.  Eight lanes serve
// one view; lane c evaluates box corner c.  FP64 is used only where the
// precision matters -- the projection (uc, vc, wc) of the tile centre and
// the anchored values U0 = uc - au wc, V0 = vc - av wc; the anchor pixel
// itself only has to be near the projection and comes from FP32.  The
// corners are evaluated in FP32 in the anchored frame (errors ~1e-5 px,
// far below the 0.01 px classification margin): u/w and v/w are
// linear-fractional in the voxel position, so over a box with w > 0 their
// extremes are at the corners, and the box is
//   SKIP      every sample is 0 (projection at or beyond -1 / n),
//   INTERIOR  every tap (floor and floor+1) lies on the detector,
//   EDGE      otherwise (clamped coordinates, checked taps).
// The footprint is the clipped pixel rectangle that the box's taps can
// touch (unbounded, fw = 0, when some corner has w <= 0).
//
// With STAGE, bounded boxes also get a staging plan: the rectangle of
// detector pixels that any tap (plus `halo` pixels each side) can read,
// NOT clipped to the detector (off-detector pixels are staged as zeros, so
// the sample loop needs neither checks nor clamps), if it fits the buffer.
// With `need_csafe` only central-safe boxes are staged.
template <typename T, bool STAGE, class G = StageGeom<T>>
__device__ void setup_batch(TileView* tvs, const ViewGeom* __restrict__ geom, int j0, int nb,
                            const TileIdx& ti, int nu, int nv, bool with_scale, int halo = 0,
                            bool need_csafe = false) {
  const int b = threadIdx.x >> 3, c = threadIdx.x & 7;
  const ViewGeom& g = geom[j0 + min(b, nb - 1)];
  const double* M = g.P;
  const double uc = fma(M[0], ti.qc[0], fma(M[1], ti.qc[1], fma(M[2], ti.qc[2], M[3])));
  const double vc = fma(M[4], ti.qc[0], fma(M[5], ti.qc[1], fma(M[6], ti.qc[2], M[7])));
  const double wc = fma(M[8], ti.qc[0], fma(M[9], ti.qc[1], fma(M[10], ti.qc[2], M[11])));
  int au = 0, av = 0;
  if (wc > 0.0) {
    const float wf = (float)wc;
    const float a = fminf(fmaxf(floorf((float)uc / wf), -1048576.0f), 1048576.0f);
    const float bq = fminf(fmaxf(floorf((float)vc / wf), -1048576.0f), 1048576.0f);
    au = (int)a;
    av = (int)bq;
  }
  TileView t;
  t.U0 = (float)fma(-(double)au, wc, uc);
  t.V0 = (float)fma(-(double)av, wc, vc);
  t.W0 = (float)wc;
  const float fau = (float)au, fav = (float)av;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float m2 = (float)M[8 + k];
    t.ru[k] = fmaf(-fau, m2, (float)M[k]);
    t.rv[k] = fmaf(-fav, m2, (float)M[4 + k]);
    t.rw[k] = m2;
  }
  t.au = au;
  t.av = av;
  t.wgt = (float)(with_scale ? g.wgt * g.scale : g.wgt);
  t.wgtd = (float)g.wgt;
  // this lane's corner
  const float d0 = (c & 1) ? ti.half[0] : -ti.half[0];
  const float d1 = (c & 2) ? ti.half[1] : -ti.half[1];
  const float d2 = (c & 4) ? ti.half[2] : -ti.half[2];
  const float w = fmaf(t.rw[2], d2, fmaf(t.rw[1], d1, fmaf(t.rw[0], d0, t.W0)));
  const float u = fmaf(t.ru[2], d2, fmaf(t.ru[1], d1, fmaf(t.ru[0], d0, t.U0)));
  const float v = fmaf(t.rv[2], d2, fmaf(t.rv[1], d1, fmaf(t.rv[0], d0, t.V0)));
  const bool pos = w > 0.0f;
  int npos = pos ? 1 : 0;
  float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  if (pos) {
    xmin = xmax = u / w;
    ymin = ymax = v / w;
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    npos += __shfl_xor_sync(0xffffffffu, npos, o);
    xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
    ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
  }
  if (c != 0 || b >= nb) return;
  const float m = 0.01f;
  // detector [0, n-1] in the anchored frame
  const float ulo = -fau, uhi = (float)(nu - 1) - fau, vlo = -fav, vhi = (float)(nv - 1) - fav;
  t.fu0 = t.fv0 = t.fw = t.fh = 0;
  t.csafe = 0;
  t.sx0 = t.sv0 = t.sh = t.scpr = t.srpp = t.smag = t.soff = t.staged = 0;
  if (npos == 0) {
    t.mode = MODE_SKIP;
  } else if (npos < 8) {
    t.mode = MODE_EDGE;
  } else if (xmax <= ulo - 1.0f - m || xmin >= uhi + 1.0f + m || ymax <= vlo - 1.0f - m ||
             ymin >= vhi + 1.0f + m) {
    t.mode = MODE_SKIP;
  } else {
    t.mode = (xmin >= ulo + m && xmax <= uhi - m && ymin >= vlo + m && ymax <= vhi - m)
                 ? MODE_INTERIOR
                 : MODE_EDGE;
    // central differences at the tap pixels use interior neighbours only:
    // taps in [1, n-2], i.e. floor in [1, n-3]
    t.csafe = xmin >= ulo + 1.0f + m && xmax <= uhi - 1.0f - m && ymin >= vlo + 1.0f + m &&
              ymax <= vhi - 1.0f - m;
    const int fl_u0 = (int)floorf(xmin - m) + au, fl_u1 = (int)floorf(xmax + m) + 1 + au;
    const int fl_v0 = (int)floorf(ymin - m) + av, fl_v1 = (int)floorf(ymax + m) + 1 + av;
    const int u0 = max(fl_u0, 0), u1 = min(fl_u1, nu - 1);
    const int v0 = max(fl_v0, 0), v1 = min(fl_v1, nv - 1);
    if (u1 >= u0 && v1 >= v0) {
      t.fu0 = u0;
      t.fv0 = v0;
      t.fw = u1 - u0 + 1;
      t.fh = v1 - v0 + 1;
    }
    if (STAGE && t.mode != MODE_SKIP && (!need_csafe || t.csafe)) {
      constexpr int CH = G::CH, P = G::P;
      const int x0 = (fl_u0 - halo) & ~(CH - 1);  // floor to a chunk boundary
      const int y0 = fl_v0 - halo;
      const int cpr = (fl_u1 + halo - x0) / CH + 1;
      const int h = fl_v1 + halo - y0 + 1;
      if (cpr * CH <= P && h <= STAGE_ROWS) {
        t.staged = 1;
        t.sx0 = x0;
        t.sv0 = y0;
        t.sh = h;
        t.scpr = cpr;
        t.srpp = 32 / cpr;
        t.smag = (65536 + cpr - 1) / cpr;
        t.soff = (int)((unsigned)(av - y0) * (unsigned)P - (unsigned)MAGIC_BITS * (unsigned)P +
                       (unsigned)(au - x0) - (unsigned)MAGIC_BITS);
      }
    }
  }
  tvs[b] = t;
}

// Detector position of one voxel in the anchored frame.
struct Sample {
  float rwi;     // 1/w
  float x, y;    // u/w - au, v/w - av (clamped in EDGE mode)
  float tu, tv;  // fractional parts
  int iu, iv;    // absolute floor pixel
  int bx, by;    // bit patterns of x + MAGIC, y + MAGIC (rounded down)
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
  s.bx = __float_as_int(rx);
  s.by = __float_as_int(ry);
  s.iu = s.bx - MAGIC_BITS + t.au;
  s.iv = s.by - MAGIC_BITS + t.av;
  s.x = x;
  s.y = y;
  return s;
}

// Four taps of a [nv][rs] image at (iu..iu+1, iv..iv+1), zero outside.
template <bool EDGE, typename T>
__device__ __forceinline__ void taps(const T* img, long long rs, int nu, int nv, const Sample& s,
                                     float& d00, float& d10, float& d01, float& d11) {
  if (!EDGE) {
    int iu = s.iu, iv = s.iv;
    bc_interior(BC_GLOBAL_TAP, iu, iv, nu, nv);
    const T* p = img + (long long)iv * rs + iu;
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

__device__ __forceinline__ f2 bilerp2(f2 tu, f2 tv, f2 d00, f2 d10, f2 d01, f2 d11) {
  const f2 top = fma2(tu, sub2(d10, d00), d00);
  const f2 bot = fma2(tu, sub2(d11, d01), d01);
  return fma2(tv, sub2(bot, top), top);
}

// ------------------------------------------------------ footprint staging

// Each (tile, view) reads a small rectangle of one detector image (the tile
// footprint from the set-up).  Voxels project ~2.6 px apart on the larger
// detectors, so a warp's 32 taps of one load are scattered over 4-6 L1
// lines; from shared memory the same taps are a single wavefront (bar bank
// conflicts).  The footprint is therefore copied to shared memory with
// cp.async in 16-byte chunks, one view ahead: the copy of view j+1 overlaps
// the arithmetic of view j.  Footprints that do not fit the buffer, or are
// unbounded, read global memory instead.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// All threads: copy the staged rectangle of record t (rows per warp pass,
// one chunk per lane, no divisions).  A chunk lies wholly on or off the
// detector (chunk starts are multiples of CH and nu is), so off-detector
// chunks and rows are written as zeros.
template <typename T, int P = StageGeom<T>::P>
__device__ __forceinline__ void stage_issue(T* buf, const T* img, long long rs, int nu, int nv,
                                            const TileView& t) {
  constexpr int CH = StageGeom<T>::CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = (lane * t.smag) >> 16, lc = lane - lr * t.scpr;
  if (lr >= t.srpp) return;
  const int cu = t.sx0 + lc * CH;
  const bool uin = cu >= 0 && cu < nu;
  for (int r = warp * t.srpp + lr; r < t.sh; r += (NT / 32) * t.srpp) {
#ifdef BP_BOUNDS_CHECK
    if (!(r < STAGE_ROWS && lc * CH + CH <= P)) {
      bc_fail(BC_STAGE_DST, r, lc);
      break;
    }
#endif
    T* dst = buf + r * P + lc * CH;
    const int row = t.sv0 + r;
    if (uin && (unsigned)row < (unsigned)nv)
      cp_async16(dst, img + (long long)row * rs + cu);
    else
      *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// All threads: convert the raw FP16/BF16 rectangle of record t (staged by
// stage_issue<T, CONV_P>) into FP32 at the same pitch, chunk by chunk with the
// copy's thread mapping.
template <typename T>
__device__ __forceinline__ void convert_stage(float* F, const T* R, const TileView& t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lr = (lane * t.smag) >> 16, lc = lane - lr * t.scpr;
  if (lr >= t.srpp) return;
  for (int r = warp * t.srpp + lr; r < t.sh; r += (NT / 32) * t.srpp) {
    const uint4 w = *reinterpret_cast<const uint4*>(R + r * CONV_P + lc * 8);
    const unsigned ws[4] = {w.x, w.y, w.z, w.w};
    float f[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (std::is_same<T, __half>::value) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&ws[q]));
        f[2 * q] = v.x;
        f[2 * q + 1] = v.y;
      } else {
        f[2 * q] = __uint_as_float(ws[q] << 16);
        f[2 * q + 1] = __uint_as_float(ws[q] & 0xffff0000u);
      }
    }
    float4* d = reinterpret_cast<float4*>(F + r * CONV_P + lc * 8);
    d[0] = make_float4(f[0], f[1], f[2], f[3]);
    d[1] = make_float4(f[4], f[5], f[6], f[7]);
  }
}

__device__ __forceinline__ void cp_async_wait0() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ float tof(T x);
template <>
__device__ __forceinline__ float tof<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ float tof<__half>(__half x) {
  return __half2float(x);
}
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// A sample's position in the staged buffer: (bx, by) are the bit patterns
// of x + MAGIC and y + MAGIC rounded down, i.e. MAGIC_BITS + floor.
// H is the stencil's reach beyond the bilinear taps (1 for the CENTRAL
// 4x4-minus-corners stencil, 0 otherwise); the staging plan covers it.
template <int P, int H = 0, typename T>
__device__ __forceinline__ const T* staged_tap(const T* buf, const TileView& t, int bx, int by) {
#ifdef BP_BOUNDS_CHECK
  constexpr int CHK = (P == CONV_P) ? 8 : 16 / (int)sizeof(T);  // elements per staged chunk
  const int ru = bx - MAGIC_BITS + t.au - t.sx0, rv = by - MAGIC_BITS + t.av - t.sv0;
  if (!(t.staged && ru - H >= 0 && ru + 1 + H < t.scpr * CHK && rv - H >= 0 &&
        rv + 1 + H < t.sh)) {
    bc_fail(BC_STAGED_TAP, ru, rv);
    bx = MAGIC_BITS + t.sx0 + H - t.au;
    by = MAGIC_BITS + t.sv0 + H - t.av;
  }
#endif
  const unsigned o = (unsigned)by * (unsigned)P + (unsigned)bx + (unsigned)t.soff;
  return buf + (int)o;
}



// ------------------------------------------------------------------ forward

// One view from global memory (footprint not staged).
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

// One view from its staged, zero-padded footprint (no checks, no clamps, tap
// offsets are compile-time constants), with packed pairs of voxels (k, k+1):
// every step of the scalar loop above, in the same order, on f32x2 pairs.
// E is the staged element type, P the staged row pitch.
template <int ZB, typename T, bool FDK, int P = StageGeom<T>::P>
__device__ __forceinline__ void forward_view_staged2(const T* buf, const TileView& t, float dx,
                                                     float dy, f2 (&acc)[ZB / 2]) {
  const float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  const float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  const float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
  const f2 U0 = pk2(u0, u0), V0 = pk2(v0, v0), W0 = pk2(w0, w0);
  const f2 RU = pk2(t.ru[2], t.ru[2]), RV = pk2(t.rv[2], t.rv[2]), RW = pk2(t.rw[2], t.rw[2]);
  const f2 M2 = pk2(MAGIC, MAGIC), TWO = pk2(2.0f, 2.0f), WG = pk2(t.wgt, t.wgt);
  f2 dz = pk2(-0.5f * (ZB - 1), 1.0f - 0.5f * (ZB - 1));  // exact: halves of small integers
#pragma unroll
  for (int p = 0; p < ZB / 2; ++p) {
    if (p) dz = add2(dz, TWO);
    const f2 u = fma2(dz, RU, U0), v = fma2(dz, RV, V0), w = fma2(dz, RW, W0);
    float wl, wh;
    up2(w, wl, wh);
    const f2 r = pk2(rcp_approx(wl), rcp_approx(wh));
    const f2 x = mul2(u, r), y = mul2(v, r);
    const f2 rx = add2_rd(x, M2), ry = add2_rd(y, M2);
    const f2 tu = sub2(x, sub2(rx, M2)), tv = sub2(y, sub2(ry, M2));
    float bxl, bxh, byl, byh;
    up2(rx, bxl, bxh);
    up2(ry, byl, byh);
    const T* ql = staged_tap<P>(buf, t, __float_as_int(bxl), __float_as_int(byl));
    const T* qh = staged_tap<P>(buf, t, __float_as_int(bxh), __float_as_int(byh));
    const f2 d00 = pk2(tof(ql[0]), tof(qh[0])), d10 = pk2(tof(ql[1]), tof(qh[1]));
    const f2 d01 = pk2(tof(ql[P]), tof(qh[P])), d11 = pk2(tof(ql[P + 1]), tof(qh[P + 1]));
    const f2 val = bilerp2(tu, tv, d00, d10, d01, d11);
    acc[p] = fma2(val, FDK ? mul2(r, mul2(r, WG)) : WG, acc[p]);
  }
}

// Views are processed in order; the records of batch k+1 are built at the
// start of batch k (two record slots), so the footprint of view j+1 is
// known, and its copy issued, while view j is computed.  With two staging
// buffers a second barrier per view guards their reuse; with three it is
// not needed (the copy into buffer (j+1) mod 3 cannot overlap a read of it:
// view j-2 was finished by every thread before the barrier of view j-1),
// but the third buffer costs occupancy: two buffers at 4 CTAs/SM measured
// faster on GB300 than three at 3 CTAs/SM.
#ifndef BP_FWD_NBUF
#define BP_FWD_NBUF 2
#endif
constexpr int FWD_NBUF = BP_FWD_NBUF;

//
// FP16/BF16 data (CONV) is staged through a raw buffer and converted once per
// (tile, view) into an FP32 buffer, so the sample loop is the FP32 one
// (no conversion per tap): wait for the raw copy of view j, barrier, convert,
// barrier, issue the raw copy of view j+1, compute view j.
template <typename T>
__host__ __device__ constexpr bool conv_staging() {
  return !std::is_same<T, float>::value;
}
template <typename T>
__host__ __device__ constexpr int fwd_smem_bytes() {
  return conv_staging<T>() ? CONV_F_BYTES + CONV_R_BYTES : FWD_NBUF * STAGE_BYTES;
}

// One tile of the forward: every view, in order, accumulated per voxel.
// All threads of the CTA call it; tvs and dyn_smem are the CTA's shared
// memory (the kernel's static record slots and dynamic staging buffers).
template <int ZB, typename T, bool FDK, bool STAGE>
__device__ __forceinline__ void forward_tile(const T* __restrict__ proj, const ProjInfo& pi,
                                             const ViewGeom* __restrict__ geom, const VolInfo& vi,
                                             float* __restrict__ vol, int tile,
                                             TileView (*tvs)[VB], unsigned char* dyn_smem) {
  constexpr bool CONV = STAGE && conv_staging<T>();
  using G = typename std::conditional<CONV, ConvGeom, StageGeom<T>>::type;
  T* bufs = reinterpret_cast<T*>(dyn_smem);  // plain: FWD_NBUF buffers of T
  float* F = reinterpret_cast<float*>(dyn_smem);  // CONV: FP32 buffer, then the raw one
  T* R = reinterpret_cast<T*>(dyn_smem + CONV_F_BYTES);
  constexpr int CAP = STAGE_BYTES / (int)sizeof(T);
  static_assert(ZB % 2 == 0, "voxel pairs");
  const TileIdx ti = tile_index<ZB>(vi, tile);
  f2 acc[ZB / 2];
#pragma unroll
  for (int k = 0; k < ZB / 2; ++k) acc[k] = pk2(0.0f, 0.0f);
  const int V = pi.nviews;
  const int nbatch = (V + VB - 1) / VB;
  setup_batch<T, STAGE, G>(tvs[0], geom, 0, min(VB, V), ti, pi.nu, pi.nv, true);
  if (nbatch > 1)
    setup_batch<T, STAGE, G>(tvs[1], geom, VB, min(VB, V - VB), ti, pi.nu, pi.nv, true);
  __syncthreads();
  if (STAGE && V > 0 && tvs[0][0].staged) {
    if constexpr (CONV)
      stage_issue<T, CONV_P>(R, proj, pi.rs, pi.nu, pi.nv, tvs[0][0]);
    else
      stage_issue(bufs, proj, pi.rs, pi.nu, pi.nv, tvs[0][0]);
  }
  cp_async_commit();
  int cur = 0;  // buffer of view v
  for (int v = 0; v < V; ++v) {
    const int k = v / VB, b = v - k * VB;
    if (b == 0 && k >= 1 && k + 1 < nbatch) {
      setup_batch<T, STAGE, G>(tvs[(k + 1) & 1], geom, (k + 1) * VB, min(VB, V - (k + 1) * VB),
                               ti, pi.nu, pi.nv, true);
      __syncthreads();
    }
    const TileView t = tvs[k & 1][b];
    const int nxt = cur == FWD_NBUF - 1 ? 0 : cur + 1;
    const int kn = (v + 1) / VB;
    const TileView* tn = v + 1 < V ? &tvs[kn & 1][v + 1 - kn * VB] : nullptr;
    if constexpr (CONV) {
      cp_async_wait0();
      __syncthreads();  // raw view v complete; every thread is done with F
      if (t.staged) convert_stage<T>(F, R, t);
      __syncthreads();  // F holds view v; R is free
      if (tn && tn->staged)
        stage_issue<T, CONV_P>(R, proj + (long long)(v + 1) * pi.vs, pi.rs, pi.nu, pi.nv, *tn);
      cp_async_commit();
    } else {
      if (STAGE && tn && tn->staged)
        stage_issue(bufs + nxt * CAP, proj + (long long)(v + 1) * pi.vs, pi.rs, pi.nu, pi.nv, *tn);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();
    }
    if (t.mode != MODE_SKIP) {
      if (STAGE && t.staged) {
        if constexpr (CONV)
          forward_view_staged2<ZB, float, FDK, CONV_P>(F, t, ti.dx, ti.dy, acc);
        else
          forward_view_staged2<ZB, T, FDK>(bufs + cur * CAP, t, ti.dx, ti.dy, acc);
      } else {
        const T* img = proj + (long long)v * pi.vs;
        float a[ZB];
#pragma unroll
        for (int k = 0; k < ZB / 2; ++k) up2(acc[k], a[2 * k], a[2 * k + 1]);
        if (t.mode == MODE_INTERIOR)
          forward_view<ZB, T, FDK, false>(img, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, a);
        else
          forward_view<ZB, T, FDK, true>(img, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, a);
#pragma unroll
        for (int k = 0; k < ZB / 2; ++k) acc[k] = pk2(a[2 * k], a[2 * k + 1]);
      }
    }
    if (!CONV && FWD_NBUF == 2) __syncthreads();
    cur = nxt;
  }
  const int i = ti.tx * TX + ti.lx, j = ti.ty * TY + ti.ly;
  if (i < vi.nx && j < vi.ny) {
#pragma unroll
    for (int k = 0; k < ZB / 2; ++k) {
      float lo, hi;
      up2(acc[k], lo, hi);
      const int z = ti.tz * ZB + 2 * k;
      if (z < vi.nz) vol[((long long)z * vi.ny + j) * vi.nx + i] = lo;
      if (z + 1 < vi.nz) vol[((long long)(z + 1) * vi.ny + j) * vi.nx + i] = hi;
    }
  }
}

template <int ZB, typename T, bool FDK, bool STAGE>
__global__ void __launch_bounds__(NT, FWD_MINB)
    forward_kernel(const T* __restrict__ proj, ProjInfo pi, const ViewGeom* __restrict__ geom,
                   VolInfo vi, float* __restrict__ vol) {
  __shared__ TileView tvs[2][VB];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  forward_tile<ZB, T, FDK, STAGE>(proj, pi, geom, vi, vol, blockIdx.x, tvs, dyn_smem);
}

// z-extent of the forward's tiles (its own tiling; the VJP's is ZB_VJP)
#ifndef BP_ZB_FWD
#define BP_ZB_FWD 16
#endif
#ifndef BP_FWD_STAGE
#define BP_FWD_STAGE 1
#endif
constexpr int ZB_FWD = BP_ZB_FWD;

// Staging needs 16-byte aligned rows and whole 16-byte chunks per row.
template <typename T>
static bool stageable(const void* proj, const ProjInfo& pi) {
  const long long es = (long long)sizeof(T), ch = 16 / es;
  return ((reinterpret_cast<uintptr_t>(proj) & 15) == 0) && (pi.rs * es) % 16 == 0 &&
         (pi.vs * es) % 16 == 0 && pi.nu % ch == 0;
}

// Opt a kernel into more than 48 KiB of dynamic shared memory, once per
// device (so that later launches -- including ones being captured into a
// CUDA graph -- make no attribute call).
template <auto Kernel>
static cudaError_t smem_attr_once(int bytes) {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

template <typename T, bool FDK>
static cudaError_t forward_dispatch(const void* proj, const ProjInfo& pi, const ViewGeom* geom,
                                    const VolInfo& vi, float* vol, cudaStream_t s) {
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const int smem = fwd_smem_bytes<T>();
  if (BP_FWD_STAGE && stageable<T>(proj, pi)) {
    cudaError_t e = smem_attr_once<forward_kernel<ZB_FWD, T, FDK, true>>(smem);
    if (e != cudaSuccess) return e;
    forward_kernel<ZB_FWD, T, FDK, true><<<ntiles, NT, smem, s>>>((const T*)proj, pi, geom, vi, vol);
  } else {
    forward_kernel<ZB_FWD, T, FDK, false><<<ntiles, NT, 0, s>>>((const T*)proj, pi, geom, vi, vol);
  }
  return cudaGetLastError();
}

cudaError_t prepare_forward(int dtype, int fdk) {
  if (dtype == 0)
    return fdk ? smem_attr_once<forward_kernel<ZB_FWD, float, true, true>>(fwd_smem_bytes<float>())
               : smem_attr_once<forward_kernel<ZB_FWD, float, false, true>>(fwd_smem_bytes<float>());
  if (dtype == 1)
    return fdk ? smem_attr_once<forward_kernel<ZB_FWD, __half, true, true>>(fwd_smem_bytes<__half>())
               : smem_attr_once<forward_kernel<ZB_FWD, __half, false, true>>(fwd_smem_bytes<__half>());
  constexpr int sb = fwd_smem_bytes<__nv_bfloat16>();
  return fdk ? smem_attr_once<forward_kernel<ZB_FWD, __nv_bfloat16, true, true>>(sb)
             : smem_attr_once<forward_kernel<ZB_FWD, __nv_bfloat16, false, true>>(sb);
}

cudaError_t launch_forward(const void* proj, int dtype, const ProjInfo& pi, const ViewGeom* geom,
                           const VolInfo& vi_in, int fdk, float* vol, cudaStream_t s) {
  VolInfo vi = vi_in;  // the forward tiles z by ZB_FWD
  vi.zb = ZB_FWD;
  vi.tiles_z = (vi.nz + ZB_FWD - 1) / ZB_FWD;
  if (dtype == 0)
    return fdk ? forward_dispatch<float, true>(proj, pi, geom, vi, vol, s)
               : forward_dispatch<float, false>(proj, pi, geom, vi, vol, s);
  if (dtype == 1)
    return fdk ? forward_dispatch<__half, true>(proj, pi, geom, vi, vol, s)
               : forward_dispatch<__half, false>(proj, pi, geom, vi, vol, s);
  return fdk ? forward_dispatch<__nv_bfloat16, true>(proj, pi, geom, vi, vol, s)
             : forward_dispatch<__nv_bfloat16, false>(proj, pi, geom, vi, vol, s);
}

// ------------------------------------------------------- gradient images

// g_u, g_v of one view in value per pixel: (d[+1] - d[-1]) / 2 inside,
// one-sided first differences on the two edge pixels (Sec. II-B.2), in
// stored units (the per-view dequantisation scale is applied with the view
// weight); output contiguous [V][nv][nu] float2.
template <typename T>
__global__ void __launch_bounds__(256) grad_images_kernel(const T* __restrict__ proj, ProjInfo pi,
                                                         float2* __restrict__ grad) {
  // one CTA per detector row (view j, row b); consecutive threads take
  // consecutive columns (measured on c2: 0.29 ms against 0.37 ms for a flat
  // grid-stride loop with 64-bit index divisions, 0.30 ms for CTAs looping
  // over rows)
  const long long rowi = blockIdx.x;
  const int j = (int)(rowi / pi.nv), b = (int)(rowi - (long long)j * pi.nv);
  const T* row = proj + (long long)j * pi.vs + (long long)b * pi.rs;
  float2* out = grad + rowi * pi.nu;
  for (int a = threadIdx.x; a < pi.nu; a += blockDim.x) {
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
    out[a] = make_float2(gu, gv);
  }
}

cudaError_t launch_grad_images(const void* proj, int dtype, const ProjInfo& pi, float2* grad,
                               cudaStream_t s) {
  const long long nb = (long long)pi.nviews * pi.nv;  // detector rows
  if (nb == 0 || pi.nu == 0) return cudaSuccess;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (dtype == 0)
    grad_images_kernel<float><<<(int)nb, 256, 0, s>>>((const float*)proj, pi, grad);
  else if (dtype == 1)
    grad_images_kernel<__half><<<(int)nb, 256, 0, s>>>((const __half*)proj, pi, grad);
  else
    grad_images_kernel<__nv_bfloat16>
        <<<(int)nb, 256, 0, s>>>((const __nv_bfloat16*)proj, pi, grad);
  return cudaGetLastError();
}

// ----------------------------------------------- block image (fused data VJP)

// The fused data VJP of interior tiles adds a sample's four bilinear weights
// with ONE 16-byte vector reduction instead of four scalar ones, into a block
// image: entry (r, c) holds the 2x2 pixel block with top-left pixel (r, c) as
// 4 consecutive floats, (r,c), (r,c+1), (r+1,c), (r+1,c+1), so a sample whose
// floor pixel is (iu, iv) adds to entry iv*nu + iu, a 16-byte aligned
// address with the same index arithmetic as the pixel itself.
// block_combine_kernel adds the blocks into dL/dproj afterwards (pixel (r, c)
// is element (dr, dc) of the entries (r-dr, c-dc)).
#ifndef BP_VJP_BLOCKS
#define BP_VJP_BLOCKS 1
#endif

__device__ __forceinline__ void red_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

// dproj[v][r][c] += the four block entries covering pixel (r, c): element 0
// of (r, c), 1 of (r, c-1), 2 of (r-1, c), 3 of (r-1, c-1).  One CTA per
// detector row.
__global__ void __launch_bounds__(256) block_combine_kernel(const float* __restrict__ blk,
                                                           float* __restrict__ dproj, int nv,
                                                           int nu) {
  const long long row = blockIdx.x;  // v * nv + r
  const bool up = row % nv != 0;
  const float* q0 = blk + row * nu * 4;
  const float* q1 = q0 - (long long)nu * 4;
  float* out = dproj + row * nu;
  for (int c = threadIdx.x; c < nu; c += blockDim.x) {
    float acc = __ldg(q0 + 4 * c);
    if (c > 0) acc += __ldg(q0 + 4 * (c - 1) + 1);
    if (up) {
      acc += __ldg(q1 + 4 * c + 2);
      if (c > 0) acc += __ldg(q1 + 4 * (c - 1) + 3);
    }
    out[c] += acc;
  }
}

long long block_image_floats(const ProjInfo& pi) {
  if (!BP_VJP_BLOCKS) return 0;
  return (long long)pi.nviews * pi.nv * pi.nu * 4;
}

cudaError_t launch_block_combine(const float* blk, const ProjInfo& pi, float* dproj,
                                cudaStream_t s) {
  const long long rows = (long long)pi.nviews * pi.nv;
  if (rows <= 0 || pi.nu <= 0) return cudaSuccess;
  if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;
  block_combine_kernel<<<(unsigned)rows, 256, 0, s>>>(blk, dproj, pi.nv, pi.nu);
  return cudaGetLastError();
}

// Four bilinear-weighted scatter-adds of one sample into a [nv][nu] image
// (global FP32 atomics; taps off the detector are dropped in EDGE mode).
// With a block image bout (see below), a sample whose four taps lie on the
// detector adds them with one vector reduction there instead.
template <bool EDGE>
__device__ __forceinline__ void scatter_sample(float* out, float* bout, int nu, int nv,
                                               const Sample& s, float sd) {
  const float b1 = sd * s.tv, b0 = sd - b1;
  const float w11 = b1 * s.tu, w01 = b1 - w11, w10 = b0 * s.tu, w00 = b0 - w10;
  if (!EDGE) {
    int iu = s.iu, iv = s.iv;
    bc_interior(BC_SCATTER, iu, iv, nu, nv);
    if (BP_VJP_BLOCKS && bout) {
      red_v4(bout + 4 * ((long long)iv * nu + iu), w00, w10, w01, w11);
      return;
    }
    float* p = out + (long long)iv * nu + iu;
    atomicAdd(p, w00);
    atomicAdd(p + 1, w10);
    atomicAdd(p + nu, w01);
    atomicAdd(p + nu + 1, w11);
  } else {
    float* p = out + (long long)s.iv * nu + s.iu;
    const bool uu0 = (unsigned)s.iu < (unsigned)nu, uu1 = (unsigned)(s.iu + 1) < (unsigned)nu;
    const bool vv0 = (unsigned)s.iv < (unsigned)nv, vv1 = (unsigned)(s.iv + 1) < (unsigned)nv;
    if (BP_VJP_BLOCKS && bout && uu0 && uu1 && vv0 && vv1) {
      red_v4(bout + 4 * ((long long)s.iv * nu + s.iu), w00, w10, w01, w11);
      return;
    }
    if (uu0 && vv0) atomicAdd(p, w00);
    if (uu1 && vv0) atomicAdd(p + 1, w10);
    if (uu0 && vv1) atomicAdd(p + nu, w01);
    if (uu1 && vv1) atomicAdd(p + nu + 1, w11);
  }
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
//
// Sources of the samples (SRC):
//   SRC_GLOBAL  gradient images (CENTRAL) or raw taps (EXACT) from global memory;
//   SRC_SMEM    the tile footprint staged in shared memory -- raw taps for
//               EXACT, and for CENTRAL the 4x4-minus-corners neighbourhood
//               whose central differences equal the gradient images there
//               (only for "central-safe" tiles, whose differences never use
//               the one-sided edge rule).
enum { SRC_GLOBAL = 0, SRC_SMEM = 1 };

//
// A staged footprint is zero-padded and covers every tap, so with SRC_SMEM
// the coordinates are never clamped (EDGE then only guards the scatter of
// the fused data VJP).
template <int ZB, typename T, bool FDK, bool EXACT, bool EDGE, bool PROJ, int SRC,
          typename E = T, int P = StageGeom<T>::P>
__device__ __forceinline__ void vjp_view(const T* img, const float2* gimg, const E* buf,
                                         float* pout, float* qout, long long rs, int nu, int nv,
                                         const TileView& t, float dx, float dy,
                                         const float (&delta)[ZB], float (&S)[3], float (&Z)[3]) {
  constexpr bool CLAMP = EDGE && SRC == SRC_GLOBAL;
  
  float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    const float dz = k - 0.5f * (ZB - 1);
    Sample s = locate<CLAMP>(fmaf(dz, t.ru[2], u0), fmaf(dz, t.rv[2], v0), fmaf(dz, t.rw[2], w0),
                             t, nu, nv);
    if (CLAMP && !s.ok) continue;
    float gu, gv, val = 0.0f, gscale = 1.0f;
    if (EXACT) {
      float d00, d10, d01, d11;
      if (SRC == SRC_SMEM) {
        const E* q = staged_tap<P>(buf, t, s.bx, s.by);
        d00 = tof(q[0]);
        d10 = tof(q[1]);
        d01 = tof(q[P]);
        d11 = tof(q[P + 1]);
      } else {
        taps<EDGE>(img, rs, nu, nv, s, d00, d10, d01, d11);
      }
      const float a = d10 - d00, b = d11 - d01;
      gu = fmaf(s.tv, b - a, a);
      const float c = d01 - d00, d = d11 - d10;
      gv = fmaf(s.tu, d - c, c);
      if (FDK) val = bilerp(s.tu, s.tv, d00, d10, d01, d11);
    } else if (SRC == SRC_SMEM) {
      // central-safe interior tile: 12 staged taps around (iu, iv)
      constexpr int p = P;
      const E* q = staged_tap<P, 1>(buf, t, s.bx, s.by);
      const float a0 = tof(q[-p]), a1 = tof(q[-p + 1]);
      const float b0 = tof(q[-1]), b1 = tof(q[0]), b2 = tof(q[1]), b3 = tof(q[2]);
      const float c0 = tof(q[p - 1]), c1 = tof(q[p]), c2 = tof(q[p + 1]), c3 = tof(q[p + 2]);
      const float e0 = tof(q[2 * p]), e1 = tof(q[2 * p + 1]);
      // twice the central-difference gradient images at the four tap pixels
      gu = bilerp(s.tu, s.tv, b2 - b0, b3 - b1, c2 - c0, c3 - c1);
      gv = bilerp(s.tu, s.tv, c1 - a0, c2 - a1, e0 - b1, e1 - b2);
      gscale = 0.5f;
      if (FDK) val = bilerp(s.tu, s.tv, b1, b2, c1, c2);
    } else {
      float2 g00, g10, g01, g11;
      const float2 z2 = make_float2(0.0f, 0.0f);
      if (!EDGE) {
        int iu = s.iu, iv = s.iv;
        bc_interior(BC_GLOBAL_TAP, iu, iv, nu, nv);
        const float2* p = gimg + (long long)iv * nu + iu;
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
    const float sg = sr * gscale;
    const float a0 = gu * sg, a1 = gv * sg;
    float a2 = -fmaf(a0, s.x, a1 * s.y);
    if (FDK) a2 = fmaf(-2.0f * sr, val, a2);
    S[0] += a0;
    S[1] += a1;
    S[2] += a2;
    Z[0] = fmaf(a0, dz, Z[0]);
    Z[1] = fmaf(a1, dz, Z[1]);
    Z[2] = fmaf(a2, dz, Z[2]);
    if (PROJ && delta[k] != 0.0f)  // fused data VJP: same sample, dequantised weight
      scatter_sample<EDGE>(pout, qout, nu, nv, s,
                           delta[k] * (FDK ? s.rwi * (s.rwi * t.wgtd) : t.wgtd));
  }
}

// The CENTRAL sample loop from a staged central-safe footprint with packed
// pairs of voxels (k, k+1): the steps of vjp_view in the same order on
// f32x2 pairs, with the w-component kept negated (na2 = -a2) so that no
// negation instruction is needed.  Even and odd voxels are summed in the two
// halves of the pair accumulators and added at the end.
template <int ZB, typename T, bool FDK, bool EDGE, bool PROJ, int P = StageGeom<T>::P>
__device__ __forceinline__ void vjp_view_central2(const T* buf, float* pout, float* qout, int nu,
                                                  int nv, const TileView& t, float dx, float dy,
                                                  const float (&delta)[ZB], float (&S)[3],
                                                  float (&Z)[3]) {
  
  const float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  const float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  const float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
  const f2 U0 = pk2(u0, u0), V0 = pk2(v0, v0), W0 = pk2(w0, w0);
  const f2 RU = pk2(t.ru[2], t.ru[2]), RV = pk2(t.rv[2], t.rv[2]), RW = pk2(t.rw[2], t.rw[2]);
  const f2 M2 = pk2(MAGIC, MAGIC), TWO = pk2(2.0f, 2.0f), HALF = pk2(0.5f, 0.5f);
  const f2 WG = pk2(t.wgt, t.wgt);
  const f2 WGD = pk2(t.wgtd, t.wgtd);
  // pixel index offset of the floor bits: (av - MAGIC_BITS) nu + au - MAGIC_BITS
  const unsigned pofs = (unsigned)(t.av - MAGIC_BITS) * (unsigned)nu + (unsigned)(t.au - MAGIC_BITS);
  const f2 zero = pk2(0.0f, 0.0f);
  f2 dz = pk2(-0.5f * (ZB - 1), 1.0f - 0.5f * (ZB - 1));
  f2 ndz = pk2(0.5f * (ZB - 1), 0.5f * (ZB - 1) - 1.0f);
  f2 S0 = zero, S1 = zero, S2 = zero, Z0 = zero, Z1 = zero, Z2 = zero;
#pragma unroll
  for (int p = 0; p < ZB / 2; ++p) {
    if (p) {
      dz = add2(dz, TWO);
      ndz = sub2(ndz, TWO);
    }
    const f2 u = fma2(dz, RU, U0), v = fma2(dz, RV, V0), w = fma2(dz, RW, W0);
    float wl, wh;
    up2(w, wl, wh);
    const f2 r = pk2(rcp_approx(wl), rcp_approx(wh));
    const f2 x = mul2(u, r), y = mul2(v, r);
    const f2 rx = add2_rd(x, M2), ry = add2_rd(y, M2);
    const f2 tu = sub2(x, sub2(rx, M2)), tv = sub2(y, sub2(ry, M2));
    float bxl, bxh, byl, byh;
    up2(rx, bxl, bxh);
    up2(ry, byl, byh);
    const T* ql = staged_tap<P, 1>(buf, t, __float_as_int(bxl), __float_as_int(byl));
    const T* qh = staged_tap<P, 1>(buf, t, __float_as_int(bxh), __float_as_int(byh));
#define BP_TAP2(o) pk2(tof(ql[o]), tof(qh[o]))
    const f2 a0 = BP_TAP2(-P), a1 = BP_TAP2(-P + 1);
    const f2 b0 = BP_TAP2(-1), b1 = BP_TAP2(0), b2 = BP_TAP2(1), b3 = BP_TAP2(2);
    const f2 c0 = BP_TAP2(P - 1), c1 = BP_TAP2(P), c2 = BP_TAP2(P + 1), c3 = BP_TAP2(P + 2);
    const f2 e0 = BP_TAP2(2 * P), e1 = BP_TAP2(2 * P + 1);
#undef BP_TAP2
    // twice the central-difference gradient images at the four tap pixels
    const f2 gu = bilerp2(tu, tv, sub2(b2, b0), sub2(b3, b1), sub2(c2, c0), sub2(c3, c1));
    const f2 gv = bilerp2(tu, tv, sub2(c1, a0), sub2(c2, a1), sub2(e0, b1), sub2(e1, b2));
    const f2 D = pk2(delta[2 * p], delta[2 * p + 1]);
    const f2 sd = mul2(D, FDK ? mul2(r, mul2(r, WG)) : WG);
    const f2 sr = mul2(sd, r);
    const f2 sg = mul2(sr, HALF);
    const f2 A0 = mul2(gu, sg), A1 = mul2(gv, sg);
    f2 NA2 = fma2(A0, x, mul2(A1, y));
    if (FDK) NA2 = fma2(add2(sr, sr), bilerp2(tu, tv, b1, b2, c1, c2), NA2);
    S0 = add2(S0, A0);
    S1 = add2(S1, A1);
    S2 = sub2(S2, NA2);
    Z0 = fma2(A0, dz, Z0);
    Z1 = fma2(A1, dz, Z1);
    Z2 = fma2(NA2, ndz, Z2);
    if (PROJ) {
      // fused data VJP, per voxel: the same sample's bilinear weights (the
      // scalar scatter's formulas, packed), dequantised view weight, four
      // FP32 atomic adds per voxel; interior tiles only (no bounds checks)
      const f2 SD = mul2(D, FDK ? mul2(r, mul2(r, WGD)) : WGD);
      const f2 Q1 = mul2(SD, tv), Q0 = sub2(SD, Q1);
      const f2 W11 = mul2(Q1, tu), W01 = sub2(Q1, W11), W10 = mul2(Q0, tu), W00 = sub2(Q0, W10);
      float w[4][2];
      up2(W00, w[0][0], w[0][1]);
      up2(W10, w[1][0], w[1][1]);
      up2(W01, w[2][0], w[2][1]);
      up2(W11, w[3][0], w[3][1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int bxi = __float_as_int(h ? bxh : bxl), byi = __float_as_int(h ? byh : byl);
#ifdef BP_BOUNDS_CHECK
        int iu = bxi - MAGIC_BITS + t.au, iv = byi - MAGIC_BITS + t.av;
        bc_interior(BC_SCATTER, iu, iv, nu, nv);
        bxi = iu + MAGIC_BITS - t.au;
        byi = iv + MAGIC_BITS - t.av;
#endif
        // (iv * nu + iu) from the floor bits, in 32-bit wraparound arithmetic
        const unsigned px = (unsigned)byi * (unsigned)nu + (unsigned)bxi + pofs;
        if (BP_VJP_BLOCKS && qout) {  // one vector reduction into the block image
          red_v4(qout + 4 * px, w[0][h], w[1][h], w[2][h], w[3][h]);
          continue;
        }
        float* q = pout + px;
        atomicAdd(q, w[0][h]);
        atomicAdd(q + 1, w[1][h]);
        atomicAdd(q + nu, w[2][h]);
        atomicAdd(q + nu + 1, w[3][h]);
      }
    }
  }
  float lo, hi;
  up2(S0, lo, hi); S[0] += lo + hi;
  up2(S1, lo, hi); S[1] += lo + hi;
  up2(S2, lo, hi); S[2] += lo + hi;
  up2(Z0, lo, hi); Z[0] += lo + hi;
  up2(Z1, lo, hi); Z[1] += lo + hi;
  up2(Z2, lo, hi); Z[2] += lo + hi;
}

// Fused data VJP by lines (below) or per sample (the scalar loop).
#ifndef BP_VJP_LINES
#define BP_VJP_LINES 1
#endif
#ifndef BP_VJP_LINE_DU
#define BP_VJP_LINE_DU 0.5f
#endif

// Data VJP of one staged central-safe (hence interior) tile-view, by lines:
// thread (a, b) walks the 16 voxels of the tile's line along the axis, x or
// y, whose voxels project closest together on the detector (there the sample
// moves by less than the per-view threshold along u per voxel and barely
// along v), in the direction of increasing u.  The bilinear weights of
// consecutive samples that fall in the same detector cell (same floor pixel)
// are summed in registers, and a cell's four pixels are added to dL/dproj
// (FP32 L2 atomics) only when the line leaves it: about 4 (du + 1/16) atomic
// adds per sample instead of 4.  The arithmetic runs on packed pairs of
// consecutive voxels (f32x2), as in the motion loop.  Exact to rounding: the
// same weights, summed in another order.  dsm holds the tile's dL/dvol as
// [z][y][x] with a row pitch of TX + 1.
template <int ZB, bool FDK>
__device__ __forceinline__ void proj_lines(float* __restrict__ pout, float* __restrict__ qout,
                                           int nu, int nv, const TileView& t,
                                           const float* __restrict__ dsm) {
  static_assert(ZB == TX && TY == TX, "lines run along a 16-voxel tile edge");
  const int a = threadIdx.x & (TX - 1), b = threadIdx.x / TX;
  const bool alongx = fabsf(t.ru[0]) <= fabsf(t.ru[1]);
  const float fa = a - 0.5f * (TX - 1), fb = b - 0.5f * (ZB - 1);
  // x-lines: voxels (k, a, b); y-lines: (a, k, b)
  const float ou = alongx ? t.ru[1] : t.ru[0], ov = alongx ? t.rv[1] : t.rv[0];
  const float ow = alongx ? t.rw[1] : t.rw[0];
  float su = alongx ? t.ru[0] : t.ru[1], sv = alongx ? t.rv[0] : t.rv[1];
  float sw = alongx ? t.rw[0] : t.rw[1];
  const float u0 = fmaf(fb, t.ru[2], fmaf(fa, ou, t.U0));
  const float v0 = fmaf(fb, t.rv[2], fmaf(fa, ov, t.V0));
  const float w0 = fmaf(fb, t.rw[2], fmaf(fa, ow, t.W0));
  // walk in the direction of increasing u: step kk visits voxel k = 15 - kk
  // when the axis runs against u (the negated steps give the same positions)
  const bool rev = su < 0.0f;
  if (rev) {
    su = -su;
    sv = -sv;
    sw = -sw;
  }
  const float* dl = alongx ? dsm + (b * TY + a) * (TX + 1) : dsm + b * TY * (TX + 1) + a;
  const int dstep = alongx ? 1 : TX + 1;
  const f2 U0 = pk2(u0, u0), V0 = pk2(v0, v0), W0 = pk2(w0, w0);
  const f2 SU = pk2(su, su), SV = pk2(sv, sv), SW = pk2(sw, sw);
  const f2 M2 = pk2(MAGIC, MAGIC), TWO = pk2(2.0f, 2.0f), WGD = pk2(t.wgtd, t.wgtd);
  const unsigned pofs = (unsigned)(t.av - MAGIC_BITS) * (unsigned)nu + (unsigned)(t.au - MAGIC_BITS);
  int cb = 0, rb = 0;  // the open cell, as floor bits
  bool have = false;
  float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
  f2 dk = pk2(-0.5f * (TX - 1), 1.0f - 0.5f * (TX - 1));
#pragma unroll 2
  for (int p = 0; p < TX / 2; ++p) {
    if (p) dk = add2(dk, TWO);
    const f2 u = fma2(dk, SU, U0), v = fma2(dk, SV, V0), w = fma2(dk, SW, W0);
    float wl, wh;
    up2(w, wl, wh);
    const f2 r = pk2(rcp_approx(wl), rcp_approx(wh));
    const f2 x = mul2(u, r), y = mul2(v, r);
    const f2 rx = add2_rd(x, M2), ry = add2_rd(y, M2);
    const f2 tu = sub2(x, sub2(rx, M2)), tv = sub2(y, sub2(ry, M2));
    const int k0 = rev ? TX - 1 - 2 * p : 2 * p, k1 = rev ? k0 - 1 : k0 + 1;
    const f2 D = pk2(dl[k0 * dstep], dl[k1 * dstep]);
    const f2 SD = mul2(D, FDK ? mul2(r, mul2(r, WGD)) : WGD);
    const f2 Q1 = mul2(SD, tv), Q0 = sub2(SD, Q1);
    const f2 W11 = mul2(Q1, tu), W01 = sub2(Q1, W11), W10 = mul2(Q0, tu), W00 = sub2(Q0, W10);
    float bxf[2], byf[2], ww[4][2];
    up2(rx, bxf[0], bxf[1]);
    up2(ry, byf[0], byf[1]);
    up2(W00, ww[0][0], ww[0][1]);
    up2(W10, ww[1][0], ww[1][1]);
    up2(W01, ww[2][0], ww[2][1]);
    up2(W11, ww[3][0], ww[3][1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int bx = __float_as_int(bxf[h]), by = __float_as_int(byf[h]);
      const bool keep = have && bx == cb && by == rb;
      if (have && !keep) {  // the line leaves the open cell: add its four pixels
        int fc = cb - MAGIC_BITS + t.au, fr = rb - MAGIC_BITS + t.av;
        bc_interior(BC_SCATTER, fc, fr, nu, nv);
        const unsigned px = (unsigned)(fr + MAGIC_BITS - t.av) * (unsigned)nu +
                            (unsigned)(fc + MAGIC_BITS - t.au) + pofs;
        if (BP_VJP_BLOCKS && qout) {
          red_v4(qout + 4 * px, a0, a1, b0, b1);
        } else {
          float* q = pout + px;
          atomicAdd(q, a0);
          atomicAdd(q + 1, a1);
          atomicAdd(q + nu, b0);
          atomicAdd(q + nu + 1, b1);
        }
      }
      a0 = (keep ? a0 : 0.0f) + ww[0][h];
      a1 = (keep ? a1 : 0.0f) + ww[1][h];
      b0 = (keep ? b0 : 0.0f) + ww[2][h];
      b1 = (keep ? b1 : 0.0f) + ww[3][h];
      cb = bx;
      rb = by;
      have = true;
    }
  }
  int fc = cb - MAGIC_BITS + t.au, fr = rb - MAGIC_BITS + t.av;
  bc_interior(BC_SCATTER, fc, fr, nu, nv);
  const unsigned px = (unsigned)(fr + MAGIC_BITS - t.av) * (unsigned)nu +
                      (unsigned)(fc + MAGIC_BITS - t.au) + pofs;
  if (BP_VJP_BLOCKS && qout) {
    red_v4(qout + 4 * px, a0, a1, b0, b1);
    return;
  }
  float* q = pout + px;
  atomicAdd(q, a0);
  atomicAdd(q + 1, a1);
  atomicAdd(q + nu, b0);
  atomicAdd(q + nu + 1, b1);
}

// One view of one tile: the sample loop (from the staged footprint when it
// was staged), then the warp reduce-scatter of the 12 sums into redv[warp].
// Staged CENTRAL (central-safe) tiles run the packed motion loop and, when
// the data VJP is fused, the line pass above; the other tiles scatter the
// data VJP per sample.
template <int ZB, typename T, bool FDK, bool EXACT, bool PROJ, typename E, int P>
__device__ __forceinline__ void vjp_tile_view(const T* img, const float2* gimg, const E* buf,
                                              bool staged, float* pout, float* qout,
                                              const ProjInfo& pi, const TileView& t,
                                              const TileIdx& ti,
                                              const float (&delta)[ZB], const float* dsm,
                                              float (*redv)[12]) {
  float S[3] = {0.0f, 0.0f, 0.0f}, Z[3] = {0.0f, 0.0f, 0.0f};
  if (staged && !EXACT) {
    // CENTRAL footprints are staged only for central-safe, hence interior,
    // tiles.  With the fused data VJP: the line pass where samples along
    // the ray-parallel axis move by at most BP_VJP_LINE_DU px per voxel
    // (there it merges most: about 4 (du + 1/16) atomics per sample), else
    // four atomics per sample from the packed loop, with fewer instructions
    if (PROJ && BP_VJP_LINES &&
        fminf(fabsf(t.ru[0]), fabsf(t.ru[1])) <= BP_VJP_LINE_DU * t.W0) {
      vjp_view_central2<ZB, E, FDK, false, false, P>(buf, pout, qout, pi.nu, pi.nv, t, ti.dx, ti.dy,
                                                     delta, S, Z);
      proj_lines<ZB, FDK>(pout, qout, pi.nu, pi.nv, t, dsm);
    } else {
      vjp_view_central2<ZB, E, FDK, false, PROJ, P>(buf, pout, qout, pi.nu, pi.nv, t, ti.dx, ti.dy,
                                                    delta, S, Z);
    }
  } else if (staged) {
    // (the per-sample paths keep scalar scatters in the fused kernel: block
    // reductions of their in-range samples measured 1 % slower there,
    // 15.12 against 14.94 ms on c2, while the data VJP alone gains 10 %)
    if (t.mode == MODE_INTERIOR || !PROJ)
      vjp_view<ZB, T, FDK, EXACT, false, PROJ, SRC_SMEM, E, P>(
          img, gimg, buf, pout, nullptr, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, delta, S, Z);
    else
      vjp_view<ZB, T, FDK, EXACT, true, PROJ, SRC_SMEM, E, P>(
          img, gimg, buf, pout, nullptr, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, delta, S, Z);
  } else {
    if (t.mode == MODE_INTERIOR)
      vjp_view<ZB, T, FDK, EXACT, false, PROJ, SRC_GLOBAL, E, P>(
          img, gimg, buf, pout, nullptr, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, delta, S, Z);
    else
      vjp_view<ZB, T, FDK, EXACT, true, PROJ, SRC_GLOBAL, E, P>(
          img, gimg, buf, pout, nullptr, pi.rs, pi.nu, pi.nv, t, ti.dx, ti.dy, delta, S, Z);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  if (!(lane & 1) && slot < 12) redv[warp][slot] = tot;
}

// Write the record of one (tile, view): fixed-order sum of the 8 warps'
// values, plus the anchors (threads 0..PSLOTS-1).
__device__ __forceinline__ void vjp_write_record(const TileView& t, const float (*redv)[12],
                                                 bool any, int j, int tile, int ntiles,
                                                 float* __restrict__ partials) {
  const int slot = threadIdx.x;
  if (slot >= PSLOTS) return;
  float val = 0.0f;
  if (slot < 12) {
    if (any && t.mode != MODE_SKIP)
      for (int w = 0; w < NT / 32; ++w) val += redv[w][slot];
  } else if (slot == 12) {
    val = (float)t.au;
  } else if (slot == 13) {
    val = (float)t.av;
  }
  partials[((long long)j * ntiles + tile) * PSLOTS + slot] = val;
}

// Motion VJP (optionally fused with the data VJP).  Grid: (view chunk, tile),
// tiles fastest, so the CTAs resident at any time share a few views whose
// data and dL/dproj rows stay in L2.  Per tile the views of the chunk are
// processed in order with the footprint of view j+1 copied to shared memory
// while view j is computed (STAGE), like the forward.
//
// FP16/BF16 data (CONV) is staged through a raw buffer and converted once per
// (tile, view) into an FP32 buffer: convert view j, barrier, issue the raw
// copy of view j+1, compute view j, wait for the copy, barrier.
// With the fused data VJP the tile's dL/dvol is also kept in shared memory
// ([z][y][x], row pitch TX + 1) for the line pass.
constexpr int DSM_BYTES = ZB_VJP * TY * (TX + 1) * 4;
template <typename T, bool PROJ = false>
__host__ __device__ constexpr int vjp_smem_bytes() {
  return (conv_staging<T>() ? CONV_F_BYTES + CONV_R_BYTES : 2 * STAGE_BYTES) +
         (PROJ ? DSM_BYTES : 0);
}

// One work item of the VJP: views [item / ntiles * vchunk, + vchunk) of tile
// item % ntiles.  All threads of the CTA call it with the CTA's shared memory.
template <int ZB, typename T, bool FDK, bool EXACT, bool PROJ, bool STAGE>
__device__ __forceinline__ void vjp_item(const float* __restrict__ dvol, const T* __restrict__ proj,
                                         const ProjInfo& pi, const float2* __restrict__ grad,
                                         const ViewGeom* __restrict__ geom, const VolInfo& vi,
                                         float* __restrict__ partials, float* __restrict__ dproj,
                                         float* __restrict__ dblk, int vchunk, int item, TileView (*tvs)[VB],
                                         float (*red)[NT / 32][12], unsigned char* dyn_smem) {
  constexpr bool CONV = STAGE && conv_staging<T>();
  using G = typename std::conditional<CONV, ConvGeom, StageGeom<T>>::type;
  T* bufs = reinterpret_cast<T*>(dyn_smem);  // plain: two buffers of T
  float* F = reinterpret_cast<float*>(dyn_smem);  // CONV: FP32 buffer, then the raw one
  T* R = reinterpret_cast<T*>(dyn_smem + CONV_F_BYTES);
  float* dsm = reinterpret_cast<float*>(dyn_smem + vjp_smem_bytes<T, false>());
  constexpr int CAP = STAGE_BYTES / (int)sizeof(T);
  constexpr int HALO = EXACT ? 0 : 1;
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const int tile = item % ntiles;
  const int vbeg = (item / ntiles) * vchunk, vend = min(pi.nviews, vbeg + vchunk);
  const TileIdx ti = tile_index<ZB>(vi, tile);
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
  if (PROJ && STAGE && !EXACT && BP_VJP_LINES) {
#pragma unroll
    for (int k = 0; k < ZB; ++k) dsm[(k * TY + ti.ly) * (TX + 1) + ti.lx] = delta[k];
  }
  const bool any = __syncthreads_or(nz);
  const int nvw = vend - vbeg, nbatch = (nvw + VB - 1) / VB;
  setup_batch<T, STAGE, G>(tvs[0], geom, vbeg, min(VB, nvw), ti, pi.nu, pi.nv, true, HALO, !EXACT);
  if (nbatch > 1)
    setup_batch<T, STAGE, G>(tvs[1], geom, vbeg + VB, min(VB, nvw - VB), ti, pi.nu, pi.nv, true,
                             HALO, !EXACT);
  __syncthreads();
  if (STAGE && any && tvs[0][0].staged) {
    if constexpr (CONV)
      stage_issue<T, CONV_P>(R, proj + (long long)vbeg * pi.vs, pi.rs, pi.nu, pi.nv, tvs[0][0]);
    else
      stage_issue(bufs, proj + (long long)vbeg * pi.vs, pi.rs, pi.nu, pi.nv, tvs[0][0]);
  }
  cp_async_commit();
  if constexpr (CONV) {
    cp_async_wait0();
    __syncthreads();
  }
  for (int v = vbeg; v < vend; ++v) {
    const int idx = v - vbeg, k = idx / VB, b = idx - k * VB;
    if (b == 0 && k >= 1) {
      // batch k-1 is complete: write its last record, then reuse its slot
      vjp_write_record(tvs[(k - 1) & 1][VB - 1], red[(idx - 1) & 1], any, v - 1, tile, ntiles,
                       partials);
      __syncthreads();
      if (k + 1 < nbatch)
        setup_batch<T, STAGE, G>(tvs[(k + 1) & 1], geom, vbeg + (k + 1) * VB,
                                 min(VB, nvw - (k + 1) * VB), ti, pi.nu, pi.nv, true, HALO,
                                 !EXACT);
      __syncthreads();
    }
    const TileView t = tvs[k & 1][b];
    const int kn = (idx + 1) / VB;
    const TileView* tn = v + 1 < vend ? &tvs[kn & 1][idx + 1 - kn * VB] : nullptr;
    if constexpr (CONV) {
      if (any && t.staged) convert_stage<T>(F, R, t);
      __syncthreads();  // F holds view v; R is free
      if (any && tn && tn->staged)
        stage_issue<T, CONV_P>(R, proj + (long long)(v + 1) * pi.vs, pi.rs, pi.nu, pi.nv, *tn);
      cp_async_commit();
    } else {
      if (STAGE && any && tn && tn->staged)
        stage_issue(bufs + ((idx + 1) & 1) * CAP, proj + (long long)(v + 1) * pi.vs, pi.rs, pi.nu,
                    pi.nv, *tn);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();
    }
    // the record of view v-1 (its sums are complete since the last barrier;
    // red[(idx - 1) & 1] is next written by view v+1, after another barrier)
    if (idx > 0 && b > 0)
      vjp_write_record(tvs[k & 1][b - 1], red[(idx - 1) & 1], any, v - 1, tile, ntiles, partials);
    if (any && t.mode != MODE_SKIP) {
      const T* img = proj + (long long)v * pi.vs;
      const float2* gimg = EXACT ? nullptr : grad + (long long)v * pi.nv * pi.nu;
      float* pout = PROJ ? dproj + (long long)v * pi.nv * pi.nu : nullptr;
      float* qout =
          PROJ && dblk ? dblk + (long long)v * 4 * pi.nv * pi.nu : nullptr;
      if constexpr (CONV)
        vjp_tile_view<ZB, T, FDK, EXACT, PROJ, float, CONV_P>(img, gimg, F, t.staged, pout, qout,
                                                              pi, t, ti, delta, dsm, red[idx & 1]);
      else
        vjp_tile_view<ZB, T, FDK, EXACT, PROJ, T, StageGeom<T>::P>(
            img, gimg, bufs + (idx & 1) * CAP, STAGE && t.staged, pout, qout, pi, t, ti, delta,
            dsm, red[idx & 1]);
    }
    if constexpr (CONV) cp_async_wait0();  // the raw copy of view v+1
    __syncthreads();  // F and the staging buffers are free; red[idx & 1] complete
  }
  if (nvw > 0) {
    const int il = nvw - 1, kl = il / VB;
    vjp_write_record(tvs[kl & 1][il - kl * VB], red[il & 1], any, vend - 1, tile, ntiles,
                     partials);
  }
}

template <int ZB, typename T, bool FDK, bool EXACT, bool PROJ, bool STAGE>
__global__ void __launch_bounds__(NT, VJP_MINB)
    vjp_motion_kernel(const float* __restrict__ dvol, const T* __restrict__ proj, ProjInfo pi,
                      const float2* __restrict__ grad, const ViewGeom* __restrict__ geom,
                      VolInfo vi, float* __restrict__ partials, float* __restrict__ dproj,
                      float* __restrict__ dblk, int vchunk) {
  __shared__ TileView tvs[2][VB];
  __shared__ float red[2][NT / 32][12];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  vjp_item<ZB, T, FDK, EXACT, PROJ, STAGE>(dvol, proj, pi, grad, geom, vi, partials, dproj, dblk,
                                           vchunk, blockIdx.x, tvs, red, dyn_smem);
}

#ifndef BP_VJP_CHUNK_MIB
#define BP_VJP_CHUNK_MIB 128
#endif
// Views per chunk of the view-chunked VJP grids: the bytes that one chunk's
// views touch (projections, gradient images, dL/dproj rows) are kept near
// BP_VJP_CHUNK_MIB, at most 32 views.  Measured on c2 (fused VJP, before
// the block image): 16 MiB 23.1 ms, 32 MiB 20.3 ms, 64 MiB 18.1 ms, 128 MiB
// 17.4 ms.
static int view_chunk(const ProjInfo& pi, long long bytes_per_px) {
  const long long per_view = (long long)pi.nu * pi.nv * bytes_per_px;
  long long c = ((long long)BP_VJP_CHUNK_MIB << 20) / (per_view > 0 ? per_view : 1);
  if (c < 1) c = 1;
  if (c > VB) c = VB;
  return (int)c;
}

template <typename T, bool FDK, bool EXACT, bool PROJ, bool STAGE>
static cudaError_t vjp_launch(const float* dvol, const void* proj, const ProjInfo& pi,
                              const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                              float* partials, float* dproj, float* blk, int vc,
                              unsigned nblocks, cudaStream_t s) {
  const int smem = STAGE ? vjp_smem_bytes<T, PROJ && !EXACT && BP_VJP_LINES>() : 0;
  if (STAGE) {
    cudaError_t e = smem_attr_once<vjp_motion_kernel<ZB_VJP, T, FDK, EXACT, PROJ, STAGE>>(smem);
    if (e != cudaSuccess) return e;
  }
  vjp_motion_kernel<ZB_VJP, T, FDK, EXACT, PROJ, STAGE><<<nblocks, NT, smem, s>>>(
      dvol, (const T*)proj, pi, grad, geom, vi, partials, dproj, blk, vc);
  return cudaGetLastError();
}

template <typename T, bool FDK, bool EXACT>
static cudaError_t vjp_dispatch(const float* dvol, const void* proj, const ProjInfo& pi,
                                const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                                float* partials, float* dproj, float* blk, cudaStream_t s) {
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const bool stage = stageable<T>(proj, pi);
  // block images only where the staged CENTRAL paths scatter
  const bool useb = dproj && blk && stage && !EXACT && BP_VJP_BLOCKS;
  // the block image is left out of the chunk's byte count: measured on c2,
  // counting its 16 bytes per pixel (smaller chunks) made the fused VJP 2.8 %
  // slower (15.37 against 14.94 ms), counting 8 bytes 1.7 %
  const long long bpp = (long long)sizeof(T) + (EXACT ? 0 : 8) + (dproj ? 4 : 0);
  const int vc = view_chunk(pi, bpp);
  const unsigned nblocks = (unsigned)((long long)ntiles * ((pi.nviews + vc - 1) / vc));
  if (dproj) {
    cudaError_t e = cudaSuccess;
    if (useb) e = cudaMemsetAsync(blk, 0, sizeof(float) * (size_t)block_image_floats(pi), s);
    if (e == cudaSuccess)
      e = stage ? vjp_launch<T, FDK, EXACT, true, true>(dvol, proj, pi, grad, geom, vi, partials,
                                                        dproj, useb ? blk : nullptr, vc, nblocks,
                                                        s)
                : vjp_launch<T, FDK, EXACT, true, false>(dvol, proj, pi, grad, geom, vi,
                                                         partials, dproj, nullptr, vc, nblocks, s);
    if (e == cudaSuccess && useb) e = launch_block_combine(blk, pi, dproj, s);
    return e;
  }
  return stage ? vjp_launch<T, FDK, EXACT, false, true>(dvol, proj, pi, grad, geom, vi, partials,
                                                        nullptr, nullptr, vc, nblocks, s)
               : vjp_launch<T, FDK, EXACT, false, false>(dvol, proj, pi, grad, geom, vi,
                                                         partials, nullptr, nullptr, vc, nblocks,
                                                         s);
}

bool vjp_uses_blocks(const void* proj, int dtype, const ProjInfo& pi, int exact) {
  if (exact || !BP_VJP_BLOCKS) return false;
  if (dtype == 0) return stageable<float>(proj, pi);
  if (dtype == 1) return stageable<__half>(proj, pi);
  return stageable<__nv_bfloat16>(proj, pi);
}

// Set the VJP kernels' shared-memory attributes on the current device
// (call before capturing a graph).
cudaError_t prepare_vjp(int dtype, int fdk, int exact) {
  cudaError_t e = cudaSuccess;
#define BP_PREP(T)                                                                                 \
  do {                                                                                             \
    const int smem = vjp_smem_bytes<T>();                                                          \
    if (fdk && exact) e = smem_attr_once<vjp_motion_kernel<ZB_VJP, T, true, true, false, true>>(smem); \
    if (fdk && !exact) e = smem_attr_once<vjp_motion_kernel<ZB_VJP, T, true, false, false, true>>(smem); \
    if (!fdk && exact) e = smem_attr_once<vjp_motion_kernel<ZB_VJP, T, false, true, false, true>>(smem); \
    if (!fdk && !exact) e = smem_attr_once<vjp_motion_kernel<ZB_VJP, T, false, false, false, true>>(smem); \
  } while (0)
  if (dtype == 0) BP_PREP(float);
  else if (dtype == 1) BP_PREP(__half);
  else BP_PREP(__nv_bfloat16);
#undef BP_PREP
  return e;
}

template <typename T>
static cudaError_t vjp_dispatch_t(int fdk, int exact, const float* dvol, const void* proj,
                                  const ProjInfo& pi, const float2* grad, const ViewGeom* geom,
                                  const VolInfo& vi, float* partials, float* dproj,
                                  float* blk, cudaStream_t s) {
  if (fdk)
    return exact ? vjp_dispatch<T, true, true>(dvol, proj, pi, grad, geom, vi, partials, dproj,
                                               blk, s)
                 : vjp_dispatch<T, true, false>(dvol, proj, pi, grad, geom, vi, partials, dproj,
                                                blk, s);
  return exact ? vjp_dispatch<T, false, true>(dvol, proj, pi, grad, geom, vi, partials, dproj,
                                              blk, s)
               : vjp_dispatch<T, false, false>(dvol, proj, pi, grad, geom, vi, partials, dproj,
                                               blk, s);
}

cudaError_t launch_vjp_motion(const float* dvol, const void* proj, int dtype, const ProjInfo& pi,
                              const float2* grad, const ViewGeom* geom, const VolInfo& vi,
                              int fdk, int exact, float* partials, float* dproj, float* blk,
                              cudaStream_t s) {
  if (vi.zb != ZB_VJP) return cudaErrorInvalidValue;
  if (dtype == 0)
    return vjp_dispatch_t<float>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials, dproj, blk,
                                 s);
  if (dtype == 1)
    return vjp_dispatch_t<__half>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials, dproj,
                                  blk, s);
  return vjp_dispatch_t<__nv_bfloat16>(fdk, exact, dvol, proj, pi, grad, geom, vi, partials,
                                       dproj, blk, s);
}

// ------------------------------------------------- VJP w.r.t. the data

// Adjoint of Eq. 3 in d_j: every voxel-view adds s = delta * c * omega times
// its four bilinear weights to four detector pixels of a contiguous
// [V][nv][nu] FP32 image (zeroed by the caller), with global FP32 atomics
// reduced in L2: one vector reduction into the block image bout (when given)
// for a sample whose four taps lie on the detector, else up to four scalar
// ones.  (Measured on GB300: shared-memory
// FP32 atomics are emulated, and vector atomics with zero lanes cost as much
// as full ones, so neither privatisation nor padded vectors are used.)
template <int ZB, bool FDK, bool EDGE>
__device__ __forceinline__ void proj_view(float* out, float* bout, int nu, int nv,
                                          const TileView& t, float dx, float dy,
                                          const float (&delta)[ZB]) {
  const float u0 = fmaf(dy, t.ru[1], fmaf(dx, t.ru[0], t.U0));
  const float v0 = fmaf(dy, t.rv[1], fmaf(dx, t.rv[0], t.V0));
  const float w0 = fmaf(dy, t.rw[1], fmaf(dx, t.rw[0], t.W0));
#pragma unroll
  for (int k = 0; k < ZB; ++k) {
    if (delta[k] == 0.0f) continue;
    const float dz = k - 0.5f * (ZB - 1);
    Sample s = locate<EDGE>(fmaf(dz, t.ru[2], u0), fmaf(dz, t.rv[2], v0), fmaf(dz, t.rw[2], w0),
                            t, nu, nv);
    if (EDGE && !s.ok) continue;
    const float sd = delta[k] * (FDK ? s.rwi * (s.rwi * t.wgtd) : t.wgtd);
    scatter_sample<EDGE>(out, bout, nu, nv, s, sd);
  }
}

template <int ZB, bool FDK>
__global__ void __launch_bounds__(NT, 2)
    vjp_proj_kernel(const float* __restrict__ dvol, ProjInfo pi, const ViewGeom* __restrict__ geom,
                    VolInfo vi, float* __restrict__ dproj, float* __restrict__ blk, int vchunk) {
  __shared__ TileView tvs[VB];
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const int tile = blockIdx.x % ntiles;
  const int vbeg = (blockIdx.x / ntiles) * vchunk, vend = min(pi.nviews, vbeg + vchunk);
  const TileIdx ti = tile_index<ZB>(vi, tile);
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
  for (int j0 = vbeg; j0 < vend; j0 += VB) {
    const int nb = min(VB, vend - j0);
    __syncthreads();
    setup_batch<float, false>(tvs, geom, j0, nb, ti, pi.nu, pi.nv, true);
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      const TileView t = tvs[b];
      if (t.mode == MODE_SKIP) continue;
      float* out = dproj + (long long)(j0 + b) * pi.nv * pi.nu;
      float* bout = blk ? blk + (long long)(j0 + b) * pi.nv * pi.nu * 4 : nullptr;
      if (t.mode == MODE_INTERIOR)
        proj_view<ZB, FDK, false>(out, bout, pi.nu, pi.nv, t, ti.dx, ti.dy, delta);
      else
        proj_view<ZB, FDK, true>(out, bout, pi.nu, pi.nv, t, ti.dx, ti.dy, delta);
    }
  }
}

cudaError_t launch_vjp_proj(const float* dvol, const ProjInfo& pi, const ViewGeom* geom,
                            const VolInfo& vi, int fdk, float* dproj, float* blk, cudaStream_t s) {
  if (vi.zb != ZB_VJP) return cudaErrorInvalidValue;
  if (!BP_VJP_BLOCKS) blk = nullptr;
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const int vc = view_chunk(pi, blk ? 20 : 4);
  const unsigned nblocks = (unsigned)((long long)ntiles * ((pi.nviews + vc - 1) / vc));
  if (blk) {
    cudaError_t e = cudaMemsetAsync(blk, 0, sizeof(float) * (size_t)block_image_floats(pi), s);
    if (e != cudaSuccess) return e;
  }
  if (fdk)
    vjp_proj_kernel<ZB_VJP, true><<<nblocks, NT, 0, s>>>(dvol, pi, geom, vi, dproj, blk, vc);
  else
    vjp_proj_kernel<ZB_VJP, false><<<nblocks, NT, 0, s>>>(dvol, pi, geom, vi, dproj, blk, vc);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && blk) e = launch_block_combine(blk, pi, dproj, s);
  return e;
}

// ------------------------------------------------------------------ batches
// The forward over the tiles of every member of a batch.  The member table is
// a __grid_constant__ parameter, so the tile code reads each job's sizes and
// pointers from read-only parameter space, as the per-job kernels read their
// arguments.  Each tile runs the per-job block code, so the results are bit
// for bit those of the per-job launches.  Members are staged (checked by the
// host) in the batch's dtype.
//
// The forward is persistent: SMs x (resident CTAs per SM) blocks take tiles
// from an atomic counter, so tiles run in order (CTAs resident at the same
// time work on neighbouring tiles) and CTAs that drew cheap tiles (off the
// detector) take more; no CTA waits on another.  (The batch's VJP stage
// launches each member's own VJP kernel: a grouped launch over all members'
// (tile, view chunk) items read the job fields through run-time-indexed
// parameter loads and ran 8.7 % slower than the per-job kernel.)

template <int ZB, typename T, bool FDK>
__global__ void __launch_bounds__(NT, FWD_MINB)
    batch_forward_kernel(const __grid_constant__ BatchTable t, unsigned* __restrict__ counter) {
  __shared__ TileView tvs[2][VB];
  __shared__ int item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int n = t.njobs, total = t.off_fwd[n];
  for (;;) {
    __syncthreads();  // every thread is done with the previous tile
    if (threadIdx.x == 0) item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int w = item;
    if (w >= total) break;
    const int j = batch_find(t.off_fwd, n, w);
    const BatchJob& J = t.job[j];
    forward_tile<ZB, T, FDK, true>((const T*)J.proj, J.pi, J.geom, J.vif, J.vol, w - t.off_fwd[j],
                                   tvs, dyn_smem);
  }
}

int forward_zb() { return ZB_FWD; }

template <typename T, bool FDK>
static cudaError_t batch_forward_t(const BatchTable& tab, unsigned* counter, int sms,
                                   cudaStream_t s) {
  const int smem = fwd_smem_bytes<T>();
  cudaError_t e = smem_attr_once<batch_forward_kernel<ZB_FWD, T, FDK>>(smem);
  if (e != cudaSuccess) return e;
  batch_forward_kernel<ZB_FWD, T, FDK><<<sms * FWD_MINB, NT, smem, s>>>(tab, counter);
  return cudaGetLastError();
}

cudaError_t launch_batch_forward(const BatchTable& tab, unsigned* counter, int dtype, int fdk,
                                 int sms, cudaStream_t s) {
  if (dtype == 0) return fdk ? batch_forward_t<float, true>(tab, counter, sms, s)
                             : batch_forward_t<float, false>(tab, counter, sms, s);
  if (dtype == 1) return fdk ? batch_forward_t<__half, true>(tab, counter, sms, s)
                             : batch_forward_t<__half, false>(tab, counter, sms, s);
  return fdk ? batch_forward_t<__nv_bfloat16, true>(tab, counter, sms, s)
             : batch_forward_t<__nv_bfloat16, false>(tab, counter, sms, s);
}

// Shared-memory attributes of the batch kernels on the current device (call
// before capturing a graph; the members' VJP kernels are prepared by
// prepare_vjp).
cudaError_t prepare_batch(int dtype, int fdk, int exact) {
  (void)exact;
  if (dtype == 0)
    return fdk ? smem_attr_once<batch_forward_kernel<ZB_FWD, float, true>>(fwd_smem_bytes<float>())
               : smem_attr_once<batch_forward_kernel<ZB_FWD, float, false>>(fwd_smem_bytes<float>());
  if (dtype == 1)
    return fdk ? smem_attr_once<batch_forward_kernel<ZB_FWD, __half, true>>(fwd_smem_bytes<__half>())
               : smem_attr_once<batch_forward_kernel<ZB_FWD, __half, false>>(fwd_smem_bytes<__half>());
  return fdk ? smem_attr_once<batch_forward_kernel<ZB_FWD, __nv_bfloat16, true>>(
                   fwd_smem_bytes<__nv_bfloat16>())
             : smem_attr_once<batch_forward_kernel<ZB_FWD, __nv_bfloat16, false>>(
                   fwd_smem_bytes<__nv_bfloat16>());
}

}  // namespace bpk
