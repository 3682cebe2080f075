// C-ABI of bp_gb300 (declared in include/bp_gb300.h): argument checks,
// workspace ownership, host/device staging and kernel launches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>


#include "bp_ctx.h"

namespace {

using namespace bpctx;

size_t dtype_size(int dt) { return dt == BP_F32 ? 4 : 2; }

int check_proj(bp_ctx* ctx, const bp_proj_desc* pd) {
  if (!pd) return fail(ctx, BP_ERR_INVALID_ARG, "proj descriptor is NULL");
  if (pd->nu < 1 || pd->nv < 1 || pd->nviews < 0)
    return fail(ctx, BP_ERR_INVALID_ARG, "nu, nv must be >= 1 and nviews >= 0");
  if (pd->dtype != BP_F32 && pd->dtype != BP_F16 && pd->dtype != BP_BF16)
    return fail(ctx, BP_ERR_INVALID_ARG, "unknown projection dtype");
  if (pd->row_stride < pd->nu || pd->view_stride < (long long)pd->nv * pd->row_stride)
    return fail(ctx, BP_ERR_INVALID_ARG, "row_stride < nu or view_stride < nv*row_stride");
  if ((long long)pd->nv * pd->row_stride + 1 > 0x7fffffffLL ||
      (long long)pd->nv * pd->nu * 2 > 0x7fffffffLL)
    return fail(ctx, BP_ERR_UNSUPPORTED, "a single view must have fewer than 2^30 elements");
  if (pd->nu > (1 << 20) || pd->nv > (1 << 20))
    return fail(ctx, BP_ERR_UNSUPPORTED, "detector dimensions above 2^20 pixels");
  return BP_OK;
}

int check_vol(bp_ctx* ctx, const bp_vol_desc* vd) {
  if (!vd) return fail(ctx, BP_ERR_INVALID_ARG, "volume descriptor is NULL");
  if (vd->nx < 0 || vd->ny < 0 || vd->nz < 0)
    return fail(ctx, BP_ERR_INVALID_ARG, "negative volume dimension");
  if (vd->nx > (1 << 20) || vd->ny > (1 << 20) || vd->nz > (1 << 20))
    return fail(ctx, BP_ERR_UNSUPPORTED, "volume dimension above 2^20");
  for (int a = 0; a < 3; ++a)
    if (!(vd->spacing[a] != 0.0) || vd->spacing[a] != vd->spacing[a])
      return fail(ctx, BP_ERR_INVALID_ARG, "voxel spacing must be finite and non-zero");
  return BP_OK;
}

VolInfo make_volinfo(const bp_vol_desc* vd, int zb) {
  VolInfo vi;
  vi.nx = vd->nx;
  vi.ny = vd->ny;
  vi.nz = vd->nz;
  vi.zb = zb;
  vi.tiles_x = (vd->nx + bpk::TX - 1) / bpk::TX;
  vi.tiles_y = (vd->ny + bpk::TY - 1) / bpk::TY;
  vi.tiles_z = (vd->nz + zb - 1) / zb;
  vi.cx = 0.5 * (vd->nx - 1);
  vi.cy = 0.5 * (vd->ny - 1);
  vi.cz = 0.5 * (vd->nz - 1);
  const double c[3] = {vi.cx, vi.cy, vi.cz};
  for (int e = 0; e < 12; ++e) vi.A[e] = 0.0;
  for (int a = 0; a < 3; ++a) {
    vi.A[4 * a + a] = vd->spacing[a];
    vi.A[4 * a + 3] = vd->origin[a] + c[a] * vd->spacing[a];
  }
  return vi;
}

ProjInfo make_projinfo(const bp_proj_desc* pd) {
  ProjInfo pi;
  pi.nu = pd->nu;
  pi.nv = pd->nv;
  pi.nviews = pd->nviews;
  pi.rs = pd->row_stride;
  pi.vs = pd->view_stride;
  return pi;
}

size_t proj_bytes(const bp_proj_desc* pd) {
  if (pd->nviews == 0) return 0;
  long long elems = (long long)(pd->nviews - 1) * pd->view_stride +
                    (long long)(pd->nv - 1) * pd->row_stride + pd->nu;
  return (size_t)elems * dtype_size(pd->dtype);
}

constexpr int ZB = bpk::ZB_VJP;

// Stage the per-view inputs and run the FP64 composition into ctx->geom.
int prepare_views(bp_ctx* ctx, const bp_proj_desc* pd, const double* P, const double* motion,
                  const double* view_weight, int weight, const VolInfo& vi, cudaStream_t s,
                  const double** dP, const double** dmotion) {
  const int V = pd->nviews;
  const void* q = nullptr;
  CK(stage_in(ctx->s_P, P, sizeof(double) * 12 * V, s, &q), "copy P");
  *dP = (const double*)q;
  CK(stage_in(ctx->s_motion, motion, sizeof(double) * 6 * V, s, &q), "copy motion");
  *dmotion = (const double*)q;
  CK(stage_in(ctx->s_vw, view_weight, sizeof(double) * V, s, &q), "copy view_weight");
  const double* dvw = (const double*)q;
  CK(stage_in(ctx->s_scale, pd->view_scale, sizeof(float) * V, s, &q), "copy view_scale");
  const float* dsc = (const float*)q;
  CK(ensure(ctx->geom, sizeof(ViewGeom) * (size_t)V), "alloc view table");
  CK(TL(K_COMPOSE, 1, bpk::launch_compose(*dP, *dmotion, dvw, dsc, V, weight == BP_WEIGHT_FDK,
                                          pd->sid, vi, (ViewGeom*)ctx->geom.p, nullptr, s)),
     "compose");
  return BP_OK;
}

}  // namespace

extern "C" {

int bp_ctx_create(int device, bp_ctx** out) {
  if (!out) return BP_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return BP_ERR_CUDA;
  }
  if (device < 0 || device >= n) return BP_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return BP_ERR_CUDA;
  }
  if (prop.major != 10 || prop.minor != 3) return BP_ERR_UNSUPPORTED;
  bp_ctx* c = new bp_ctx();
  c->device = device;
  *out = c;
  return BP_OK;
}

void bp_ctx_destroy(bp_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  Buf* bufs[] = {&ctx->geom,   &ctx->grad,   &ctx->partials,   &ctx->shblk,      &ctx->fdk_tab,
                 &ctx->s_proj,
                 &ctx->s_P,    &ctx->s_motion, &ctx->s_vw,     &ctx->s_scale,    &ctx->s_vol,
                 &ctx->s_dvol, &ctx->s_out_motion, &ctx->s_out_P, &ctx->s_out_proj,
                 &ctx->s_theta, &ctx->s_grad, &ctx->s_m1,       &ctx->s_m2,       &ctx->s_loss,
                 &ctx->s_nodes, &ctx->s_out_nodes, &ctx->probe, &ctx->blkimg};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  resolve_timing(ctx);
  for (cudaEvent_t e : ctx->spare) cudaEventDestroy(e);
  delete ctx;
}

const char* bp_last_error(const bp_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

long long bp_ctx_workspace_bytes(const bp_ctx* ctx) {
  if (!ctx) return 0;
  const Buf* bufs[] = {&ctx->geom,   &ctx->grad,   &ctx->partials,   &ctx->shblk,      &ctx->fdk_tab,
                       &ctx->s_proj,
                       &ctx->s_P,    &ctx->s_motion, &ctx->s_vw,     &ctx->s_scale,    &ctx->s_vol,
                       &ctx->s_dvol, &ctx->s_out_motion, &ctx->s_out_P, &ctx->s_out_proj,
                       &ctx->s_theta, &ctx->s_grad, &ctx->s_m1,       &ctx->s_m2,       &ctx->s_loss,
                       &ctx->s_nodes, &ctx->s_out_nodes, &ctx->probe, &ctx->blkimg};
  long long t = 0;
  for (const Buf* b : bufs) t += (long long)b->n;
  return t;
}

int bp_ctx_set_timing(bp_ctx* ctx, int enable) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  resolve_timing(ctx);
  for (int k = 0; k < K_COUNT; ++k) {
    ctx->total_ms[k] = 0.0;
    ctx->count[k] = 0;
  }
  ctx->timing = enable != 0;
  return BP_OK;
}

int bp_ctx_timing(bp_ctx* ctx, const char* kernel, double* total_ms, long long* launches) {
  if (!ctx || !kernel) return BP_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  resolve_timing(ctx);
  for (int k = 0; k < K_COUNT; ++k)
    if (std::strcmp(kernel, kKernelNames[k]) == 0) {
      if (total_ms) *total_ms = ctx->total_ms[k];
      if (launches) *launches = ctx->count[k];
      return BP_OK;
    }
  return fail(ctx, BP_ERR_INVALID_ARG, std::string("unknown kernel name ") + kernel);
}

long long bp_ctx_launch_count(const bp_ctx* ctx) { return ctx ? ctx->launches : 0; }

int bp_probe(bp_ctx* ctx, int kind, double* result, void* stream) {
  if (!ctx || !result || kind < 0 || kind > 3) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "bp_probe");
  const long long words = 16LL << 20;  // 64 MiB of scratch for the atomics
  CK(ensure(ctx->probe, (size_t)words * 4), "bp_probe: scratch");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(ctx->probe.p, 0, (size_t)words * 4, s), "bp_probe: clear");
  CK(bpk::run_probe(kind, (float*)ctx->probe.p, words, sms, result, s), "bp_probe");
  return BP_OK;
}

int bp_bounds_check(bp_ctx* ctx, int op, unsigned int* flags, long long* first_failure) {
  if (!ctx || !flags || !first_failure || op < 0 || op > 2) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  const cudaError_t e = bpk::bounds_status(flags, first_failure, op, nullptr);
  if (e == cudaErrorNotSupported)
    return fail(ctx, BP_ERR_UNSUPPORTED, "bp_bounds_check: library built without BP_BOUNDS_CHECK");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_bounds_check");
  return BP_OK;
}

int bp_compose(bp_ctx* ctx, int nviews, const double* P, const double* motion, double* Phat,
               void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  if (nviews < 0 || (nviews > 0 && (!P || !Phat)))
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_compose: nviews < 0 or NULL P/Phat");
  if (nviews == 0) return BP_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const void* q;
  CK(stage_in(ctx->s_P, P, sizeof(double) * 12 * nviews, s, &q), "copy P");
  const double* dP = (const double*)q;
  CK(stage_in(ctx->s_motion, motion, sizeof(double) * 6 * nviews, s, &q), "copy motion");
  const double* dm = (const double*)q;
  void* o;
  bool host;
  CK(stage_out(ctx->s_out_P, Phat, sizeof(double) * 12 * nviews, &o, &host), "alloc Phat");
  VolInfo vi{};
  CK(TL(K_COMPOSE, 1, bpk::launch_compose(dP, dm, nullptr, nullptr, nviews, 0, 0.0, vi, nullptr,
                                          (double*)o, s)),
     "compose");
  if (host) {
    CK(cudaMemcpyAsync(Phat, o, sizeof(double) * 12 * nviews, cudaMemcpyDeviceToHost, s),
       "copy Phat");
    CK(cudaStreamSynchronize(s), "sync");
  }
  return BP_OK;
}

int bp_forward(bp_ctx* ctx, const void* proj, const bp_proj_desc* pdesc, const double* P,
               const double* motion, const double* view_weight, int weight,
               const bp_vol_desc* vdesc, float* vol, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_proj(ctx, pdesc);
  if (st) return st;
  st = check_vol(ctx, vdesc);
  if (st) return st;
  if (weight != BP_WEIGHT_NONE && weight != BP_WEIGHT_FDK)
    return fail(ctx, BP_ERR_INVALID_ARG, "unknown weight mode");
  const long long nvox = (long long)vdesc->nx * vdesc->ny * vdesc->nz;
  if (nvox > 0 && !vol) return fail(ctx, BP_ERR_INVALID_ARG, "vol is NULL");
  if (pdesc->nviews > 0 && (!proj || !P))
    return fail(ctx, BP_ERR_INVALID_ARG, "proj or P is NULL");
  if (nvox == 0) return BP_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  void* dvol;
  bool host_vol;
  CK(stage_out(ctx->s_vol, vol, sizeof(float) * nvox, &dvol, &host_vol), "alloc vol");
  if (pdesc->nviews == 0) {
    CK(cudaMemsetAsync(dvol, 0, sizeof(float) * nvox, s), "zero vol");
  } else {
    const VolInfo vi = make_volinfo(vdesc, ZB);
    const void* dproj;
    CK(stage_in(ctx->s_proj, proj, proj_bytes(pdesc), s, &dproj), "copy proj");
    const double *dP, *dm;
    st = prepare_views(ctx, pdesc, P, motion, view_weight, weight, vi, s, &dP, &dm);
    if (st) return st;
    CK(TL(K_FORWARD, 1, bpk::launch_forward(dproj, pdesc->dtype, make_projinfo(pdesc),
                                          (const ViewGeom*)ctx->geom.p, vi,
                                          weight == BP_WEIGHT_FDK, (float*)dvol, s)),
       "forward kernel");
  }
  if (host_vol) {
    CK(cudaMemcpyAsync(vol, dvol, sizeof(float) * nvox, cudaMemcpyDeviceToHost, s), "copy vol");
    CK(cudaStreamSynchronize(s), "sync");
  }
  return BP_OK;
}

int bp_vjp(bp_ctx* ctx, const float* dL_dvol, const void* proj, const bp_proj_desc* pdesc,
           const double* P, const double* motion, const double* view_weight, int weight,
           int deriv, const bp_vol_desc* vdesc, double* dL_dmotion, double* dL_dPhat,
           float* dL_dproj, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_proj(ctx, pdesc);
  if (st) return st;
  st = check_vol(ctx, vdesc);
  if (st) return st;
  if (weight != BP_WEIGHT_NONE && weight != BP_WEIGHT_FDK)
    return fail(ctx, BP_ERR_INVALID_ARG, "unknown weight mode");
  if (deriv != BP_DERIV_CENTRAL && deriv != BP_DERIV_BILINEAR_EXACT)
    return fail(ctx, BP_ERR_INVALID_ARG, "unknown derivative mode");
  const int V = pdesc->nviews;
  const long long nvox = (long long)vdesc->nx * vdesc->ny * vdesc->nz;
  const bool want_geo = dL_dmotion || dL_dPhat;
  if (!want_geo && !dL_dproj) return BP_OK;
  if (V > 0 && (!P || (want_geo && !proj))) return fail(ctx, BP_ERR_INVALID_ARG, "proj or P is NULL");
  if (nvox > 0 && !dL_dvol) return fail(ctx, BP_ERR_INVALID_ARG, "dL_dvol is NULL");
  if (V == 0) return BP_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const VolInfo vi = make_volinfo(vdesc, ZB);
  const ProjInfo pi = make_projinfo(pdesc);
  const int ntiles = vi.tiles_x * vi.tiles_y * vi.tiles_z;
  const void* q;
  CK(stage_in(ctx->s_dvol, dL_dvol, sizeof(float) * nvox, s, &q), "copy dL_dvol");
  const float* ddvol = (const float*)q;
  const void* dproj = nullptr;
  if (want_geo) CK(stage_in(ctx->s_proj, proj, proj_bytes(pdesc), s, &dproj), "copy proj");
  const double *dP, *dm;
  st = prepare_views(ctx, pdesc, P, motion, view_weight, weight, vi, s, &dP, &dm);
  if (st) return st;
  void *om = nullptr, *oP = nullptr, *oD = nullptr;
  bool hm = false, hP = false, hD = false;
  CK(stage_out(ctx->s_out_motion, dL_dmotion, sizeof(double) * 6 * V, &om, &hm), "alloc out");
  CK(stage_out(ctx->s_out_P, dL_dPhat, sizeof(double) * 12 * V, &oP, &hP), "alloc out");
  const size_t dproj_bytes = sizeof(float) * (size_t)V * pdesc->nv * pdesc->nu;
  CK(stage_out(ctx->s_out_proj, dL_dproj, dproj_bytes, &oD, &hD), "alloc out");
  // the data VJP is fused into the motion-VJP kernel when both are wanted
  const bool fuse = want_geo && dL_dproj && nvox > 0;
  if (dL_dproj) CK(cudaMemsetAsync(oD, 0, dproj_bytes, s), "zero dL_dproj");
  if (want_geo) {
    const float2* grad = nullptr;
    if (deriv == BP_DERIV_CENTRAL) {
      CK(ensure(ctx->grad, sizeof(float2) * (size_t)V * pdesc->nv * pdesc->nu), "alloc grad");
      CK(TL(K_GRAD, 1, bpk::launch_grad_images(dproj, pdesc->dtype, pi, (float2*)ctx->grad.p, s)),
         "grad images");
      grad = (const float2*)ctx->grad.p;
    }
    if (nvox > 0) {
      CK(ensure(ctx->partials, sizeof(float) * bpk::PSLOTS * (size_t)V * ntiles), "alloc partials");
      // the fused data VJP of staged CENTRAL tiles goes through a block
      // image (one vector reduction per sample), added into dL_dproj by a
      // second kernel of the same launch
      const bool blocks = fuse && bpk::vjp_uses_blocks(dproj, pdesc->dtype, pi,
                                                       deriv == BP_DERIV_BILINEAR_EXACT);
      if (blocks)
        CK(ensure(ctx->blkimg, sizeof(float) * (size_t)bpk::block_image_floats(pi)),
           "alloc block image");
      CK(TL(fuse ? K_VJP_FUSED : K_VJP_MOTION, blocks ? 2 : 1,
            bpk::launch_vjp_motion(ddvol, dproj, pdesc->dtype, pi, grad,
                                   (const ViewGeom*)ctx->geom.p, vi, weight == BP_WEIGHT_FDK,
                                   deriv == BP_DERIV_BILINEAR_EXACT, (float*)ctx->partials.p,
                                   fuse ? (float*)oD : nullptr,
                                   blocks ? (float*)ctx->blkimg.p : nullptr, s)),
         "vjp kernel");
    }
    CK(TL(K_REDUCE, 1, bpk::launch_reduce_chain((const float*)ctx->partials.p, nvox > 0 ? ntiles : 0,
                                              vi, dP, dm, V, (double*)oP, (double*)om, s)),
       "reduce kernel");
  }
  if (dL_dproj && !fuse && nvox > 0) {
    ProjInfo po = pi;
    po.rs = pdesc->nu;
    po.vs = (long long)pdesc->nu * pdesc->nv;
    const long long bf = bpk::block_image_floats(po);
    if (bf > 0) CK(ensure(ctx->blkimg, sizeof(float) * (size_t)bf), "alloc block image");
    CK(TL(K_VJP_PROJ, bf > 0 ? 2 : 1,
          bpk::launch_vjp_proj(ddvol, po, (const ViewGeom*)ctx->geom.p, vi,
                               weight == BP_WEIGHT_FDK, (float*)oD,
                               bf > 0 ? (float*)ctx->blkimg.p : nullptr, s)),
       "proj vjp kernel");
  }
  if (hm) CK(cudaMemcpyAsync(dL_dmotion, om, sizeof(double) * 6 * V, cudaMemcpyDeviceToHost, s), "copy out");
  if (hP) CK(cudaMemcpyAsync(dL_dPhat, oP, sizeof(double) * 12 * V, cudaMemcpyDeviceToHost, s), "copy out");
  if (hD) CK(cudaMemcpyAsync(dL_dproj, oD, dproj_bytes, cudaMemcpyDeviceToHost, s), "copy out");
  if (hm || hP || hD) CK(cudaStreamSynchronize(s), "sync");
  return BP_OK;
}

int bp_sharpness(bp_ctx* ctx, const float* vol, const bp_vol_desc* vdesc, double* loss,
                 float* dL_dvol, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_vol(ctx, vdesc);
  if (st) return st;
  const long long nvox = (long long)vdesc->nx * vdesc->ny * vdesc->nz;
  if (!loss) return fail(ctx, BP_ERR_INVALID_ARG, "loss is NULL");
  if (nvox > 0 && !vol) return fail(ctx, BP_ERR_INVALID_ARG, "vol is NULL");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (nvox == 0) {
    if (is_host(loss)) {
      *loss = 0.0;
      return BP_OK;
    }
    CK(cudaMemsetAsync(loss, 0, sizeof(double), s), "zero loss");
    return BP_OK;
  }
  const void* q;
  CK(stage_in(ctx->s_vol, vol, sizeof(float) * nvox, s, &q), "copy vol");
  void *ol, *og;
  bool hl, hg;
  CK(stage_out(ctx->s_loss, loss, sizeof(double), &ol, &hl), "alloc loss");
  CK(stage_out(ctx->s_dvol, dL_dvol, sizeof(float) * nvox, &og, &hg), "alloc grad");
  const int nb = bpk::sharpness_blocks(nvox);
  CK(ensure(ctx->shblk, sizeof(double) * nb), "alloc block sums");
  CK(TL(K_SHARPNESS, 2, bpk::launch_sharpness((const float*)q, vdesc->nx, vdesc->ny, vdesc->nz,
                                              (double*)ctx->shblk.p, nb, (double*)ol,
                                              (float*)og, s)),
     "sharpness kernel");
  if (hl) CK(cudaMemcpyAsync(loss, ol, sizeof(double), cudaMemcpyDeviceToHost, s), "copy loss");
  if (hg) CK(cudaMemcpyAsync(dL_dvol, og, sizeof(float) * nvox, cudaMemcpyDeviceToHost, s), "copy grad");
  if (hl || hg) CK(cudaStreamSynchronize(s), "sync");
  return BP_OK;
}

int bp_tv(bp_ctx* ctx, const float* vol, const bp_vol_desc* vdesc, double eps, double* loss,
          float* dL_dvol, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_vol(ctx, vdesc);
  if (st) return st;
  const long long nvox = (long long)vdesc->nx * vdesc->ny * vdesc->nz;
  if (!loss) return fail(ctx, BP_ERR_INVALID_ARG, "loss is NULL");
  if (nvox > 0 && !vol) return fail(ctx, BP_ERR_INVALID_ARG, "vol is NULL");
  if (!(eps > 0.0)) return fail(ctx, BP_ERR_INVALID_ARG, "eps must be > 0");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (nvox == 0) {
    if (is_host(loss)) {
      *loss = 0.0;
      return BP_OK;
    }
    CK(cudaMemsetAsync(loss, 0, sizeof(double), s), "zero loss");
    return BP_OK;
  }
  const void* q;
  CK(stage_in(ctx->s_vol, vol, sizeof(float) * nvox, s, &q), "copy vol");
  void *ol, *og;
  bool hl, hg;
  CK(stage_out(ctx->s_loss, loss, sizeof(double), &ol, &hl), "alloc loss");
  CK(stage_out(ctx->s_dvol, dL_dvol, sizeof(float) * nvox, &og, &hg), "alloc grad");
  const int nb = bpk::sharpness_blocks(nvox);
  CK(ensure(ctx->shblk, sizeof(double) * nb), "alloc block sums");
  CK(TL(K_SHARPNESS, 2, bpk::launch_tv((const float*)q, vdesc->nx, vdesc->ny, vdesc->nz,
                                       (float)eps, (double*)ctx->shblk.p, nb, (double*)ol,
                                       nullptr, 0, (float*)og, s)),
     "tv kernel");
  if (hl) CK(cudaMemcpyAsync(loss, ol, sizeof(double), cudaMemcpyDeviceToHost, s), "copy loss");
  if (hg) CK(cudaMemcpyAsync(dL_dvol, og, sizeof(float) * nvox, cudaMemcpyDeviceToHost, s), "copy grad");
  if (hl || hg) CK(cudaStreamSynchronize(s), "sync");
  return BP_OK;
}

}  // extern "C"

namespace {

// Run an in-place optimiser update on theta (and moments) that may live on
// the host: copy in, update, copy back.
template <typename F>
int opt_step(bp_ctx* ctx, int V, double* theta, const double* grad, double* m1, double* m2,
             cudaStream_t s, F launch) {
  const size_t b = sizeof(double) * 6 * V;
  double* dt = theta;
  double* dm1 = m1;
  double* dm2 = m2;
  const bool ht = is_host(theta), h1 = m1 && is_host(m1), h2 = m2 && is_host(m2);
  const void* q;
  CK(stage_in(ctx->s_grad, grad, b, s, &q), "copy grad");
  if (ht) {
    CK(ensure(ctx->s_theta, b), "alloc");
    CK(cudaMemcpyAsync(ctx->s_theta.p, theta, b, cudaMemcpyHostToDevice, s), "copy theta");
    dt = (double*)ctx->s_theta.p;
  }
  if (h1) {
    CK(ensure(ctx->s_m1, b), "alloc");
    CK(cudaMemcpyAsync(ctx->s_m1.p, m1, b, cudaMemcpyHostToDevice, s), "copy m1");
    dm1 = (double*)ctx->s_m1.p;
  }
  if (h2) {
    CK(ensure(ctx->s_m2, b), "alloc");
    CK(cudaMemcpyAsync(ctx->s_m2.p, m2, b, cudaMemcpyHostToDevice, s), "copy m2");
    dm2 = (double*)ctx->s_m2.p;
  }
  CK(launch(dt, (const double*)q, dm1, dm2), "optimiser kernel");
  if (ht) CK(cudaMemcpyAsync(theta, dt, b, cudaMemcpyDeviceToHost, s), "copy theta");
  if (h1) CK(cudaMemcpyAsync(m1, dm1, b, cudaMemcpyDeviceToHost, s), "copy m1");
  if (h2) CK(cudaMemcpyAsync(m2, dm2, b, cudaMemcpyDeviceToHost, s), "copy m2");
  if (ht || h1 || h2) CK(cudaStreamSynchronize(s), "sync");
  return BP_OK;
}

}  // namespace

extern "C" {

int bp_gd_step(bp_ctx* ctx, int nviews, double* theta, const double* grad, double s0, double t,
               int n, int gauge, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  if (nviews < 0 || (nviews > 0 && (!theta || !grad)))
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_gd_step: bad arguments");
  if (nviews == 0) return BP_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  return opt_step(ctx, nviews, theta, grad, nullptr, nullptr, s,
                  [&](double* th, const double* gr, double*, double*) {
                    return TL(K_OPT, 1, bpk::launch_gd(nviews, th, gr, s0, t, n, gauge, s));
                  });
}

int bp_adam_step(bp_ctx* ctx, int nviews, double* theta, const double* grad, double* m1,
                 double* m2, double lr, double beta1, double beta2, double eps, int n, int gauge,
                 void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  if (nviews < 0 || (nviews > 0 && (!theta || !grad || !m1 || !m2)) || n < 1)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_adam_step: bad arguments");
  if (nviews == 0) return BP_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  return opt_step(ctx, nviews, theta, grad, m1, m2, s,
                  [&](double* th, const double* gr, double* a, double* b) {
                    return TL(K_OPT, 1, bpk::launch_adam(nviews, th, gr, a, b, lr, beta1, beta2, eps, n,
                                                         gauge, s));
                  });
}

static int check_spline(bp_ctx* ctx, int n_nodes, int nviews) {
  if (n_nodes < 3 || nviews < 2)
    return fail(ctx, BP_ERR_INVALID_ARG, "Akima motion: need n_nodes >= 3 and nviews >= 2");
  if (n_nodes > bpk::AKIMA_MAX_NODES)
    return fail(ctx, BP_ERR_UNSUPPORTED, "Akima motion: more than 512 nodes");
  return BP_OK;
}

int bp_akima_motion(bp_ctx* ctx, int n_nodes, int nviews, const double* nodes, double* theta,
                    void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_spline(ctx, n_nodes, nviews);
  if (st) return st;
  if (!nodes || !theta) return fail(ctx, BP_ERR_INVALID_ARG, "bp_akima_motion: NULL array");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const void* q;
  CK(stage_in(ctx->s_nodes, nodes, sizeof(double) * 6 * n_nodes, s, &q), "copy nodes");
  void* o;
  bool host;
  CK(stage_out(ctx->s_out_motion, theta, sizeof(double) * 6 * nviews, &o, &host), "alloc theta");
  CK(TL(K_SPLINE, 1, bpk::launch_akima_eval(n_nodes, nviews, (const double*)q, (double*)o, s)),
     "akima");
  if (host) {
    CK(cudaMemcpyAsync(theta, o, sizeof(double) * 6 * nviews, cudaMemcpyDeviceToHost, s),
       "copy theta");
    CK(cudaStreamSynchronize(s), "sync");
  }
  return BP_OK;
}

int bp_akima_motion_vjp(bp_ctx* ctx, int n_nodes, int nviews, const double* nodes,
                        const double* dL_dtheta, double* dL_dnodes, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  int st = check_spline(ctx, n_nodes, nviews);
  if (st) return st;
  if (!nodes || !dL_dtheta || !dL_dnodes)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_akima_motion_vjp: NULL array");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const void* q;
  CK(stage_in(ctx->s_nodes, nodes, sizeof(double) * 6 * n_nodes, s, &q), "copy nodes");
  const double* dn = (const double*)q;
  CK(stage_in(ctx->s_grad, dL_dtheta, sizeof(double) * 6 * nviews, s, &q), "copy dL/dtheta");
  void* o;
  bool host;
  CK(stage_out(ctx->s_out_nodes, dL_dnodes, sizeof(double) * 6 * n_nodes, &o, &host),
     "alloc dL/dnodes");
  CK(TL(K_SPLINE, 1, bpk::launch_akima_vjp(n_nodes, nviews, dn, (const double*)q, (double*)o, s)),
     "akima vjp");
  if (host) {
    CK(cudaMemcpyAsync(dL_dnodes, o, sizeof(double) * 6 * n_nodes, cudaMemcpyDeviceToHost, s),
       "copy dL/dnodes");
    CK(cudaStreamSynchronize(s), "sync");
  }
  return BP_OK;
}

int bp_fdk_filter(bp_ctx* ctx, const float* raw, int nviews, int nv, int nu, double pitch,
                  double sid, double sdd, double arc, int ext, float* out, void* stream) {
  if (!ctx) return BP_ERR_INVALID_ARG;
  ctx->err.clear();
  if (nviews < 0 || nv < 0 || nu < 1 || ext < 0)
    return fail(ctx, BP_ERR_INVALID_ARG,
                "bp_fdk_filter: nviews, nv, ext >= 0 and nu >= 1 needed");
  if ((long long)nu + 2LL * ext > bpk::FDK_MAX_NU)
    return fail(ctx, BP_ERR_UNSUPPORTED, "bp_fdk_filter: nu + 2 ext > 8192");
  if (!(pitch > 0.0) || !(sid > 0.0) || !(sdd > 0.0) || !(arc > 0.0))
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_fdk_filter: pitch, sid, sdd, arc must be > 0");
  if (arc < 2.0 * 3.14159265358979323846 && nviews > 1 && 0.5 * (arc - 3.14159265358979323846) <=
                                                          atan(0.5 * (nu - 1) * pitch / sdd))
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_fdk_filter: short-scan arc below pi + fan angle");
  const size_t n = (size_t)nviews * nv * nu;
  if (n == 0) return BP_OK;
  if (!raw || !out) return fail(ctx, BP_ERR_INVALID_ARG, "bp_fdk_filter: NULL array");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const void* q;
  CK(stage_in(ctx->s_proj, raw, sizeof(float) * n, s, &q), "copy raw");
  void* o;
  bool host;
  CK(stage_out(ctx->s_out_proj, out, sizeof(float) * n, &o, &host), "alloc out");
  CK(ensure(ctx->fdk_tab, sizeof(float) * bpk::fdk_table_floats(nviews, nu, ext)),
     "alloc tables");
  CK(TL(K_FDK, 2, bpk::launch_fdk_filter((const float*)q, nviews, nv, nu, ext, pitch, sid, sdd,
                                         arc, (float*)ctx->fdk_tab.p, (float*)o, s)),
     "fdk filter");
  if (host) {
    CK(cudaMemcpyAsync(out, o, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "copy out");
    CK(cudaStreamSynchronize(s), "sync");
  }
  return BP_OK;
}

}  // extern "C"
