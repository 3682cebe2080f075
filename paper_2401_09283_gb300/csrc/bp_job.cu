// Motion-estimation jobs (C-ABI in include/bp_gb300.h): device-resident
// state and one captured CUDA graph per iteration of the gradient-based
// motion estimation of Sec. II-C (compose -> backprojection -> loss -> VJP ->
// FP64 reduction and chain rule -> optimiser update).
#include <algorithm>
#include <chrono>
#include <thread>

#include "bp_ctx.h"

using namespace bpctx;

struct bp_job {
  bp_ctx* ctx = nullptr;
  int device = 0;
  bp_proj_desc pd{};
  bp_vol_desc vd{};
  bp_opt_desc opt{};
  int weight = 0, deriv = 0, max_iters = 0;
  bpk::VolInfo vi{};
  bpk::ProjInfo pi{};
  int ntiles = 0, nblk = 0;
  void* base = nullptr;  // one allocation, carved below
  void* proj = nullptr;
  float* scale = nullptr;
  double *P = nullptr, *vw = nullptr, *theta = nullptr, *m1 = nullptr, *m2 = nullptr,
         *gth = nullptr, *blk = nullptr, *hist = nullptr;
  int nodes = 0;                               // Akima motion model: N_n (0: per view)
  double *x = nullptr, *gx = nullptr;          // node values and their gradient [N_n][6]
  bpk::ViewGeom* geom = nullptr;
  float2* grad = nullptr;
  float *partials = nullptr, *vol = nullptr, *dvol = nullptr;
  int* iter = nullptr;
  long long bytes = 0;
  cudaStream_t own = nullptr;   // the job's stream: allocation, copies, read-back
  cudaEvent_t done = nullptr;   // recorded after the last queued iteration
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool cancelled = false;
  int queued = 0;               // iterations queued so far (motion_step or batches)
  bp_batch* batch = nullptr;    // the batch this job is a member of, if any
};

struct bp_batch {
  bp_ctx* ctx = nullptr;
  int device = 0, sms = 0, max_jobs = 0;
  std::vector<bp_job*> members;
  bool dirty = true;                // the member set changed since the graph was made
  bpk::BatchTable table{};          // the graph's member table (a kernel parameter)
  unsigned* counter = nullptr;      // the persistent forward's work counter (device)
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t last = nullptr;       // after the latest queued step
  // branches of the VJP stage: a stream and a join event per member
  std::vector<cudaStream_t> br_streams;
  std::vector<cudaEvent_t> br_joins;
  cudaEvent_t br_fork = nullptr;
  struct Retired {                  // graphs of earlier member sets, freed once idle
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaEvent_t done;
  };
  std::vector<Retired> retired;
};

namespace {

constexpr int ZB = bpk::ZB_VJP;
constexpr long long kAlign = 256;

long long align_up(long long x) { return (x + kAlign - 1) / kAlign * kAlign; }

// The job's buffers in allocation order (sizes in bytes).
struct Layout {
  long long proj, scale, P, vw, theta, m1, m2, gth, x, gx, geom, grad, partials, vol, dvol, blk,
      hist, iter, total;
};

Layout layout(const bp_proj_desc* pd, const bp_vol_desc* vd, int deriv, int max_iters) {
  Layout L;
  const long long V = pd->nviews, npx = (long long)pd->nu * pd->nv;
  const long long nvox = (long long)vd->nx * vd->ny * vd->nz;
  const long long tiles = (long long)((vd->nx + 15) / 16) * ((vd->ny + 15) / 16) * ((vd->nz + ZB - 1) / ZB);
  L.proj = align_up(V * npx * (pd->dtype == BP_F32 ? 4 : 2));
  L.scale = align_up(V * 4);
  L.P = align_up(V * 96);
  L.vw = align_up(V * 8);
  L.theta = L.gth = align_up(V * 48);
  // optimiser state holds either V per-view rows or up to AKIMA_MAX_NODES
  // node rows; node buffers are always reserved, so the size does not
  // depend on the motion model
  L.m1 = L.m2 = align_up((V > bpk::AKIMA_MAX_NODES ? V : bpk::AKIMA_MAX_NODES) * 48LL);
  L.x = L.gx = align_up(bpk::AKIMA_MAX_NODES * 48LL);
  L.geom = align_up(V * (long long)sizeof(bpk::ViewGeom));
  L.grad = deriv == BP_DERIV_CENTRAL ? align_up(V * npx * 8) : 0;
  L.partials = align_up(V * tiles * bpk::PSLOTS * 4);
  L.vol = L.dvol = align_up(nvox * 4);
  L.blk = align_up(bpk::sharpness_blocks(nvox) * 8LL);
  L.hist = align_up((long long)max_iters * 8);
  L.iter = kAlign;
  L.total = L.proj + L.scale + L.P + L.vw + L.theta + L.gth + L.m1 + L.m2 + L.x + L.gx + L.geom +
            L.grad + L.partials + 2 * L.vol + L.blk + L.hist + L.iter;
  return L;
}

// Free everything without a device-wide synchronisation: other jobs keep
// running (stream-ordered free after the job's last queued iteration).
void release(bp_job* j) {
  if (j->own && j->done) cudaStreamWaitEvent(j->own, j->done, 0);
  if (j->base) cudaFreeAsync(j->base, j->own);
  if (j->own) cudaStreamSynchronize(j->own);
  if (j->exec) cudaGraphExecDestroy(j->exec);
  if (j->graph) cudaGraphDestroy(j->graph);
  if (j->cap) cudaStreamDestroy(j->cap);
  if (j->done) cudaEventDestroy(j->done);
  if (j->own) cudaStreamDestroy(j->own);
  j->exec = nullptr;
  j->graph = nullptr;
  j->cap = nullptr;
  j->base = nullptr;
  j->done = nullptr;
  j->own = nullptr;
}

// Record one iteration on stream s.
cudaError_t record_iteration(bp_job* j, cudaStream_t s) {
  const int fdk = j->weight == BP_WEIGHT_FDK;
  const int V = j->pd.nviews;
  cudaError_t e;
  if (j->nodes) {
    e = bpk::launch_akima_eval(j->nodes, V, j->x, j->theta, s);
    if (e != cudaSuccess) return e;
  }
  e = bpk::launch_compose(j->P, j->theta, j->vw, j->scale, V, fdk, j->pd.sid, j->vi, j->geom,
                          nullptr, s);
  if (e != cudaSuccess) return e;
  e = bpk::launch_forward(j->proj, j->pd.dtype, j->pi, j->geom, j->vi, fdk, j->vol, s);
  if (e != cudaSuccess) return e;
  if (j->opt.loss == BP_LOSS_TV)
    e = bpk::launch_tv(j->vol, j->vd.nx, j->vd.ny, j->vd.nz, (float)j->opt.tv_eps, j->blk, j->nblk,
                       j->hist, j->iter, j->max_iters, j->dvol, s);
  else
    e = bpk::launch_sharpness_hist(j->vol, j->vd.nx, j->vd.ny, j->vd.nz, j->blk, j->nblk,
                                   j->hist, j->iter, j->max_iters, j->dvol, s);
  if (e != cudaSuccess) return e;
  e = bpk::launch_vjp_motion(j->dvol, j->proj, j->pd.dtype, j->pi, j->grad, j->geom, j->vi, fdk,
                             j->deriv == BP_DERIV_BILINEAR_EXACT, j->partials, nullptr, nullptr, s);
  if (e != cudaSuccess) return e;
  e = bpk::launch_reduce_chain(j->partials, j->ntiles, j->vi, j->P, j->theta, V, nullptr, j->gth,
                               s);
  if (e != cudaSuccess) return e;
  // the optimiser's variables: per-view theta, or the spline nodes
  int rows = V;
  double *var = j->theta, *grad = j->gth;
  if (j->nodes) {
    e = bpk::launch_akima_vjp(j->nodes, V, j->x, j->gth, j->gx, s);
    if (e != cudaSuccess) return e;
    rows = j->nodes;
    var = j->x;
    grad = j->gx;
  }
  if (j->opt.optimizer == BP_OPT_ADAM)
    return bpk::launch_adam_dev(rows, var, grad, j->m1, j->m2, j->opt.lr, j->opt.lr_rot,
                                j->opt.beta1, j->opt.beta2, j->opt.eps, j->iter, j->opt.gauge, s);
  return bpk::launch_gd_dev(rows, var, grad, j->opt.lr, j->opt.lr_rot, j->opt.decay, j->iter,
                            j->opt.gauge, s);
}

// compose, forward, 2 loss, VJP, reduce, update (+ spline and its VJP)
int kernels_per_iteration(const bp_job* j) { return j->nodes ? 9 : 7; }

}  // namespace

extern "C" {

long long bp_job_bytes_for(const bp_proj_desc* pdesc, const bp_vol_desc* vdesc, int deriv,
                           int max_iters) {
  if (!pdesc || !vdesc || max_iters < 0) return -1;
  return layout(pdesc, vdesc, deriv, max_iters).total;
}

long long bp_job_bytes(const bp_job* job) { return job ? job->bytes : 0; }

int bp_ctx_set_hbm_budget(bp_ctx* ctx, long long bytes) {
  if (!ctx || bytes < 0) return BP_ERR_INVALID_ARG;
  ctx->hbm_budget = bytes;
  return BP_OK;
}

int bp_job_create(bp_ctx* ctx, const void* proj, const bp_proj_desc* pdesc, const double* P,
                  const double* view_weight, int weight, int deriv, const bp_vol_desc* vdesc,
                  const bp_opt_desc* opt, const double* theta0, int max_iters, bp_job** out) {
  if (!ctx || !out) return BP_ERR_INVALID_ARG;
  *out = nullptr;
  ctx->err.clear();
  if (!pdesc || !vdesc || !opt || !proj || !P)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_job_create: NULL argument");
  if (pdesc->nu < 1 || pdesc->nv < 1 || pdesc->nviews < 1 || vdesc->nx < 1 || vdesc->ny < 1 ||
      vdesc->nz < 1 || max_iters < 0)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_job_create: empty problem or negative max_iters");
  if (pdesc->dtype != BP_F32 && pdesc->dtype != BP_F16 && pdesc->dtype != BP_BF16)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_job_create: unknown dtype");
  if (pdesc->row_stride < pdesc->nu || pdesc->view_stride < (long long)pdesc->nv * pdesc->row_stride)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_job_create: bad strides");
  if ((weight != BP_WEIGHT_NONE && weight != BP_WEIGHT_FDK) ||
      (deriv != BP_DERIV_CENTRAL && deriv != BP_DERIV_BILINEAR_EXACT) ||
      (opt->optimizer != BP_OPT_GD && opt->optimizer != BP_OPT_ADAM) ||
      (opt->loss != BP_LOSS_SHARPNESS && opt->loss != BP_LOSS_TV) ||
      (opt->loss == BP_LOSS_TV && !(opt->tv_eps > 0.0)))
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_job_create: unknown weight/deriv/optimizer/loss");
  if (opt->motion_nodes != 0 &&
      (opt->motion_nodes < 3 || opt->motion_nodes > bpk::AKIMA_MAX_NODES || pdesc->nviews < 2))
    return fail(ctx, BP_ERR_INVALID_ARG,
                "bp_job_create: motion_nodes must be 0 or 3..512 (with >= 2 views)");
  DeviceGuard g(ctx->device);
  const Layout L = layout(pdesc, vdesc, deriv, max_iters);
  // admission by device memory
  long long avail;
  if (ctx->hbm_budget > 0) {
    avail = ctx->hbm_budget - ctx->job_bytes;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "meminfo");
    avail = (long long)fr - (256LL << 20);
  }
  if (L.total > avail)
    return fail(ctx, BP_ERR_OOM, "bp_job_create: job needs " + std::to_string(L.total) +
                                     " bytes, " + std::to_string(avail > 0 ? avail : 0) +
                                     " available under the budget");
  bp_job* j = new bp_job();
  j->ctx = ctx;
  j->device = ctx->device;
  j->pd = *pdesc;
  j->vd = *vdesc;
  j->opt = *opt;
  j->weight = weight;
  j->deriv = deriv;
  j->max_iters = max_iters;
  j->bytes = L.total;
  cudaError_t e = cudaStreamCreateWithFlags(&j->own, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocAsync(&j->base, (size_t)L.total, j->own);
  if (e != cudaSuccess) {
    release(j);
    delete j;
    return cuda_fail(ctx, e, "bp_job_create: allocation");
  }
  cudaStream_t os = j->own;
  char* p = (char*)j->base;
  auto take = [&](long long n) {
    char* q = p;
    p += n;
    return (void*)q;
  };
  j->proj = take(L.proj);
  j->scale = (float*)take(L.scale);
  j->P = (double*)take(L.P);
  j->vw = (double*)take(L.vw);
  j->theta = (double*)take(L.theta);
  j->m1 = (double*)take(L.m1);
  j->m2 = (double*)take(L.m2);
  j->gth = (double*)take(L.gth);
  j->x = (double*)take(L.x);
  j->gx = (double*)take(L.gx);
  j->nodes = opt->motion_nodes;
  j->geom = (bpk::ViewGeom*)take(L.geom);
  j->grad = L.grad ? (float2*)take(L.grad) : nullptr;
  j->partials = (float*)take(L.partials);
  j->vol = (float*)take(L.vol);
  j->dvol = (float*)take(L.dvol);
  j->blk = (double*)take(L.blk);
  j->hist = (double*)take(L.hist);
  j->iter = (int*)take(L.iter);
  const int V = pdesc->nviews;
  const size_t es = pdesc->dtype == BP_F32 ? 4 : 2;
  // inputs (host or device: cudaMemcpyDefault under unified addressing)
  if (pdesc->view_stride == (long long)pdesc->nv * pdesc->row_stride) {
    e = cudaMemcpy2DAsync(j->proj, es * pdesc->nu, proj, es * pdesc->row_stride, es * pdesc->nu,
                          (size_t)pdesc->nv * V, cudaMemcpyDefault, os);
  } else {
    for (int v = 0; v < V && e == cudaSuccess; ++v)
      e = cudaMemcpy2DAsync((char*)j->proj + es * (size_t)v * pdesc->nu * pdesc->nv,
                            es * pdesc->nu, (const char*)proj + es * (size_t)v * pdesc->view_stride,
                            es * pdesc->row_stride, es * pdesc->nu, (size_t)pdesc->nv,
                            cudaMemcpyDefault, os);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(j->P, P, 96 * (size_t)V, cudaMemcpyDefault, os);
  if (e == cudaSuccess) {
    if (view_weight) e = cudaMemcpyAsync(j->vw, view_weight, 8 * (size_t)V, cudaMemcpyDefault, os);
    else j->vw = nullptr;
  }
  if (e == cudaSuccess) {
    if (pdesc->view_scale)
      e = cudaMemcpyAsync(j->scale, pdesc->view_scale, 4 * (size_t)V, cudaMemcpyDefault, os);
    else j->scale = nullptr;
  }
  if (e == cudaSuccess) {
    double* init = j->nodes ? j->x : j->theta;
    const size_t rows = j->nodes ? (size_t)j->nodes : (size_t)V;
    if (theta0) e = cudaMemcpyAsync(init, theta0, 48 * rows, cudaMemcpyDefault, os);
    else e = cudaMemsetAsync(init, 0, 48 * rows, os);
    if (e == cudaSuccess && j->nodes) e = cudaMemsetAsync(j->theta, 0, 48 * (size_t)V, os);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(j->m1, 0, (size_t)L.m1, os);
  if (e == cudaSuccess) e = cudaMemsetAsync(j->m2, 0, (size_t)L.m2, os);
  if (e == cudaSuccess) e = cudaMemsetAsync(j->iter, 0, sizeof(int), os);
  if (e == cudaSuccess && max_iters > 0) e = cudaMemsetAsync(j->hist, 0, 8 * (size_t)max_iters, os);
  j->pd.row_stride = pdesc->nu;
  j->pd.view_stride = (long long)pdesc->nu * pdesc->nv;
  j->pd.view_scale = j->scale;
  j->vi.nx = vdesc->nx;
  j->vi.ny = vdesc->ny;
  j->vi.nz = vdesc->nz;
  j->vi.zb = ZB;
  j->vi.tiles_x = (vdesc->nx + 15) / 16;
  j->vi.tiles_y = (vdesc->ny + 15) / 16;
  j->vi.tiles_z = (vdesc->nz + ZB - 1) / ZB;
  j->vi.cx = 0.5 * (vdesc->nx - 1);
  j->vi.cy = 0.5 * (vdesc->ny - 1);
  j->vi.cz = 0.5 * (vdesc->nz - 1);
  const double c[3] = {j->vi.cx, j->vi.cy, j->vi.cz};
  for (int k = 0; k < 12; ++k) j->vi.A[k] = 0.0;
  for (int a = 0; a < 3; ++a) {
    j->vi.A[4 * a + a] = vdesc->spacing[a];
    j->vi.A[4 * a + 3] = vdesc->origin[a] + c[a] * vdesc->spacing[a];
  }
  j->pi.nu = pdesc->nu;
  j->pi.nv = pdesc->nv;
  j->pi.nviews = V;
  j->pi.rs = pdesc->nu;
  j->pi.vs = (long long)pdesc->nu * pdesc->nv;
  j->ntiles = j->vi.tiles_x * j->vi.tiles_y * j->vi.tiles_z;
  j->nblk = bpk::sharpness_blocks((long long)vdesc->nx * vdesc->ny * vdesc->nz);
  if (e == cudaSuccess && j->grad) {
    e = bpk::launch_grad_images(j->proj, pdesc->dtype, j->pi, j->grad, os);
    ctx->launches += 1;
  }
  if (e == cudaSuccess) e = bpk::prepare_forward(pdesc->dtype, weight == BP_WEIGHT_FDK);
  if (e == cudaSuccess)
    e = bpk::prepare_vjp(pdesc->dtype, weight == BP_WEIGHT_FDK, deriv == BP_DERIV_BILINEAR_EXACT);
  if (e == cudaSuccess) e = cudaEventRecord(j->done, os);
  if (e == cudaSuccess) e = cudaStreamSynchronize(os);
  if (e != cudaSuccess) {
    release(j);
    delete j;
    return cuda_fail(ctx, e, "bp_job_create");
  }
  ctx->job_bytes += j->bytes;
  *out = j;
  return BP_OK;
}

int motion_step(bp_job* j, int n_iters, void* stream) {
  if (!j || n_iters < 0) return BP_ERR_INVALID_ARG;
  bp_ctx* ctx = j->ctx;
  ctx->err.clear();
  if (j->cancelled) return fail(ctx, BP_ERR_CANCELLED, "motion_step: the job was cancelled");
  if (j->batch)
    return fail(ctx, BP_ERR_INVALID_ARG, "motion_step: the job is a member of a batch");
  if (n_iters == 0) return BP_OK;
  DeviceGuard g(j->device);
  if (!j->exec) {
    cudaError_t e = cudaStreamCreateWithFlags(&j->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(j->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "motion_step: capture");
    cudaError_t le = record_iteration(j, j->cap);
    e = cudaStreamEndCapture(j->cap, &j->graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&j->exec, j->graph, 0);
    if (e != cudaSuccess) {
      if (j->graph) cudaGraphDestroy(j->graph);
      j->graph = nullptr;
      j->exec = nullptr;
      return cuda_fail(ctx, e, "motion_step: graph");
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the first replay waits for the job's set-up and any earlier read-back
  cudaError_t e = cudaStreamWaitEvent(s, j->done, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "motion_step: wait");
  for (int i = 0; i < n_iters; ++i) {
    e = cudaGraphLaunch(j->exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "motion_step: launch");
  }
  ctx->launches += (long long)kernels_per_iteration(j) * n_iters;
  j->queued += n_iters;
  e = cudaEventRecord(j->done, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "motion_step: record");
  return BP_OK;
}

int bp_job_get_motion(const bp_job* j, double* theta_host, double* loss_history,
                      int* iters_done) {
  if (!j) return BP_ERR_INVALID_ARG;
  DeviceGuard g(j->device);
  // read back on the job's own stream after its last queued iteration; no
  // device-wide synchronisation, so other jobs keep running
  cudaStream_t os = j->own;
  cudaError_t e = cudaStreamWaitEvent(os, j->done, 0);
  if (e == cudaSuccess && theta_host && j->nodes)  // theta of the current nodes
    e = bpk::launch_akima_eval(j->nodes, j->pd.nviews, j->x, j->theta, os);
  if (e == cudaSuccess && theta_host)
    e = cudaMemcpyAsync(theta_host, j->theta, 48 * (size_t)j->pd.nviews, cudaMemcpyDeviceToHost, os);
  if (e == cudaSuccess && loss_history && j->max_iters > 0)
    e = cudaMemcpyAsync(loss_history, j->hist, 8 * (size_t)j->max_iters, cudaMemcpyDeviceToHost, os);
  if (e == cudaSuccess && iters_done)
    e = cudaMemcpyAsync(iters_done, j->iter, sizeof(int), cudaMemcpyDeviceToHost, os);
  if (e == cudaSuccess) e = cudaStreamSynchronize(os);
  if (e != cudaSuccess) return cuda_fail(j->ctx, e, "bp_job_get_motion");
  return BP_OK;
}

int bp_job_get_nodes(const bp_job* j, double* nodes_host) {
  if (!j || !nodes_host) return BP_ERR_INVALID_ARG;
  if (!j->nodes) return fail(j->ctx, BP_ERR_INVALID_ARG, "bp_job_get_nodes: per-view job");
  DeviceGuard g(j->device);
  cudaStream_t os = j->own;
  cudaError_t e = cudaStreamWaitEvent(os, j->done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nodes_host, j->x, 48 * (size_t)j->nodes, cudaMemcpyDeviceToHost, os);
  if (e == cudaSuccess) e = cudaStreamSynchronize(os);
  if (e != cudaSuccess) return cuda_fail(j->ctx, e, "bp_job_get_nodes");
  return BP_OK;
}

const float* bp_job_volume(const bp_job* j) { return j ? j->vol : nullptr; }

void bp_job_destroy(bp_job* j) {
  if (!j) return;
  DeviceGuard g(j->device);
  if (j->batch) {  // leave the batch: later steps no longer see this job
    auto& m = j->batch->members;
    m.erase(std::remove(m.begin(), m.end(), j), m.end());
    j->batch->dirty = true;
    j->batch = nullptr;
  }
  j->ctx->job_bytes -= j->bytes;
  release(j);
  delete j;
}

}  // extern "C"

// ------------------------------------------------------------------ control

extern "C" {

int bp_job_cancel(bp_job* j) {
  if (!j) return BP_ERR_INVALID_ARG;
  j->cancelled = true;
  return BP_OK;
}

int bp_job_wait(const bp_job* j, double timeout_ms) {
  if (!j) return BP_ERR_INVALID_ARG;
  DeviceGuard g(j->device);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(j->done);
    if (e == cudaSuccess) return BP_OK;
    if (e != cudaErrorNotReady) return cuda_fail(j->ctx, e, "bp_job_wait");
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ms >= 0.0 && ms >= timeout_ms)
      return fail(j->ctx, BP_ERR_TIMEOUT,
                  "bp_job_wait: queued iterations still running after " +
                      std::to_string(timeout_ms) + " ms");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int bp_job_iterations_queued(const bp_job* j) { return j ? j->queued : -1; }

}  // extern "C"

// ------------------------------------------------------------------- batches

namespace {

bool same_config(const bp_job* a, const bp_job* b) {
  return a->pd.dtype == b->pd.dtype && a->weight == b->weight && a->deriv == b->deriv &&
         a->opt.loss == b->opt.loss && a->opt.optimizer == b->opt.optimizer;
}

// Fill one table from the members (host side).
void fill_table(bp_batch* b, bpk::BatchTable& T) {
  const int n = (int)b->members.size();
  T.njobs = n;
  T.off_view[0] = T.off_fwd[0] = T.off_loss[0] = 0;
  const int zbf = bpk::forward_zb();
  for (int k = 0; k < n; ++k) {
    const bp_job* j = b->members[k];
    bpk::BatchJob& J = T.job[k];
    J.proj = j->proj;
    J.grad = j->grad;
    J.P = j->P;
    J.vw = j->vw;
    J.scale = j->scale;
    J.theta = j->theta;
    J.gth = j->gth;
    J.m1 = j->m1;
    J.m2 = j->m2;
    J.geom = j->geom;
    J.vol = j->vol;
    J.dvol = j->dvol;
    J.partials = j->partials;
    J.blk = j->blk;
    J.hist = j->hist;
    J.iter = j->iter;
    J.pi = j->pi;
    J.vi = j->vi;
    J.vif = j->vi;
    J.vif.zb = zbf;
    J.vif.tiles_z = (j->vd.nz + zbf - 1) / zbf;
    J.sid = j->pd.sid;
    J.lr_t = j->opt.lr;
    J.lr_r = j->opt.lr_rot;
    J.beta1 = j->opt.beta1;
    J.beta2 = j->opt.beta2;
    J.eps = j->opt.eps;
    J.decay = j->opt.decay;
    J.tv_eps = (float)j->opt.tv_eps;
    J.V = j->pd.nviews;
    J.ntiles_f = J.vif.tiles_x * J.vif.tiles_y * J.vif.tiles_z;
    J.ntiles_v = j->ntiles;
    J.nblk = j->nblk;
    J.max_iters = j->max_iters;
    J.gauge = j->opt.gauge;
    T.off_view[k + 1] = T.off_view[k] + J.V;
    T.off_fwd[k + 1] = T.off_fwd[k] + J.ntiles_f;
    T.off_loss[k + 1] = T.off_loss[k] + J.nblk;
  }
}

}  // namespace

extern "C" {

int bp_batch_create(bp_ctx* ctx, int max_jobs, bp_batch** out) {
  if (!ctx || !out) return BP_ERR_INVALID_ARG;
  *out = nullptr;
  ctx->err.clear();
  if (max_jobs < 1 || max_jobs > bpk::BATCH_MAX_JOBS)
    return fail(ctx, BP_ERR_INVALID_ARG,
                "bp_batch_create: max_jobs must be 1.." + std::to_string(bpk::BATCH_MAX_JOBS));
  DeviceGuard g(ctx->device);
  bp_batch* b = new bp_batch();
  b->ctx = ctx;
  b->device = ctx->device;
  b->max_jobs = max_jobs;
  cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->counter, 256);
  if (e == cudaSuccess) e = cudaMemset(b->counter, 0, 256);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    bp_batch_destroy(b);
    return cuda_fail(ctx, e, "bp_batch_create");
  }
  *out = b;
  return BP_OK;
}

int bp_batch_set_jobs(bp_batch* b, bp_job* const* jobs, int n_jobs) {
  if (!b || n_jobs < 0 || (n_jobs > 0 && !jobs)) return BP_ERR_INVALID_ARG;
  bp_ctx* ctx = b->ctx;
  ctx->err.clear();
  if (n_jobs > b->max_jobs)
    return fail(ctx, BP_ERR_INVALID_ARG, "bp_batch_set_jobs: more jobs than the batch holds");
  for (int k = 0; k < n_jobs; ++k) {
    const bp_job* j = jobs[k];
    if (!j) return fail(ctx, BP_ERR_INVALID_ARG, "bp_batch_set_jobs: NULL job");
    for (int q = 0; q < k; ++q)
      if (jobs[q] == j) return fail(ctx, BP_ERR_INVALID_ARG, "bp_batch_set_jobs: job listed twice");
    if (j->device != b->device)
      return fail(ctx, BP_ERR_INVALID_ARG, "bp_batch_set_jobs: job on another device");
    if (j->cancelled) return fail(ctx, BP_ERR_CANCELLED, "bp_batch_set_jobs: cancelled job");
    if (j->batch && j->batch != b)
      return fail(ctx, BP_ERR_INVALID_ARG, "bp_batch_set_jobs: job is in another batch");
    if (j->nodes)
      return fail(ctx, BP_ERR_UNSUPPORTED,
                  "bp_batch_set_jobs: only per-view motion (motion_nodes = 0) is batched");
    const int ch = j->pd.dtype == BP_F32 ? 4 : 8;  // elements per 16-byte staging chunk
    if (j->pd.nu % ch)
      return fail(ctx, BP_ERR_UNSUPPORTED,
                  "bp_batch_set_jobs: detector width must be a multiple of 16 bytes");
    if (!same_config(j, jobs[0]))
      return fail(ctx, BP_ERR_INVALID_ARG,
                  "bp_batch_set_jobs: members differ in dtype, weight, derivative, loss or "
                  "optimiser");
  }
  std::vector<bp_job*> next(jobs, jobs + n_jobs);
  if (next != b->members) b->dirty = true;
  for (bp_job* j : b->members) j->batch = nullptr;
  b->members = next;
  for (bp_job* j : b->members) j->batch = b;
  return BP_OK;
}

namespace {

// Free the graphs of earlier member sets whose replays have finished (all,
// waiting for them, when wait is set).
void free_retired(bp_batch* b, bool wait) {
  auto& r = b->retired;
  for (size_t k = 0; k < r.size();) {
    if (wait) cudaEventSynchronize(r[k].done);
    if (cudaEventQuery(r[k].done) == cudaSuccess) {
      cudaGraphExecDestroy(r[k].exec);
      cudaGraphDestroy(r[k].graph);
      cudaEventDestroy(r[k].done);
      r.erase(r.begin() + (long)k);
    } else {
      cudaGetLastError();
      ++k;
    }
  }
}

}  // namespace

int bp_batch_step(bp_batch* b, int n_iters, void* stream) {
  if (!b || n_iters < 0) return BP_ERR_INVALID_ARG;
  bp_ctx* ctx = b->ctx;
  ctx->err.clear();
  DeviceGuard g(b->device);
  // cancelled members stop advancing from this step on
  auto& m = b->members;
  const size_t before = m.size();
  for (bp_job* j : m)
    if (j->cancelled) j->batch = nullptr;
  m.erase(std::remove_if(m.begin(), m.end(), [](const bp_job* j) { return j->cancelled; }),
          m.end());
  if (m.size() != before) b->dirty = true;
  free_retired(b, false);
  if (n_iters == 0 || m.empty()) return BP_OK;
  const bp_job* j0 = m[0];
  const int fdk = j0->weight == BP_WEIGHT_FDK, exact = j0->deriv == BP_DERIV_BILINEAR_EXACT;
  const int loss = j0->opt.loss == BP_LOSS_TV ? 1 : 0;
  const int opt = j0->opt.optimizer == BP_OPT_ADAM ? 1 : 0;
  cudaError_t e;
  if (b->dirty || !b->exec) {
    // a new member set: one graph of the iteration with this member table
    // (the earlier graph is freed once its queued replays have run)
    if (b->exec) {
      cudaEvent_t fresh = nullptr;
      e = cudaEventCreateWithFlags(&fresh, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: event");
      b->retired.push_back({b->graph, b->exec, b->last});
      b->last = fresh;
      b->graph = nullptr;
      b->exec = nullptr;
    }
    fill_table(b, b->table);
    e = bpk::prepare_batch(j0->pd.dtype, fdk, exact);
    if (e == cudaSuccess) e = bpk::prepare_vjp(j0->pd.dtype, fdk, exact);
    if (e == cudaSuccess && !b->br_fork)
      e = cudaEventCreateWithFlags(&b->br_fork, cudaEventDisableTiming);
    while (e == cudaSuccess && b->br_streams.size() < m.size()) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (st) b->br_streams.push_back(st);
      if (ev) b->br_joins.push_back(ev);
      if (b->br_joins.size() < b->br_streams.size()) {  // keep the two lists paired
        cudaStreamDestroy(b->br_streams.back());
        b->br_streams.pop_back();
      }
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: capture");
    bpk::BatchBranches br;
    br.n = (int)b->br_streams.size();
    br.streams = b->br_streams.data();
    br.fork = b->br_fork;
    br.joins = b->br_joins.data();
    const cudaError_t le = bpk::launch_batch_iteration(b->table, b->counter, j0->pd.dtype, fdk,
                                                       exact, loss, opt, b->sms, b->cap, &br);
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      if (b->graph) cudaGraphDestroy(b->graph);
      b->graph = nullptr;
      b->exec = nullptr;
      return cuda_fail(ctx, e, "bp_batch_step: graph");
    }
    b->dirty = false;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (bp_job* j : m) {  // the members' set-up and earlier work come first
    e = cudaStreamWaitEvent(s, j->done, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: wait");
  }
  for (int i = 0; i < n_iters; ++i) {
    e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: launch");
  }
  ctx->launches += (long long)(bpk::BATCH_KERNELS + (int)m.size()) * n_iters;
  for (bp_job* j : m) {
    j->queued += n_iters;
    e = cudaEventRecord(j->done, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: record");
  }
  e = cudaEventRecord(b->last, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_batch_step: record");
  return BP_OK;
}

int bp_batch_size(const bp_batch* b) { return b ? (int)b->members.size() : -1; }

void bp_batch_destroy(bp_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  if (b->last) cudaEventSynchronize(b->last);
  free_retired(b, true);
  for (bp_job* j : b->members) j->batch = nullptr;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t st : b->br_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->br_joins) cudaEventDestroy(ev);
  if (b->br_fork) cudaEventDestroy(b->br_fork);
  if (b->counter) cudaFree(b->counter);
  if (b->last) cudaEventDestroy(b->last);
  delete b;
}

}  // extern "C"
