// Private: the context object and host helpers shared by the C-ABI
// translation units (bp_api.cu, bp_job.cu).
#pragma once

#include <cstring>
#include <string>
#include <vector>

#include "bp_gb300.h"
#include "bp_internal.cuh"

namespace bpctx {

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

enum KernelId {
  K_COMPOSE, K_FORWARD, K_GRAD, K_VJP_MOTION, K_REDUCE, K_VJP_PROJ, K_VJP_FUSED, K_SHARPNESS,
  K_OPT, K_SPLINE, K_FDK, K_COUNT
};
const char* const kKernelNames[K_COUNT] = {"compose",  "forward",   "grad_images",
                                           "vjp_motion", "reduce_chain", "vjp_proj",
                                           "vjp_fused",  "sharpness", "optimizer",
                                           "spline",   "fdk_filter"};
struct Pending {
  int id;
  cudaEvent_t a, b;
};
}  // namespace bpctx

struct bp_ctx {
  int device = 0;
  std::string err;
  // kernel accounting: launch counter (always) and optional event timing
  long long launches = 0;
  bool timing = false;
  std::vector<bpctx::Pending> pending;
  std::vector<cudaEvent_t> spare;
  double total_ms[bpctx::K_COUNT] = {};
  long long count[bpctx::K_COUNT] = {};
  // workspace
  bpctx::Buf geom, grad, partials, shblk, fdk_tab, probe, blkimg;
  // staging of host arguments
  bpctx::Buf s_proj, s_P, s_motion, s_vw, s_scale, s_vol, s_dvol, s_out_motion, s_out_P, s_out_proj,
      s_theta, s_grad, s_m1, s_m2, s_loss, s_nodes, s_out_nodes;
  // jobs
  long long hbm_budget = 0;  // bytes all jobs of this context may hold (0 = free memory)
  long long job_bytes = 0;   // bytes held by live jobs
};

namespace bpctx {

using bpk::ProjInfo;
using bpk::ViewGeom;
using bpk::VolInfo;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline int fail(bp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

inline int cuda_fail(bp_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? BP_ERR_OOM : BP_ERR_CUDA, m);
}

#define CK(expr, where)                              \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

inline cudaEvent_t take_event(bp_ctx* c) {
  if (!c->spare.empty()) {
    cudaEvent_t e = c->spare.back();
    c->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Fold finished event pairs into the per-kernel totals (synchronises them).
inline void resolve_timing(bp_ctx* c) {
  for (const Pending& p : c->pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->total_ms[p.id] += ms;
      c->count[p.id] += 1;
    } else {
      cudaGetLastError();
    }
    c->spare.push_back(p.a);
    c->spare.push_back(p.b);
  }
  c->pending.clear();
}

// Launch nk kernels through f(); with timing on, bracket them by events.
template <class F>
inline cudaError_t timed(bp_ctx* c, int id, int nk, cudaStream_t s, F f) {
  c->launches += nk;
  if (!c->timing) return f();
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return f();
  cudaEventRecord(a, s);
  cudaError_t e = f();
  cudaEventRecord(b, s);
  c->pending.push_back({id, a, b});
  if (c->pending.size() > 4096) resolve_timing(c);
  return e;
}

#define TL(id, nk, expr) timed(ctx, id, nk, s, [&]() { return (expr); })

// Grow a workspace buffer (contents are not preserved).
inline cudaError_t ensure(Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return cudaSuccess;
  if (b.p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return e;
  }
  b.n = bytes;
  return cudaSuccess;
}

inline bool is_host(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Returns a device pointer holding `bytes` of the caller's array (copied to
// `stage` when the caller's pointer is host memory).
inline cudaError_t stage_in(Buf& stage, const void* p, size_t bytes, cudaStream_t s, const void** out) {
  if (!p || !is_host(p)) {
    *out = p;
    return cudaSuccess;
  }
  cudaError_t e = ensure(stage, bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(stage.p, p, bytes, cudaMemcpyHostToDevice, s);
  *out = stage.p;
  return e;
}

// Device destination for an output (a staging buffer when it is host memory).
inline cudaError_t stage_out(Buf& stage, void* p, size_t bytes, void** out, bool* host) {
  *host = p && is_host(p);
  if (!*host) {
    *out = p;
    return cudaSuccess;
  }
  cudaError_t e = ensure(stage, bytes);
  *out = stage.p;
  return e;
}

}  // namespace bpctx
