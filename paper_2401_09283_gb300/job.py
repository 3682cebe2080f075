"""Motion-estimation jobs (Sec. II-C) through the C-ABI job entry points.

A job owns device copies of the projections and all optimiser state;
motion_step() replays one captured CUDA graph per iteration (compose ->
backprojection -> sharpness loss -> motion VJP -> FP64 reduction and chain
rule -> Adam or the decaying gradient step of Eq. 6).  With motion_nodes > 0
the motion is the Akima spline model of Sec. II-B.1 and the optimiser works
on the 6 N_n node values (spline and spline VJP run inside the graph)."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import native as N

OPT = {"gd": 0, "adam": 1}
LOSS = {"sharpness": 0, "tv": 1}


class MotionJob:
    def __init__(self, proj, P, *, vol_shape, spacing, origin, sid, view_weight=None,
                 weight="fdk", deriv="central", optimizer="adam", lr=0.1, lr_rot=1e-3,
                 decay=0.97, betas=(0.9, 0.999), eps=1e-8, gauge=True, theta0=None,
                 max_iters=100, view_scale=None, device=None, loss="sharpness", tv_eps=1e-3,
                 motion_nodes=0):
        self.V = int(P.shape[0])
        self.nodes = int(motion_nodes)
        self.max_iters = int(max_iters)
        if device is None:
            device = N.device_of(proj, P)
        self.device = device
        self.ctx = N.context(device)
        pd = N.proj_desc(proj, sid, view_scale)
        vd = N.vol_desc(vol_shape, spacing, origin)
        od = N.OptDesc(OPT[optimizer], float(lr), float(lr_rot), float(decay), float(betas[0]),
                       float(betas[1]), float(eps), int(bool(gauge)), LOSS[loss], float(tv_eps),
                       self.nodes)
        Pc = P if isinstance(P, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(P))
        self._keep = (proj, Pc, view_weight, theta0, view_scale)
        h = ctypes.c_void_p()
        rc = N.lib().bp_job_create(self.ctx, N.ptr(proj), ctypes.byref(pd), N.ptr(Pc),
                                   N.ptr(view_weight), N.WEIGHT[weight], N.DERIV[deriv],
                                   ctypes.byref(vd), ctypes.byref(od), N.ptr(theta0),
                                   self.max_iters, ctypes.byref(h))
        N.check("bp_job_create", rc, self.ctx)
        self.handle = h
        self._keep = None

    @staticmethod
    def bytes_for(proj_shape, dtype_code, vol_shape, deriv="central", max_iters=100):
        V, nv, nu = proj_shape
        pd = N.ProjDesc(nu, nv, V, dtype_code, nu, nu * nv, None, 0.0)
        vd = N.vol_desc(vol_shape, (1, 1, 1), (0, 0, 0))
        return int(N.lib().bp_job_bytes_for(ctypes.byref(pd), ctypes.byref(vd), N.DERIV[deriv],
                                            int(max_iters)))

    @property
    def nbytes(self):
        return int(N.lib().bp_job_bytes(self.handle))

    def step(self, n=1, stream=None):
        """Queue n iterations on `stream` (default: the current torch stream)."""
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = N.lib().motion_step(self.handle, int(n), stream)
        N.check("motion_step", rc, self.ctx)

    def motion(self):
        """(theta (V,6), loss history (max_iters,), iterations done) on the host."""
        th = np.zeros((self.V, 6))
        hist = np.zeros(max(1, self.max_iters))
        it = ctypes.c_int()
        rc = N.lib().bp_job_get_motion(self.handle, th.ctypes.data, hist.ctypes.data,
                                       ctypes.byref(it))
        N.check("bp_job_get_motion", rc, self.ctx)
        return th, hist[: self.max_iters], int(it.value)

    def node_values(self):
        """Current spline node values (N_n,6) of a job with the Akima model."""
        x = np.zeros((self.nodes, 6))
        rc = N.lib().bp_job_get_nodes(self.handle, x.ctypes.data)
        N.check("bp_job_get_nodes", rc, self.ctx)
        return x

    def cancel(self):
        """Stop advancing the job (motion_step then raises BP_ERR_CANCELLED)."""
        N.check("bp_job_cancel", N.lib().bp_job_cancel(self.handle), self.ctx)

    def wait(self, timeout_ms=-1.0):
        """Wait for the queued iterations; False if they still run after
        timeout_ms (BP_ERR_TIMEOUT), True when done."""
        rc = N.lib().bp_job_wait(self.handle, float(timeout_ms))
        if rc == N.BP_ERR_TIMEOUT:
            return False
        N.check("bp_job_wait", rc, self.ctx)
        return True

    @property
    def iterations_queued(self):
        return int(N.lib().bp_job_iterations_queued(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            N.lib().bp_job_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_hbm_budget(nbytes, device=None):
    """Bytes that the live jobs of a device's context may hold (0 = free memory)."""
    ctx = N.context(device)
    N.check("bp_ctx_set_hbm_budget", N.lib().bp_ctx_set_hbm_budget(ctx, int(nbytes)), ctx)


class Batch:
    """Resident jobs advanced together (bp_batch_*): every stage of an
    iteration but the VJP is one launch over the work items of all members
    (the backprojection persistent); the members' VJP kernels run as parallel
    branches of the same captured graph."""

    def __init__(self, max_jobs=8, device=None):
        self.ctx = N.context(device)
        h = ctypes.c_void_p()
        N.check("bp_batch_create", N.lib().bp_batch_create(self.ctx, int(max_jobs), ctypes.byref(h)),
                self.ctx)
        self.handle = h
        self.jobs = []

    def set_jobs(self, jobs):
        arr = (ctypes.c_void_p * max(1, len(jobs)))(*[j.handle.value for j in jobs])
        N.check("bp_batch_set_jobs", N.lib().bp_batch_set_jobs(self.handle, arr, len(jobs)),
                self.ctx)
        self.jobs = list(jobs)

    def step(self, n=1, stream=None):
        """Queue n iterations of every member on `stream`."""
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        N.check("bp_batch_step", N.lib().bp_batch_step(self.handle, int(n), stream), self.ctx)

    @property
    def size(self):
        return int(N.lib().bp_batch_size(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            N.lib().bp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
