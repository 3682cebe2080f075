"""ctypes binding of the bp_gb300 C-ABI (include/bp_gb300.h).

Argument marshalling only: every computation runs in the CUDA library.
Tensors may be CUDA tensors (device pointers) or CPU tensors / numpy arrays
(host pointers, staged by the library).  If the shared library has not been
built, importing the functions raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from .build import LIB

BP_OK = 0
BP_ERR_TIMEOUT = -5
BP_ERR_CANCELLED = -6
STATUS = {0: "BP_OK", -1: "BP_ERR_INVALID_ARG", -2: "BP_ERR_OOM", -3: "BP_ERR_CUDA",
          -4: "BP_ERR_UNSUPPORTED", -5: "BP_ERR_TIMEOUT", -6: "BP_ERR_CANCELLED"}
F32, F16, BF16 = 0, 1, 2
WEIGHT = {"none": 0, "fdk": 1}
DERIV = {"central": 0, "exact": 1}

c_int, c_double, c_void_p, c_ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong


class VolDesc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("spacing", c_double * 3),
                ("origin", c_double * 3)]


class ProjDesc(ctypes.Structure):
    _fields_ = [("nu", c_int), ("nv", c_int), ("nviews", c_int), ("dtype", c_int),
                ("row_stride", c_ll), ("view_stride", c_ll), ("view_scale", c_void_p),
                ("sid", c_double)]


class OptDesc(ctypes.Structure):
    _fields_ = [("optimizer", c_int), ("lr", c_double), ("lr_rot", c_double), ("decay", c_double),
                ("beta1", c_double), ("beta2", c_double), ("eps", c_double), ("gauge", c_int),
                ("loss", c_int), ("tv_eps", c_double), ("motion_nodes", c_int)]


class BPError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__("%s failed: %s (%d): %s" % (fn, STATUS.get(code, "?"), code, msg))
        self.code = code


_lib = None
_lock = threading.Lock()
_ctx = {}

EXPORTS = ["bp_ctx_create", "bp_ctx_destroy", "bp_last_error", "bp_ctx_workspace_bytes",
           "bp_ctx_launch_count", "bp_ctx_set_timing", "bp_ctx_timing",
           "bp_compose", "bp_forward", "bp_vjp", "bp_sharpness", "bp_tv", "bp_sharpness_noalloc",
           "bp_gd_step", "bp_adam_step", "bp_job_create", "bp_job_bytes_for", "bp_job_bytes",
           "bp_ctx_set_hbm_budget", "motion_step", "bp_job_get_motion", "bp_job_volume",
           "bp_job_destroy", "bp_akima_motion", "bp_akima_motion_vjp", "bp_job_get_nodes",
           "bp_fdk_filter", "bp_job_cancel", "bp_job_wait", "bp_job_iterations_queued",
           "bp_batch_create", "bp_batch_set_jobs", "bp_batch_step", "bp_batch_size",
           "bp_batch_destroy", "bp_bounds_check", "bp_probe"]


def library_path():
    """The release library, or the one BP_GB300_LIB names (e.g. the
    bounds-checking debug build)."""
    return os.environ.get("BP_GB300_LIB") or LIB


def lib():
    """Load the shared library (raises if it was not built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                path = library_path()
                if not os.path.exists(path):
                    raise RuntimeError("bp_gb300 CUDA library not found at %s; build it with "
                                       "`python -m paper_2401_09283_gb300.build` or "
                                       "__graft_entry__.build()" % path)
                L = ctypes.CDLL(path)
                vp, dp, ip = c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int)
                del dp, ip
                L.bp_ctx_create.argtypes = [c_int, ctypes.POINTER(c_void_p)]
                L.bp_ctx_destroy.argtypes = [vp]
                L.bp_ctx_destroy.restype = None
                L.bp_last_error.argtypes = [vp]
                L.bp_last_error.restype = ctypes.c_char_p
                L.bp_ctx_workspace_bytes.argtypes = [vp]
                L.bp_ctx_workspace_bytes.restype = c_ll
                L.bp_ctx_launch_count.argtypes = [vp]
                L.bp_ctx_launch_count.restype = c_ll
                L.bp_ctx_set_timing.argtypes = [vp, c_int]
                L.bp_ctx_timing.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(c_double),
                                            ctypes.POINTER(c_ll)]
                L.bp_compose.argtypes = [vp, c_int, vp, vp, vp, vp]
                L.bp_forward.argtypes = [vp, vp, ctypes.POINTER(ProjDesc), vp, vp, vp, c_int,
                                         ctypes.POINTER(VolDesc), vp, vp]
                L.bp_vjp.argtypes = [vp, vp, vp, ctypes.POINTER(ProjDesc), vp, vp, vp, c_int,
                                     c_int, ctypes.POINTER(VolDesc), vp, vp, vp, vp]
                L.bp_sharpness.argtypes = [vp, vp, ctypes.POINTER(VolDesc), vp, vp, vp]
                L.bp_tv.argtypes = [vp, vp, ctypes.POINTER(VolDesc), c_double, vp, vp, vp]
                L.bp_sharpness_noalloc.argtypes = [vp, ctypes.POINTER(VolDesc), vp, vp, vp]
                L.bp_gd_step.argtypes = [vp, c_int, vp, vp, c_double, c_double, c_int, c_int, vp]
                L.bp_adam_step.argtypes = [vp, c_int, vp, vp, vp, vp, c_double, c_double,
                                           c_double, c_double, c_int, c_int, vp]
                L.bp_job_create.argtypes = [vp, vp, ctypes.POINTER(ProjDesc), vp, vp, c_int, c_int,
                                            ctypes.POINTER(VolDesc), ctypes.POINTER(OptDesc), vp,
                                            c_int, ctypes.POINTER(c_void_p)]
                L.bp_job_bytes_for.argtypes = [ctypes.POINTER(ProjDesc), ctypes.POINTER(VolDesc),
                                               c_int, c_int]
                L.bp_job_bytes_for.restype = c_ll
                L.bp_job_bytes.argtypes = [vp]
                L.bp_job_bytes.restype = c_ll
                L.bp_ctx_set_hbm_budget.argtypes = [vp, c_ll]
                L.motion_step.argtypes = [vp, c_int, vp]
                L.bp_job_get_motion.argtypes = [vp, vp, vp, ctypes.POINTER(c_int)]
                L.bp_job_volume.argtypes = [vp]
                L.bp_job_volume.restype = c_void_p
                L.bp_job_destroy.argtypes = [vp]
                L.bp_job_destroy.restype = None
                L.bp_akima_motion.argtypes = [vp, c_int, c_int, vp, vp, vp]
                L.bp_job_get_nodes.argtypes = [vp, vp]
                L.bp_fdk_filter.argtypes = [vp, vp, c_int, c_int, c_int, c_double, c_double,
                                            c_double, c_double, c_int, vp, vp]
                L.bp_akima_motion_vjp.argtypes = [vp, c_int, c_int, vp, vp, vp, vp]
                L.bp_job_cancel.argtypes = [vp]
                L.bp_job_wait.argtypes = [vp, c_double]
                L.bp_job_iterations_queued.argtypes = [vp]
                L.bp_batch_create.argtypes = [vp, c_int, ctypes.POINTER(c_void_p)]
                L.bp_batch_set_jobs.argtypes = [vp, ctypes.POINTER(c_void_p), c_int]
                L.bp_batch_step.argtypes = [vp, c_int, vp]
                L.bp_batch_size.argtypes = [vp]
                L.bp_batch_destroy.argtypes = [vp]
                L.bp_batch_destroy.restype = None
                L.bp_bounds_check.argtypes = [vp, c_int, ctypes.POINTER(ctypes.c_uint),
                                              ctypes.POINTER(c_ll)]
                L.bp_probe.argtypes = [vp, c_int, ctypes.POINTER(c_double), vp]
                _lib = L
    return _lib


def exported_symbols():
    L = lib()
    return {name: hasattr(L, name) for name in EXPORTS}


def context(device=None):
    """The library context of a CUDA device (created on first use)."""
    if device is None:
        device = torch.cuda.current_device()
    device = int(device)
    if device not in _ctx:
        h = c_void_p()
        rc = lib().bp_ctx_create(device, ctypes.byref(h))
        if rc != BP_OK:
            raise BPError("bp_ctx_create", rc, "device %d (GB300 sm_103 required)" % device)
        _ctx[device] = h
    return _ctx[device]


def check(name, rc, ctx):
    if rc != BP_OK:
        msg = lib().bp_last_error(ctx)
        raise BPError(name, rc, msg.decode() if msg else "")


# ------------------------------------------------------------------ marshalling

def ptr(x):
    """Raw pointer of a tensor / ndarray (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors passed to bp_gb300 must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to bp_gb300 must be C-contiguous")
        return x.ctypes.data
    raise TypeError("unsupported array type %r" % type(x))


def stream_of(*xs):
    for x in xs:
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return torch.cuda.current_stream(x.device).cuda_stream
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0


def device_of(*xs):
    for x in xs:
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return x.device.index
    return torch.cuda.current_device()


def vol_desc(shape, spacing, origin):
    nz, ny, nx = shape
    return VolDesc(int(nx), int(ny), int(nz), (c_double * 3)(*map(float, spacing)),
                   (c_double * 3)(*map(float, origin)))


_DT = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16,
       np.dtype(np.float32): F32, np.dtype(np.float16): F16}


def proj_desc(proj, sid=0.0, view_scale=None):
    dt = proj.dtype if isinstance(proj, torch.Tensor) else np.dtype(proj.dtype)
    if dt not in _DT:
        raise TypeError("projections must be float32, float16 or bfloat16, got %s" % dt)
    V, nv, nu = proj.shape
    return ProjDesc(int(nu), int(nv), int(V), _DT[dt], int(nu), int(nu) * int(nv),
                    ptr(view_scale), float(sid))


KERNELS = ("compose", "forward", "grad_images", "vjp_motion", "reduce_chain", "vjp_proj",
           "vjp_fused", "sharpness", "optimizer", "spline", "fdk_filter")


def set_timing(enable=True, device=None):
    ctx = context(device)
    check("bp_ctx_set_timing", lib().bp_ctx_set_timing(ctx, int(bool(enable))), ctx)


def kernel_times(device=None):
    """{kernel: (total device ms, launches)} since set_timing(True)."""
    ctx = context(device)
    out = {}
    for k in KERNELS:
        ms = c_double()
        n = c_ll()
        check("bp_ctx_timing", lib().bp_ctx_timing(ctx, k.encode(), ctypes.byref(ms),
                                                   ctypes.byref(n)), ctx)
        out[k] = (ms.value, n.value)
    return out


def launch_count(device=None):
    return int(lib().bp_ctx_launch_count(context(device)))


def probe(kind, device=None):
    """bp_probe: a throughput measurement (per second) on the device."""
    ctx = context(device)
    out = c_double()
    check("bp_probe", lib().bp_probe(ctx, int(kind), ctypes.byref(out), None), ctx)
    return out.value
