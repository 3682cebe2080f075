"""Oracle: plain FP64 CPU restatement of the paper's backprojection (Eq. 3),
its analytic Jacobian (Eqs. 4-5), the rigid motion composition (Eq. 1), the
chain rule (Eq. 2), the gradient-descent update (Eq. 6), Adam, a sharpness
loss, total variation, the reprojection error (Sec. IV-A) and the Akima
spline motion model (Sec. II-B.1) and the FDK preprocessing of the raw
projections (cosine weight, short-scan weights, Shepp-Logan ramp).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
never does.  It shares no code with the CUDA library.

The arithmetic lives in ``orc.c`` (compiled by ``oracle/build.py`` with gcc);
this module only marshals numpy arrays through ctypes.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, finite differences or brute force.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

WEIGHT_NONE = 0
WEIGHT_FDK = 1
DERIV_CENTRAL = 0
DERIV_BILINEAR_EXACT = 1

_lib = None


class _Vol(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("sx", ctypes.c_double), ("sy", ctypes.c_double), ("sz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build_oracle()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_rigid.argtypes = [dp, dp]
        lib.orc_rigid_grad.argtypes = [dp, dp]
        lib.orc_compose.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.orc_bp_forward.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                                       ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Vol), dp]
        lib.orc_gradient_images.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_bp_vjp.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(_Vol), dp, dp, dp]
        lib.orc_chain_motion.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        lib.orc_sharpness.argtypes = [ctypes.POINTER(_Vol), dp, dp]
        lib.orc_sharpness.restype = ctypes.c_double
        lib.orc_tv.argtypes = [ctypes.POINTER(_Vol), dp, ctypes.c_double, dp]
        lib.orc_tv.restype = ctypes.c_double
        lib.orc_gd_step.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int]
        lib.orc_adam_step.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int]
        lib.orc_rpe.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, ctypes.c_double,
                                ctypes.c_double]
        lib.orc_rpe.restype = ctypes.c_double
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        lib.orc_akima_eval.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp]
        lib.orc_parker.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_parker.restype = ctypes.c_double
        lib.orc_fdk_filter.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, dp]
        lib.orc_akima_jacobian.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vol(shape, spacing, origin):
    nz, ny, nx = shape
    return _Vol(nx, ny, nz, *[float(s) for s in spacing], *[float(o) for o in origin])


def num_threads() -> int:
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS or all cores)."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    _load().orc_set_num_threads(int(n))


def rigid(theta):
    """Eq. 1: 4x4 rigid transform for theta = (tx,ty,tz,rx,ry,rz)."""
    th = _f64(theta)
    T = np.zeros((4, 4))
    _load().orc_rigid(_ptr(th), _ptr(T))
    return T


def rigid_grad(theta):
    """dT/dtheta_m, shape (6,4,4)."""
    th = _f64(theta)
    dT = np.zeros((6, 4, 4))
    _load().orc_rigid_grad(_ptr(th), _ptr(dT))
    return dT


def compose(P, theta=None):
    """Eq. 1 per view: Phat_j = P_j T(theta_j); P (V,3,4), theta (V,6) or None."""
    P = _f64(P)
    V = P.shape[0]
    th = None if theta is None else _f64(theta)
    out = np.zeros((V, 3, 4))
    _load().orc_compose(V, _ptr(P), _ptr(th), _ptr(out))
    return out


def bp_forward(Phat, proj, vol_shape, spacing, origin, view_weight=None,
               weight_mode=WEIGHT_NONE, sid=0.0):
    """Eq. 3 over the voxel grid; proj (V,nv,nu); returns vol (nz,ny,nx)."""
    Phat = _f64(Phat)
    proj = _f64(proj)
    V, nv, nu = proj.shape
    vw = None if view_weight is None else _f64(view_weight)
    vol = np.zeros(tuple(vol_shape))
    g = _vol(vol_shape, spacing, origin)
    _load().orc_bp_forward(V, _ptr(Phat), _ptr(proj), nu, nv, _ptr(vw), int(weight_mode),
                           float(sid), ctypes.byref(g), _ptr(vol))
    return vol


def gradient_images(img):
    """Central-difference gradient images (g_u, g_v) of one 2D projection."""
    img = _f64(img)
    nv, nu = img.shape
    gu = np.zeros_like(img)
    gv = np.zeros_like(img)
    _load().orc_gradient_images(_ptr(img), nu, nv, _ptr(gu), _ptr(gv))
    return gu, gv


def bp_vjp(Phat, proj, dL_dvol, spacing, origin, view_weight=None, weight_mode=WEIGHT_NONE,
           deriv_mode=DERIV_CENTRAL, sid=0.0, want_P=True, want_proj=True):
    """Eqs. 4-5: returns (dL/dPhat (V,3,4) or None, dL/dproj (V,nv,nu) or None)."""
    Phat = _f64(Phat)
    proj = _f64(proj)
    dvol = _f64(dL_dvol)
    V, nv, nu = proj.shape
    vw = None if view_weight is None else _f64(view_weight)
    gP = np.zeros((V, 3, 4)) if want_P else None
    gD = np.zeros_like(proj) if want_proj else None
    g = _vol(dvol.shape, spacing, origin)
    _load().orc_bp_vjp(V, _ptr(Phat), _ptr(proj), nu, nv, _ptr(vw), int(weight_mode),
                       int(deriv_mode), float(sid), ctypes.byref(g), _ptr(dvol), _ptr(gP),
                       _ptr(gD))
    return gP, gD


def chain_motion(P, theta, dL_dPhat):
    """Eq. 2 through Eq. 1: dL/dtheta (V,6) from dL/dPhat (V,3,4)."""
    P = _f64(P)
    th = _f64(theta)
    G = _f64(dL_dPhat)
    V = P.shape[0]
    out = np.zeros((V, 6))
    _load().orc_chain_motion(V, _ptr(P), _ptr(th), _ptr(G), _ptr(out))
    return out


def sharpness(vol, spacing=(1, 1, 1), origin=(0, 0, 0), want_grad=True):
    """Sharpness loss L = -(1/K) sum of squared forward differences; (L, dL/dI)."""
    vol = _f64(vol)
    g = _vol(vol.shape, spacing, origin)
    grad = np.zeros_like(vol) if want_grad else None
    L = _load().orc_sharpness(ctypes.byref(g), _ptr(vol), _ptr(grad))
    return float(L), grad


def tv(vol, eps, want_grad=True):
    """Smoothed isotropic total variation L = (1/K) sum sqrt(|grad+ I|^2 + eps^2)
    over voxels with all forward neighbours inside; (L, dL/dI)."""
    vol = _f64(vol)
    g = _vol(vol.shape, (1, 1, 1), (0, 0, 0))
    grad = np.zeros_like(vol) if want_grad else None
    L = _load().orc_tv(ctypes.byref(g), _ptr(vol), float(eps), _ptr(grad))
    return float(L), grad


def gd_step(theta, grad, s0, t, n, gauge=True):
    """Eq. 6 step n (0-based) in place on a copy; returns the new theta."""
    th = _f64(theta).copy()
    gr = _f64(grad)
    _load().orc_gd_step(th.shape[0], _ptr(th), _ptr(gr), float(s0), float(t), int(n),
                        int(bool(gauge)))
    return th


def adam_step(theta, grad, m1, m2, lr, n, b1=0.9, b2=0.999, eps=1e-8, gauge=True):
    """Adam step n (1-based); returns (theta, m1, m2) as new arrays."""
    th = _f64(theta).copy()
    a = _f64(m1).copy()
    b = _f64(m2).copy()
    gr = _f64(grad)
    _load().orc_adam_step(th.shape[0], _ptr(th), _ptr(gr), _ptr(a), _ptr(b), float(lr),
                          float(b1), float(b2), float(eps), int(n), int(bool(gauge)))
    return th, a, b


def rpe(Pa, Pb, pts, du, dv):
    """Mean reprojection error in detector mm between geometries Pa and Pb."""
    Pa = _f64(Pa)
    Pb = _f64(Pb)
    pts = _f64(pts)
    return float(_load().orc_rpe(Pa.shape[0], _ptr(Pa), _ptr(Pb), pts.shape[0], _ptr(pts),
                                 float(du), float(dv)))


def akima_eval(y, xe, x=None):
    """Akima spline through (x_i, y_i) (x defaults to 0..n-1) at points xe."""
    y = _f64(y)
    n = y.shape[0]
    x = _f64(np.arange(n) if x is None else x)
    xe = _f64(xe)
    out = np.zeros(xe.shape[0])
    _load().orc_akima_eval(n, _ptr(x), _ptr(y), xe.shape[0], _ptr(xe), _ptr(out))
    return out


def akima_jacobian(y, xe, x=None):
    """d spline(xe_q) / d y_k, shape (len(xe), n), by forward-mode duals."""
    y = _f64(y)
    n = y.shape[0]
    x = _f64(np.arange(n) if x is None else x)
    xe = _f64(xe)
    J = np.zeros((xe.shape[0], n))
    _load().orc_akima_jacobian(n, _ptr(x), _ptr(y), xe.shape[0], _ptr(xe), _ptr(J))
    return J


def motion_knots(n_nodes, nviews):
    """Knots of the motion splines: evenly spread over the view index, one at
    the first view and one at the last (Sec. II-B.1)."""
    return np.linspace(0.0, nviews - 1.0, n_nodes)


def akima_motion(nodes, nviews):
    """theta (V,6): the six splines through nodes (N_n,6) at views 0..V-1."""
    nodes = _f64(nodes)
    x = motion_knots(nodes.shape[0], nviews)
    xe = np.arange(nviews, dtype=np.float64)
    return np.stack([akima_eval(nodes[:, p], xe, x) for p in range(6)], axis=1)


def akima_motion_vjp(nodes, nviews, dL_dtheta):
    """dL/dnodes (N_n,6) = J^T dL/dtheta per parameter, J from akima_jacobian."""
    nodes = _f64(nodes)
    g = _f64(dL_dtheta)
    x = motion_knots(nodes.shape[0], nviews)
    xe = np.arange(nviews, dtype=np.float64)
    return np.stack([akima_jacobian(nodes[:, p], xe, x).T @ g[:, p] for p in range(6)], axis=1)


def parker(beta, gamma, arc):
    """Short-scan redundancy weight of the ray (beta from the scan start, fan
    angle gamma) for a scan arc `arc` (rad)."""
    return float(_load().orc_parker(float(beta), float(gamma), float(arc)))


def fdk_filter(raw, pitch, sid, sdd, arc, ext=0):
    """Cosine weight, short-scan (or full-scan 1/2) weight and Shepp-Logan
    ramp of raw line integrals (V,nv,nu), by direct convolution; ext > 0
    extends every weighted row by ext pixels per side falling linearly to 0
    (truncation correction)."""
    raw = _f64(raw)
    V, nv, nu = raw.shape
    out = np.zeros_like(raw)
    _load().orc_fdk_filter(V, nu, nv, _ptr(raw), float(pitch), float(sid), float(sdd), float(arc),
                           int(ext), _ptr(out))
    return out
