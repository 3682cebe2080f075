"""Tensor-level entry points with the names of the C-ABI.

Each function checks shapes/dtypes, allocates outputs with torch on the
inputs' device and calls the CUDA library; nothing is computed here.

Shapes: proj (V, nv, nu) float32/float16/bfloat16; P (V, 3, 4) float64;
motion (V, 6) float64 (tx, ty, tz [mm], rx, ry, rz [rad]); volumes
(nz, ny, nx) float32.
"""
from __future__ import annotations

import ctypes

import torch

from . import native as N


def _f64(x, name):
    if x is None:
        return None
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(x)
    if x.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    return x.contiguous()


def bp_compose(P, motion=None):
    """Eq. 1: Phat_j = P_j T(motion_j); returns (V,3,4) float64 on P's device."""
    P = _f64(P, "P")
    motion = _f64(motion, "motion")
    out = torch.empty_like(P)
    ctx = N.context(N.device_of(P, motion))
    rc = N.lib().bp_compose(ctx, P.shape[0], N.ptr(P), N.ptr(motion), N.ptr(out),
                            N.stream_of(P, motion))
    N.check("bp_compose", rc, ctx)
    return out


def bp_forward(proj, P, motion=None, *, vol_shape, spacing, origin, view_weight=None,
               weight="fdk", sid=0.0, view_scale=None, out=None):
    """Eq. 3 with motion composition (Eq. 1); returns the float32 volume."""
    P = _f64(P, "P")
    motion = _f64(motion, "motion")
    view_weight = _f64(view_weight, "view_weight")
    if out is None:
        dev = proj.device if isinstance(proj, torch.Tensor) else torch.device("cpu")
        out = torch.empty(tuple(vol_shape), dtype=torch.float32, device=dev)
    pd = N.proj_desc(proj, sid, view_scale)
    vd = N.vol_desc(vol_shape, spacing, origin)
    ctx = N.context(N.device_of(proj, P, out))
    rc = N.lib().bp_forward(ctx, N.ptr(proj), ctypes.byref(pd), N.ptr(P), N.ptr(motion),
                            N.ptr(view_weight), N.WEIGHT[weight], ctypes.byref(vd), N.ptr(out),
                            N.stream_of(proj, out))
    N.check("bp_forward", rc, ctx)
    return out


def bp_vjp(dL_dvol, proj, P, motion=None, *, spacing, origin, view_weight=None, weight="fdk",
           deriv="central", sid=0.0, view_scale=None, want_motion=True, want_Phat=False,
           want_proj=False, out_motion=None, out_Phat=None, out_proj=None):
    """VJPs of bp_forward (Eqs. 4-5 and the chain rule of Eq. 2).

    Returns (dL/dmotion (V,6) f64 | None, dL/dPhat (V,3,4) f64 | None,
    dL/dproj (V,nv,nu) f32 | None)."""
    P = _f64(P, "P")
    motion = _f64(motion, "motion")
    view_weight = _f64(view_weight, "view_weight")
    V, nv, nu = proj.shape
    dev = dL_dvol.device if isinstance(dL_dvol, torch.Tensor) else torch.device("cpu")
    if want_motion and out_motion is None:
        out_motion = torch.empty((V, 6), dtype=torch.float64, device=dev)
    if want_Phat and out_Phat is None:
        out_Phat = torch.empty((V, 3, 4), dtype=torch.float64, device=dev)
    if want_proj and out_proj is None:
        out_proj = torch.empty((V, nv, nu), dtype=torch.float32, device=dev)
    pd = N.proj_desc(proj, sid, view_scale)
    vd = N.vol_desc(dL_dvol.shape, spacing, origin)
    ctx = N.context(N.device_of(dL_dvol, proj, P))
    rc = N.lib().bp_vjp(ctx, N.ptr(dL_dvol), N.ptr(proj), ctypes.byref(pd), N.ptr(P),
                        N.ptr(motion), N.ptr(view_weight), N.WEIGHT[weight], N.DERIV[deriv],
                        ctypes.byref(vd), N.ptr(out_motion if want_motion else None),
                        N.ptr(out_Phat if want_Phat else None),
                        N.ptr(out_proj if want_proj else None), N.stream_of(dL_dvol, proj))
    N.check("bp_vjp", rc, ctx)
    return (out_motion if want_motion else None, out_Phat if want_Phat else None,
            out_proj if want_proj else None)


def bp_sharpness(vol, want_grad=True, loss_out=None, grad_out=None):
    """Sharpness loss and dL/dvol; returns (loss 0-d float64, grad | None)."""
    dev = vol.device if isinstance(vol, torch.Tensor) else torch.device("cpu")
    loss = loss_out if loss_out is not None else torch.empty((), dtype=torch.float64, device=dev)
    grad = grad_out if grad_out is not None else (torch.empty_like(vol) if want_grad else None)
    vd = N.vol_desc(vol.shape, (1, 1, 1), (0, 0, 0))
    ctx = N.context(N.device_of(vol))
    rc = N.lib().bp_sharpness(ctx, N.ptr(vol), ctypes.byref(vd), N.ptr(loss), N.ptr(grad),
                              N.stream_of(vol))
    N.check("bp_sharpness", rc, ctx)
    return loss, grad


def bp_tv(vol, eps=1e-3, want_grad=True, loss_out=None, grad_out=None):
    """Smoothed isotropic total variation and dL/dvol; returns (loss, grad | None)."""
    dev = vol.device if isinstance(vol, torch.Tensor) else torch.device("cpu")
    loss = loss_out if loss_out is not None else torch.empty((), dtype=torch.float64, device=dev)
    grad = grad_out if grad_out is not None else (torch.empty_like(vol) if want_grad else None)
    vd = N.vol_desc(vol.shape, (1, 1, 1), (0, 0, 0))
    ctx = N.context(N.device_of(vol))
    rc = N.lib().bp_tv(ctx, N.ptr(vol), ctypes.byref(vd), float(eps), N.ptr(loss), N.ptr(grad),
                       N.stream_of(vol))
    N.check("bp_tv", rc, ctx)
    return loss, grad


def bp_akima_motion(nodes, nviews, out=None):
    """Sec. II-B.1: theta (V,6) float64 from Akima spline nodes (N_n,6)."""
    nodes = _f64(nodes, "nodes")
    if out is None:
        out = torch.empty((nviews, 6), dtype=torch.float64, device=nodes.device)
    ctx = N.context(N.device_of(nodes, out))
    rc = N.lib().bp_akima_motion(ctx, nodes.shape[0], int(nviews), N.ptr(nodes), N.ptr(out),
                                 N.stream_of(nodes, out))
    N.check("bp_akima_motion", rc, ctx)
    return out


def bp_akima_motion_vjp(nodes, dL_dtheta, out=None):
    """dL/dnodes (N_n,6) = (dtheta/dnodes)^T dL/dtheta for the Akima motion model."""
    nodes = _f64(nodes, "nodes")
    g = _f64(dL_dtheta, "dL_dtheta")
    if out is None:
        out = torch.empty_like(nodes)
    ctx = N.context(N.device_of(nodes, g, out))
    rc = N.lib().bp_akima_motion_vjp(ctx, nodes.shape[0], g.shape[0], N.ptr(nodes), N.ptr(g),
                                     N.ptr(out), N.stream_of(nodes, g, out))
    N.check("bp_akima_motion_vjp", rc, ctx)
    return out


def bp_fdk_filter(raw, *, pitch, sid, sdd, arc, ext=0, out=None):
    """FDK preprocessing of raw line integrals (V,nv,nu) float32: cosine weight,
    short-scan (or full-scan 1/2) weights, optional truncation extension by
    `ext` pixels per side (linear fall-off to 0), Shepp-Logan ramp along rows."""
    if raw.dtype != torch.float32:
        raise TypeError("raw must be float32")
    raw = raw.contiguous()
    V, nv, nu = raw.shape
    if out is None:
        out = torch.empty_like(raw)
    ctx = N.context(N.device_of(raw, out))
    rc = N.lib().bp_fdk_filter(ctx, N.ptr(raw), V, nv, nu, float(pitch), float(sid), float(sdd),
                               float(arc), int(ext), N.ptr(out), N.stream_of(raw, out))
    N.check("bp_fdk_filter", rc, ctx)
    return out


def bp_gd_step(theta, grad, s0, t, n, gauge=True):
    """Eq. 6 step n in place on theta (V,6) float64."""
    ctx = N.context(N.device_of(theta))
    rc = N.lib().bp_gd_step(ctx, theta.shape[0], N.ptr(theta), N.ptr(grad), float(s0), float(t),
                            int(n), int(bool(gauge)), N.stream_of(theta))
    N.check("bp_gd_step", rc, ctx)
    return theta


def bp_adam_step(theta, grad, m1, m2, lr, n, beta1=0.9, beta2=0.999, eps=1e-8, gauge=True):
    """Adam step n (>= 1) in place on theta, m1, m2 (V,6) float64."""
    ctx = N.context(N.device_of(theta))
    rc = N.lib().bp_adam_step(ctx, theta.shape[0], N.ptr(theta), N.ptr(grad), N.ptr(m1),
                              N.ptr(m2), float(lr), float(beta1), float(beta2), float(eps), int(n),
                              int(bool(gauge)), N.stream_of(theta))
    N.check("bp_adam_step", rc, ctx)
    return theta
