"""Differentiable backprojection: a torch.autograd.Function over the C-ABI.

forward  = bp_forward (Eq. 3 with the motion composition of Eq. 1);
backward = bp_vjp: dL/dmotion through Eqs. 4-5 and the chain rule (Eq. 2),
           dL/dproj as the adjoint of Eq. 3.
Only the inputs are saved; projected coordinates are recomputed in backward,
as the paper does to avoid the full Jacobian (Sec. II-B.2 and Sec. V).
With deriv="exact" the backward is the exact derivative of the bilinear
forward (use it for gradient checks); deriv="central" uses the paper's
central-difference gradient images.
"""
from __future__ import annotations

import torch

from . import bp


class _Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, proj, motion, P, vol_shape, spacing, origin, sid, view_weight, weight, deriv):
        vol = bp.bp_forward(proj.contiguous(), P, motion.contiguous(), vol_shape=vol_shape,
                            spacing=spacing, origin=origin, view_weight=view_weight,
                            weight=weight, sid=sid)
        ctx.save_for_backward(proj, motion, P, view_weight)
        ctx.geo = (spacing, origin, sid, weight, deriv)
        return vol

    @staticmethod
    def backward(ctx, gvol):
        proj, motion, P, view_weight = ctx.saved_tensors
        spacing, origin, sid, weight, deriv = ctx.geo
        want_p, want_m = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_p or want_m):
            return (None,) * 10
        gm, _, gd = bp.bp_vjp(gvol.contiguous().to(torch.float32), proj.contiguous(), P,
                              motion.contiguous(), spacing=spacing, origin=origin,
                              view_weight=view_weight, weight=weight, deriv=deriv, sid=sid,
                              want_motion=want_m, want_Phat=False, want_proj=want_p)
        if gd is not None:
            gd = gd.to(proj.dtype)
        return gd, gm, None, None, None, None, None, None, None, None


def backproject(proj, motion, P, *, vol_shape, spacing, origin, sid, view_weight=None,
                weight="fdk", deriv="central"):
    """Differentiable w.r.t. proj (V,nv,nu) and motion (V,6) float64."""
    return _Backproject.apply(proj, motion, P, tuple(vol_shape), tuple(spacing), tuple(origin),
                              float(sid), view_weight, weight, deriv)


class _AkimaMotion(torch.autograd.Function):
    @staticmethod
    def forward(ctx, nodes, nviews):
        ctx.save_for_backward(nodes)
        return bp.bp_akima_motion(nodes.contiguous(), nviews)

    @staticmethod
    def backward(ctx, gtheta):
        (nodes,) = ctx.saved_tensors
        return bp.bp_akima_motion_vjp(nodes.contiguous(), gtheta.contiguous()), None


def akima_motion(nodes, nviews):
    """Motion model of Sec. II-B.1 as a differentiable function: per-view
    theta (V,6) from Akima spline node values (N_n,6), float64.  Chain it into
    `backproject` to optimise the 6 N_n node values instead of 6 V
    per-view parameters."""
    return _AkimaMotion.apply(nodes, int(nviews))
