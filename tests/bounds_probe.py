"""Run by tests/test_gpu_bounds.py in a child process whose BP_GB300_LIB
points at the bounds-checking debug build: forward and VJP cases that reach
every staging and edge path (c1 with both derivative modes and both
weights, fused data VJP, ragged sizes, a volume far larger than the
detector's field, FP16 and BF16 staging), against the FP64 oracle; then the
device flag word, then the self test of the reporting path.  Prints one JSON
line."""
import ctypes
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from cases import random_case, rel_l2, scan_case  # noqa: E402
from paper_2401_09283_gb300 import bp  # noqa: E402
from paper_2401_09283_gb300 import native as N  # noqa: E402

DEV = torch.device("cuda:0")


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


def status(op):
    flags, first = ctypes.c_uint(), ctypes.c_longlong()
    ctx = N.context(0)
    N.check("bp_bounds_check", N.lib().bp_bounds_check(ctx, op, ctypes.byref(flags),
                                                       ctypes.byref(first)), ctx)
    return int(flags.value), int(first.value)


def case(proj, P, th, vol_shape, spacing, origin, vw, weight, deriv, sid, dtype=torch.float32):
    mode = oracle.WEIGHT_FDK if weight == "fdk" else oracle.WEIGHT_NONE
    dmode = oracle.DERIV_CENTRAL if deriv == "central" else oracle.DERIV_BILINEAR_EXACT
    scale = None
    pj = proj.astype(np.float64)
    p = cuda(proj)
    if dtype != torch.float32:
        sc = np.maximum(np.abs(proj).reshape(len(proj), -1).max(axis=1), 1e-30).astype(np.float32)
        stored = torch.as_tensor(proj / sc[:, None, None]).to(dtype)
        pj = stored.float().numpy().astype(np.float64) * sc[:, None, None]
        p, scale = stored.to(DEV), cuda(sc)
    geo = dict(spacing=spacing, origin=origin, view_weight=cuda(vw), weight=weight, sid=sid,
               view_scale=scale)
    vol = bp.bp_forward(p, cuda(P), cuda(th), vol_shape=vol_shape, **geo).cpu().numpy()
    Ph = oracle.compose(P, th)
    ref = oracle.bp_forward(Ph, pj, vol_shape, spacing, origin, vw, mode, sid)
    rng = np.random.default_rng(3)
    delta = rng.standard_normal(vol_shape).astype(np.float32)
    gm, gP, gD = bp.bp_vjp(cuda(delta), p, cuda(P), cuda(th), deriv=deriv, want_Phat=True,
                           want_proj=True, **geo)
    oP, oD = oracle.bp_vjp(Ph, pj, delta.astype(np.float64), spacing, origin, vw, mode, dmode, sid)
    return max(rel_l2(vol, ref), rel_l2(gD.cpu().numpy(), oD)), rel_l2(gP.cpu().numpy(), oP)


def main():
    out = {"library": N.library_path(), "cases": []}
    cfg, P, th, proj, _ = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    for weight in ("fdk", "none"):
        for deriv in ("central", "exact"):
            e = case(proj, P, th, cfg.vol_shape, cfg.spacing3, cfg.origin, vw, weight, deriv,
                     cfg.sid)
            out["cases"].append(["c1-%s-%s" % (weight, deriv), e])
    for dt in (torch.float16, torch.bfloat16):
        e = case(proj, P, th, cfg.vol_shape, cfg.spacing3, cfg.origin, vw, "fdk", "central",
                 cfg.sid, dt)
        out["cases"].append(["c1-%s" % str(dt), e])
    for seed, shape in ((5, (19, 21, 37)), (6, (40, 44, 48))):
        rc, P2, th2, proj2, _, origin = random_case(seed, shape=shape)
        vw2 = np.full(rc.views, rc.delta_beta)
        e = case(proj2, P2, th2, shape, (rc.spacing,) * 3, origin, vw2, "fdk", "central", rc.sid)
        out["cases"].append(["ragged-%d" % seed, e])
    # a volume much larger than the field of view: edge, skipped and unbounded tiles
    big = (48, 96, 96)
    o = tuple(-(n - 1) / 2.0 * 2.5 for n in big[::-1])
    e = case(proj, P, th, big, (2.5,) * 3, o, vw, "fdk", "central", cfg.sid)
    out["cases"].append(["wide-field", e])
    torch.cuda.synchronize()
    out["flags"], out["first"] = status(1)
    out["selftest"] = status(2)
    out["cleared"] = status(1) and status(0)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
