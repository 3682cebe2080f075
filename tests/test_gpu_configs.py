"""Parity against the FP64 oracle on the configurations the other GPU tests
do not reach at full size:

* c4 (192^3 at 1.33 mm, 180 views, 320x240, FP32): the whole volume, the
  motion gradient of every view and the data VJP, element by element;
* the paper's own setup (Sec. III-IV): 128^3 at 2 mm, 360 views over the
  full circle (c_j = 2 pi / V), SID 785 mm, 700x500 detector at 0.64 mm;
* serving jobs (c5) in FP16 storage with a per-view scale: the smallest
  size (128^3, 120 views) in full and the largest (384^3, 496 views,
  488x366 at 0.853 mm) on sampled sub-blocks and views.

Every comparison also reports the worst per-view relative error of the
motion gradient beside the rel-L2 of each parameter group.  The scans are
simulated by the input generator on the GPU through torch (closed-form line
integrals and FFT filtering; none of it is the library's code) with the
moved geometry composed by the oracle.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from cases import motion_errors, per_view_worst, rel_l2
from paper_2401_09283_gb300 import bp
from paper_2401_09283_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")
VOL_TOL = 1e-5
FP16_TOL = 2e-3
GRAD_TOL = 1e-3


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


@functools.lru_cache(maxsize=None)
def simulated(cfg):
    """(P, theta*, filtered projections float32 numpy) of a config; the
    data is simulated through the moved matrices P_j T(theta*_j)."""
    P = W.projection_matrices(cfg)
    th = W.motion_curves(cfg)
    sc = W.make_scan(cfg, moved_P=oracle.compose(P, th), device=DEV)
    proj = sc.proj.float().cpu().numpy()
    torch.cuda.empty_cache()
    return P, th, proj


def geo(cfg):
    return dict(spacing=cfg.spacing3, origin=cfg.origin, weight="fdk", sid=cfg.sid)


def sub_origin(cfg, k0, j0, i0):
    o = cfg.origin
    return (o[0] + i0 * cfg.spacing, o[1] + j0 * cfg.spacing, o[2] + k0 * cfg.spacing)


def report(name, errs):
    print("%s motion gradient: rel-L2 translations %.3g, rotations %.3g, worst view %.3g"
          % ((name,) + tuple(errs)))


def check_full(cfg, proj_gpu, proj_ref, P, th, vw, scale=None, data_views=None):
    """Forward (whole volume), motion gradient (every view) and data VJP
    (`data_views`, default all) of the GPU path against the oracle on
    proj_ref (the FP32 data, or the dequantised stored data)."""
    g = geo(cfg)
    sc = None if scale is None else cuda(scale)
    vol = bp.bp_forward(proj_gpu, cuda(P), cuda(th), vol_shape=cfg.vol_shape,
                        view_weight=cuda(vw), view_scale=sc, **g).cpu().numpy()
    Ph = oracle.compose(P, th)
    ref = oracle.bp_forward(Ph, proj_ref, cfg.vol_shape, cfg.spacing3, cfg.origin, vw,
                            oracle.WEIGHT_FDK, cfg.sid)
    e_vol = rel_l2(vol, ref)
    print("%s volume rel-L2 %.3g" % (cfg.name, e_vol))
    assert e_vol <= VOL_TOL
    delta = W.upstream_gradient(cfg)
    gm, gP, gD = bp.bp_vjp(cuda(delta), proj_gpu, cuda(P), cuda(th), view_weight=cuda(vw),
                           view_scale=sc, want_Phat=True, want_proj=True, **g)
    gm, gP, gD = gm.cpu().numpy(), gP.cpu().numpy(), gD.cpu().numpy()
    full_data = data_views is None
    oP, oD = oracle.bp_vjp(Ph, proj_ref, delta.astype(np.float64), cfg.spacing3, cfg.origin, vw,
                           oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid, want_proj=full_data)
    om = oracle.chain_motion(P, th, oP)
    errs = motion_errors(gm, om)
    report(cfg.name, errs)
    assert max(errs) <= GRAD_TOL
    assert rel_l2(gP, oP) <= GRAD_TOL and per_view_worst(gP, oP) <= GRAD_TOL
    if not full_data:
        sel = np.asarray(data_views)
        _, oD = oracle.bp_vjp(Ph[sel], proj_ref[sel], delta.astype(np.float64), cfg.spacing3,
                              cfg.origin, vw[sel], oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL,
                              cfg.sid, want_P=False)
        gD = gD[sel]
    e_d = rel_l2(gD, oD)
    print("%s data VJP rel-L2 %.3g" % (cfg.name, e_d))
    assert e_d <= VOL_TOL


def test_c4_full_size():
    """Config 4 at full size, FP32: every voxel, every view."""
    cfg = W.C4
    P, th, proj = simulated(cfg)
    vw = np.full(cfg.views, cfg.delta_beta)
    check_full(cfg, cuda(proj), proj.astype(np.float64), P, th, vw)


def test_paper_geometry_full_scan():
    """The paper's own setup: full 2 pi scan (redundancy weight 1/2 folded
    into the filtered data, c_j = 2 pi / V), SID 785 mm, 700 x 500 detector.
    Whole volume and every view's motion gradient; the data VJP of 12 views."""
    cfg = W.PAPER
    P, th, proj = simulated(cfg)
    vw = np.full(cfg.views, cfg.delta_beta)
    assert abs(vw.sum() - 2 * np.pi) < 1e-12
    views = np.linspace(0, cfg.views - 1, 12).astype(int)
    check_full(cfg, cuda(proj), proj.astype(np.float64), P, th, vw, data_views=views)


def half_storage(proj):
    """FP16 storage with a per-view scale (max |value| of the view), as the
    serving form stores its requests: (stored fp16 tensor on the GPU,
    scale float32, dequantised data float64)."""
    V = proj.shape[0]
    scale = np.maximum(np.abs(proj).reshape(V, -1).max(axis=1), 1e-30).astype(np.float32)
    stored = torch.as_tensor(proj / scale[:, None, None]).half()
    deq = stored.float().numpy().astype(np.float64) * scale[:, None, None]
    return stored.to(DEV), scale, deq


def test_serving_job_smallest_fp16():
    """Serving job of 128^3 voxels (2 mm) and 120 views, FP16 storage: the
    whole volume against the oracle on the stored data (kernel arithmetic,
    1e-5) and on the FP32 data (storage error, 2e-3); every view's motion
    gradient."""
    cfg = W.serving_job_config(0, 128, 120)
    P, th, proj = simulated(cfg)
    vw = np.full(cfg.views, cfg.delta_beta)
    stored, scale, deq = half_storage(proj)
    check_full(cfg, stored, deq, P, th, vw, scale=scale)
    vol = bp.bp_forward(stored, cuda(P), cuda(th), vol_shape=cfg.vol_shape, view_weight=cuda(vw),
                        view_scale=cuda(scale), **geo(cfg)).cpu().numpy()
    ref32 = oracle.bp_forward(oracle.compose(P, th), proj.astype(np.float64), cfg.vol_shape,
                              cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK, cfg.sid)
    e32 = rel_l2(vol, ref32)
    print("%s FP16 storage error of the volume %.3g" % (cfg.name, e32))
    assert e32 <= FP16_TOL


def test_serving_job_largest_fp16_sampled():
    """The largest serving job (384^3 at 0.667 mm, 496 views, 488 x 366 at
    0.853 mm), FP16 storage, in the launch configuration of a served job:
    the forward over the whole volume compared on two seeded 32^3
    sub-blocks; the motion gradient and the data VJP of 16 seeded views
    over the whole volume (a view's sums depend on that view only)."""
    cfg = W.serving_job_config(1, 384, 496)
    assert (cfg.nu, cfg.nv) == (488, 366)
    P, th, proj = simulated(cfg)
    vw = np.full(cfg.views, cfg.delta_beta)
    stored, scale, deq = half_storage(proj)
    g = geo(cfg)
    vol = bp.bp_forward(stored, cuda(P), cuda(th), vol_shape=cfg.vol_shape, view_weight=cuda(vw),
                        view_scale=cuda(scale), **g).cpu().numpy()
    Ph = oracle.compose(P, th)
    rng = np.random.default_rng(51)
    n = 32
    for _ in range(2):
        k0, j0, i0 = (int(rng.integers(0, cfg.n - n)) for _ in range(3))
        so = sub_origin(cfg, k0, j0, i0)
        got = vol[k0:k0 + n, j0:j0 + n, i0:i0 + n]
        refq = oracle.bp_forward(Ph, deq, (n, n, n), cfg.spacing3, so, vw, oracle.WEIGHT_FDK,
                                 cfg.sid)
        ref32 = oracle.bp_forward(Ph, proj.astype(np.float64), (n, n, n), cfg.spacing3, so, vw,
                                  oracle.WEIGHT_FDK, cfg.sid)
        eq, e32 = rel_l2(got, refq), rel_l2(got, ref32)
        print("%s sub-block %s: vs stored data %.3g, vs FP32 data %.3g" % (cfg.name, (k0, j0, i0),
                                                                          eq, e32))
        assert eq <= VOL_TOL
        assert e32 <= FP16_TOL
    delta = W.upstream_gradient(cfg)
    gm, gP, gD = bp.bp_vjp(cuda(delta), stored, cuda(P), cuda(th), view_weight=cuda(vw),
                           view_scale=cuda(scale), want_Phat=True, want_proj=True, **g)
    sel = np.sort(rng.choice(cfg.views, 16, replace=False))
    gm, gP, gD = gm.cpu().numpy()[sel], gP.cpu().numpy()[sel], gD[torch.as_tensor(sel)].cpu().numpy()
    oP, oD = oracle.bp_vjp(Ph[sel], deq[sel], delta.astype(np.float64), cfg.spacing3, cfg.origin,
                           vw[sel], oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid)
    om = oracle.chain_motion(P[sel], th[sel], oP)
    errs = motion_errors(gm, om)
    report(cfg.name, errs)
    assert max(errs) <= GRAD_TOL
    assert rel_l2(gP, oP) <= GRAD_TOL
    e_d = rel_l2(gD, oD)
    print("%s data VJP rel-L2 %.3g" % (cfg.name, e_d))
    assert e_d <= VOL_TOL
