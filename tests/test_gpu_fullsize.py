"""Parity at full size, in the launch configuration the benchmark times:
the oracle computes sampled outputs one by one.

c2 (256^3, 248 views, 616x480, FP32, FDK): the forward on 16^3 sub-blocks;
the motion gradient and the data VJP of sampled views over the whole volume
(a view's 12 sums and its image depend on that view only).
c3 (512^3 at 0.5 mm, 496 views, 1240x960) in FP16 and BF16 storage with a
per-view scale: a seeded 64^3 sub-block and 32 seeded views.
"""
import numpy as np
import pytest
import torch

import oracle
from cases import BF16_STORAGE_TOL, FP16_STORAGE_TOL, motion_errors, rel_l2, scan_case
from paper_2401_09283_gb300 import bp
from paper_2401_09283_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


def sub_origin(cfg, k0, j0, i0):
    o = cfg.origin
    return (o[0] + i0 * cfg.spacing, o[1] + j0 * cfg.spacing, o[2] + k0 * cfg.spacing)


def test_c2_full_size_sampled():
    cfg, P, th, proj, _ = scan_case("c2")
    vw = np.full(cfg.views, cfg.delta_beta)
    geo = dict(spacing=cfg.spacing3, origin=cfg.origin, weight="fdk", sid=cfg.sid)
    pd, Pd, thd, vwd = cuda(proj), cuda(P), cuda(th), cuda(vw)
    vol = bp.bp_forward(pd, Pd, thd, vol_shape=cfg.vol_shape, view_weight=vwd, **geo)
    vol = vol.cpu().numpy()
    Ph = oracle.compose(P, th)
    pj = proj.astype(np.float64)
    rng = np.random.default_rng(22)
    n = 16
    for _ in range(3):
        k0, j0, i0 = (int(rng.integers(0, cfg.n - n)) for _ in range(3))
        ref = oracle.bp_forward(Ph, pj, (n, n, n), cfg.spacing3, sub_origin(cfg, k0, j0, i0), vw,
                                oracle.WEIGHT_FDK, cfg.sid)
        got = vol[k0:k0 + n, j0:j0 + n, i0:i0 + n]
        assert rel_l2(got, ref) <= 1e-5
    # motion gradient and data VJP (fused kernel) of sampled views
    delta = W.upstream_gradient(cfg)
    gm, gP, gD = bp.bp_vjp(cuda(delta), pd, Pd, thd, view_weight=vwd, want_Phat=True,
                           want_proj=True, **geo)
    gm, gP, gD = gm.cpu().numpy(), gP.cpu().numpy(), gD.cpu().numpy()
    views = np.sort(rng.choice(cfg.views, 4, replace=False))
    oP, oD = oracle.bp_vjp(Ph[views], pj[views], delta.astype(np.float64), cfg.spacing3,
                           cfg.origin, vw[views], oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL,
                           cfg.sid)
    om = oracle.chain_motion(P[views], th[views], oP)
    assert rel_l2(gP[views], oP) <= 1e-3
    errs = motion_errors(gm[views], om)
    print("c2 motion gradient: rel-L2 translations %.3g, rotations %.3g, worst view %.3g" % errs)
    assert max(errs) <= 1e-3
    assert rel_l2(gD[views], oD) <= 1e-5


@pytest.mark.parametrize("dtype,tol", [(torch.float16, FP16_STORAGE_TOL),
                                       (torch.bfloat16, BF16_STORAGE_TOL)])
def test_c3_half_storage_sampled(dtype, tol):
    rng = np.random.default_rng(3)
    cfg = W.C3
    views = tuple(int(v) for v in np.sort(rng.choice(cfg.views, 32, replace=False)))
    _, P, th, proj, _ = scan_case("c3", views=views)
    sel = np.array(views)
    P, th = P[sel], th[sel]
    n = 64
    k0, j0, i0 = (int(rng.integers(0, cfg.n - n)) for _ in range(3))
    vw = np.full(len(sel), cfg.delta_beta)
    scale = np.maximum(np.abs(proj).reshape(len(sel), -1).max(axis=1), 1e-30).astype(np.float32)
    stored = torch.as_tensor(proj / scale[:, None, None]).to(dtype)
    deq = stored.float().numpy().astype(np.float64) * scale[:, None, None]
    # GPU: the whole 512^3 volume from the 32 views; compare the sub-block
    vol = bp.bp_forward(stored.to(DEV), cuda(P), cuda(th), vol_shape=cfg.vol_shape,
                        spacing=cfg.spacing3, origin=cfg.origin, view_weight=cuda(vw),
                        weight="fdk", sid=cfg.sid, view_scale=cuda(scale)).cpu().numpy()
    got = vol[k0:k0 + n, j0:j0 + n, i0:i0 + n]
    Ph = oracle.compose(P, th)
    so = sub_origin(cfg, k0, j0, i0)
    ref32 = oracle.bp_forward(Ph, proj.astype(np.float64), (n, n, n), cfg.spacing3, so, vw,
                              oracle.WEIGHT_FDK, cfg.sid)
    refq = oracle.bp_forward(Ph, deq, (n, n, n), cfg.spacing3, so, vw, oracle.WEIGHT_FDK, cfg.sid)
    e_q, e_32 = rel_l2(got, refq), rel_l2(got, ref32)
    print("c3 %s volume rel-L2: vs oracle on stored data %.3g, vs FP32 data %.3g" % (dtype, e_q, e_32))
    assert e_q <= 1e-5
    assert e_32 <= tol
    # motion gradient of the sub-block (upstream gradient zero elsewhere)
    delta = np.zeros(cfg.vol_shape, np.float32)
    delta[k0:k0 + n, j0:j0 + n, i0:i0 + n] = rng.standard_normal((n, n, n))
    gm, _, _ = bp.bp_vjp(cuda(delta), stored.to(DEV), cuda(P), cuda(th), spacing=cfg.spacing3,
                         origin=cfg.origin, view_weight=cuda(vw), weight="fdk", sid=cfg.sid,
                         view_scale=cuda(scale))
    oP, _ = oracle.bp_vjp(Ph, deq, delta[k0:k0 + n, j0:j0 + n, i0:i0 + n].astype(np.float64),
                          cfg.spacing3, so, vw, oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid,
                          want_proj=False)
    om = oracle.chain_motion(P, th, oP)
    g = gm.cpu().numpy()
    errs = motion_errors(g, om)
    print("c3 %s motion gradient: rel-L2 translations %.3g, rotations %.3g, worst view %.3g"
          % ((dtype,) + errs))
    assert max(errs) <= 1e-3
