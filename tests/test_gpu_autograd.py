"""The autograd wrapper (differentiation form, config 4): gradients w.r.t.
motion and projections against finite differences and torch's gradcheck."""
import numpy as np
import pytest
import torch

import oracle
from cases import scan_case
from paper_2401_09283_gb300.autograd import backproject

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")


def setup(name):
    cfg, P, th, proj, delta = scan_case(name)
    t = lambda x: torch.as_tensor(np.ascontiguousarray(x)).to(DEV)
    args = dict(vol_shape=cfg.vol_shape, spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid,
                view_weight=t(np.full(cfg.views, cfg.delta_beta)), weight="fdk")
    return cfg, t(P), t(th), t(proj), t(delta), args


def test_backward_matches_the_vjp_and_oracle_c4g():
    cfg, P, th, proj, delta, args = setup("c4g")
    proj = proj.clone().requires_grad_(True)
    th = th.clone().requires_grad_(True)
    vol = backproject(proj, th, P, deriv="exact", **args)
    (vol.double() * delta.double()).sum().backward()
    Pn, thn = P.cpu().numpy(), th.detach().cpu().numpy()
    Ph = oracle.compose(Pn, thn)
    vw = args["view_weight"].cpu().numpy()
    oP, oD = oracle.bp_vjp(Ph, proj.detach().cpu().numpy().astype(np.float64),
                           delta.cpu().numpy().astype(np.float64), cfg.spacing3, cfg.origin, vw,
                           oracle.WEIGHT_FDK, oracle.DERIV_BILINEAR_EXACT, cfg.sid)
    om = oracle.chain_motion(Pn, thn, oP)
    g = th.grad.cpu().numpy()
    for sl in (slice(0, 3), slice(3, 6)):
        assert np.linalg.norm(g[:, sl] - om[:, sl]) <= 1e-3 * np.linalg.norm(om[:, sl])
    gd = proj.grad.cpu().numpy()
    assert np.linalg.norm(gd - oD) <= 1e-5 * np.linalg.norm(oD)


def test_gradcheck_motion_c4g():
    """torch.autograd.gradcheck on the 16^3 / 12-view / 32x24 instance, motion
    in FP64 (kernels in FP32).  Fast mode compares directional derivatives
    v^T J u, so the rare bilinear kinks average out; eps and the tolerances
    are set for FP32 arithmetic."""
    cfg, P, th, proj, _, args = setup("c4g")
    th = th.clone().requires_grad_(True)

    def f(m):
        return backproject(proj, m, P, deriv="exact", **args).double()

    assert torch.autograd.gradcheck(f, (th,), eps=1e-4, atol=2e-3, rtol=2e-2, fast_mode=True,
                                    nondet_tol=1e-6)


def test_gradcheck_projections_c4g():
    """torch.autograd.gradcheck over the projections on the c4g instance, in
    full (non-fast) mode: every one of the 12 x 24 x 32 inputs against every
    output voxel.  The backprojection is linear in the data, so a central
    difference with eps = 1 has no truncation error and its only error is
    the FP32 rounding of the two forwards (about 1e-7 absolute on values of
    order 1); the Jacobian entries are bilinear weights times c_j (sid/w)^2,
    at most about 0.3.  Tolerances: 1e-5 absolute plus 1e-4 relative.  The
    data VJP sums with FP32 atomics, so two backward passes may differ in
    the last bits (nondet_tol)."""
    cfg, P, th, proj, _, args = setup("c4g")
    p64 = proj.double().clone().requires_grad_(True)

    def f(p):
        return backproject(p.float(), th, P, deriv="exact", **args).double()

    assert torch.autograd.gradcheck(f, (p64,), eps=1.0, atol=1e-5, rtol=1e-4, fast_mode=False,
                                    nondet_tol=1e-6)


@pytest.mark.slow
def test_fd_24_motion_parameters_c4():
    """Config 4 (192^3, 180 views, 320x240): the autograd gradient of
    L = <delta, vol> (FP32 kernels, exact bilinear derivative) on 24 seeded
    parameters against central finite differences.  A view's parameters
    change only that view's backprojection, so the FD is taken on the FP64
    oracle's single-view forward (FD of FP32 volumes is rounding-dominated).

    Bilinear interpolation has kinks at pixel boundaries.  At the config's
    h = 1e-3 mm / 1e-4 rad a voxel 128 mm off-axis moves 0.016 px per step,
    so a few % of the voxel-views straddle a boundary and the FD is
    kink-limited (measured median ~3e-2 on this phantom data); at
    h = 1e-7 mm / 1e-9 rad, still well above FP64 rounding for a 7e6-term
    sum, the FD converges to the derivative."""
    cfg, P, th, proj, delta, args = setup("c4")
    thg = th.clone().requires_grad_(True)
    vol = backproject(proj, thg, P, deriv="exact", **args)
    (vol.double() * delta.double()).sum().backward()
    g = thg.grad.cpu().numpy()
    Pn, thn = P.cpu().numpy(), th.cpu().numpy()
    pj = proj.cpu().numpy().astype(np.float64)
    dl = delta.cpu().numpy().astype(np.float64)
    vw = args["view_weight"].cpu().numpy()
    rng = np.random.default_rng(24)
    picks = [(int(rng.integers(cfg.views)), int(rng.integers(6))) for _ in range(24)]

    def fd(j, m, h):
        def L(tj):
            Ph = oracle.compose(Pn[j:j + 1], tj[None])
            v = oracle.bp_forward(Ph, pj[j:j + 1], cfg.vol_shape, cfg.spacing3, cfg.origin,
                                  vw[j:j + 1], oracle.WEIGHT_FDK, cfg.sid)
            return float(np.sum(dl * v))
        tp, tm = thn[j].copy(), thn[j].copy()
        tp[m] += h
        tm[m] -= h
        return (L(tp) - L(tm)) / (2 * h)

    fine, coarse = [], []
    for j, m in picks:
        scale = np.abs(g[:, m]).max()
        for out, h in ((fine, 1e-7 if m < 3 else 1e-9), (coarse, 1e-3 if m < 3 else 1e-4)):
            f = fd(j, m, h)
            out.append(abs(f - g[j, m]) / max(abs(f), 1e-2 * scale))
    fine, coarse = np.array(fine), np.array(coarse)
    assert np.median(fine) < 1e-3, fine
    assert np.mean(fine < 1e-2) >= 0.9, fine
    assert np.median(coarse) < 1e-1, coarse


def test_fd_projection_gradient_c4g():
    cfg, P, th, proj, delta, args = setup("c4g")
    pg = proj.clone().requires_grad_(True)
    vol = backproject(pg, th, P, **args)
    (vol.double() * delta.double()).sum().backward()
    g = pg.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    with torch.no_grad():
        for _ in range(10):
            idx = tuple(int(rng.integers(n)) for n in proj.shape)
            h = 0.5
            pp, pm = proj.clone(), proj.clone()
            pp[idx] += h
            pm[idx] -= h
            Lp = (backproject(pp, th, P, **args).double() * delta.double()).sum().item()
            Lm = (backproject(pm, th, P, **args).double() * delta.double()).sum().item()
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-4 * max(1.0, np.abs(g).max())
