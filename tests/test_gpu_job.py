"""Motion-estimation jobs (device-resident state, one CUDA graph per
iteration) against the step-by-step C-ABI calls and against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from cases import scan_case
from paper_2401_09283_gb300 import bp
from paper_2401_09283_gb300.job import MotionJob, set_hbm_budget

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


def c1_inputs():
    cfg, P, th_true, proj, _ = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    geo = dict(vol_shape=cfg.vol_shape, spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid)
    return cfg, P, th_true, proj, vw, geo


def test_job_graph_matches_step_by_step_calls():
    cfg, P, _, proj, vw, geo = c1_inputs()
    lr = 0.05
    n = 5
    job = MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), optimizer="adam", lr=lr,
                    lr_rot=lr, max_iters=8, **geo)
    job.step(n)
    th_job, hist, it = job.motion()
    assert it == n
    assert np.all(hist[n:] == 0.0) and np.all(hist[:n] < 0.0)
    # the same iterations through the single-call entry points
    p, Pd, vwd = cuda(proj), cuda(P), cuda(vw)
    theta = torch.zeros((cfg.views, 6), dtype=torch.float64, device=DEV)
    m1, m2 = torch.zeros_like(theta), torch.zeros_like(theta)
    losses = []
    for i in range(1, n + 1):
        vol = bp.bp_forward(p, Pd, theta, view_weight=vwd, weight="fdk", **geo)
        loss, dvol = bp.bp_sharpness(vol)
        losses.append(float(loss))
        gm, _, _ = bp.bp_vjp(dvol, p, Pd, theta, spacing=cfg.spacing3, origin=cfg.origin,
                             view_weight=vwd, weight="fdk", sid=cfg.sid)
        bp.bp_adam_step(theta, gm, m1, m2, lr, i)
    torch.cuda.synchronize()
    assert np.allclose(hist[:n], losses, rtol=1e-12, atol=0)
    assert np.abs(theta.cpu().numpy() - th_job).max() <= 1e-9
    job.close()


def test_job_gd_matches_oracle_loop():
    """Two steps of Eq. 6 (x <- x - s0 t^n df/dx) on c1 against the oracle's
    forward, loss, VJP, chain rule and step."""
    cfg, P, _, proj, vw, geo = c1_inputs()
    pj = proj.astype(np.float64)
    th = np.zeros((cfg.views, 6))
    # scale s0 so that the first step moves the largest parameter by 0.2
    Ph = oracle.compose(P, th)
    vol = oracle.bp_forward(Ph, pj, cfg.vol_shape, cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK,
                            cfg.sid)
    _, dvol = oracle.sharpness(vol)
    gP, _ = oracle.bp_vjp(Ph, pj, dvol, cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK,
                          oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
    g0 = oracle.chain_motion(P, th, gP)
    s0, t = 0.2 / np.abs(g0).max(), 0.97
    ths = []
    for n in range(2):
        Ph = oracle.compose(P, th)
        vol = oracle.bp_forward(Ph, pj, cfg.vol_shape, cfg.spacing3, cfg.origin, vw,
                                oracle.WEIGHT_FDK, cfg.sid)
        _, dvol = oracle.sharpness(vol)
        gP, _ = oracle.bp_vjp(Ph, pj, dvol, cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK,
                              oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
        g = oracle.chain_motion(P, th, gP)
        th = oracle.gd_step(th, g, s0, t, n)
        ths.append(th)
    job = MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), optimizer="gd", lr=s0, lr_rot=s0,
                    decay=t, max_iters=2, **geo)
    job.step(1)
    th1, _, _ = job.motion()
    job.step(1)
    th2, _, it = job.motion()
    assert it == 2
    for got, ref in ((th1, ths[0]), (th2, ths[1])):
        for sl in (slice(0, 3), slice(3, 6)):
            assert np.linalg.norm(got[:, sl] - ref[:, sl]) <= 2e-3 * np.linalg.norm(ref[:, sl])
    job.close()


def test_job_admission_by_hbm_budget():
    cfg, P, _, proj, vw, geo = c1_inputs()
    need = MotionJob.bytes_for(proj.shape, 0, cfg.vol_shape, "central", 10)
    set_hbm_budget(need - 1)
    with pytest.raises(RuntimeError, match="BP_ERR_OOM"):
        MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), max_iters=10, **geo)
    set_hbm_budget(2 * need - 1)
    a = MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), max_iters=10, **geo)
    assert a.nbytes == need
    with pytest.raises(RuntimeError, match="BP_ERR_OOM"):
        MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), max_iters=10, **geo)  # 2 x need
    a.close()
    b = MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), max_iters=10, **geo)  # freed: fits
    b.close()
    set_hbm_budget(0)


def test_job_from_host_memory_and_reduces_loss():
    cfg, P, _, proj, vw, geo = c1_inputs()
    job = MotionJob(torch.as_tensor(proj), torch.as_tensor(P), view_weight=torch.as_tensor(vw),
                    optimizer="adam", lr=0.1, lr_rot=2e-3, max_iters=30, device=0, **geo)
    job.step(30)
    th, hist, it = job.motion()
    assert it == 30 and np.isfinite(th).all()
    assert hist[-1] < hist[0]
    assert np.allclose(th.mean(axis=0), 0.0, atol=1e-12)  # gauge
    job.close()


def test_job_akima_model_matches_oracle_loop():
    """Two GD steps on the 6 N_n spline node values (Sec. II-B.1): theta from
    the splines, forward, loss, VJP, chain rule, spline VJP, Eq. 6 on nodes,
    gauge over nodes -- against the same loop through the oracle."""
    cfg, P, _, proj, vw, geo = c1_inputs()
    pj = proj.astype(np.float64)
    nn = 6
    rng = np.random.default_rng(11)
    x = rng.standard_normal((nn, 6)) * np.array([0.5, 0.5, 0.5, 0.005, 0.005, 0.005])
    x -= x.mean(axis=0)

    def grad_nodes(x):
        th = oracle.akima_motion(x, cfg.views)
        Ph = oracle.compose(P, th)
        vol = oracle.bp_forward(Ph, pj, cfg.vol_shape, cfg.spacing3, cfg.origin, vw,
                                oracle.WEIGHT_FDK, cfg.sid)
        _, dvol = oracle.sharpness(vol)
        gP, _ = oracle.bp_vjp(Ph, pj, dvol, cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK,
                              oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
        return oracle.akima_motion_vjp(x, cfg.views, oracle.chain_motion(P, th, gP))

    g0 = grad_nodes(x)
    s0, t = 0.2 / np.abs(g0).max(), 0.97
    xs, xo = [], x.copy()
    for n in range(2):
        xo = oracle.gd_step(xo, grad_nodes(xo), s0, t, n)
        xs.append(xo)
    job = MotionJob(cuda(proj), cuda(P), view_weight=cuda(vw), optimizer="gd", lr=s0, lr_rot=s0,
                    decay=t, max_iters=2, theta0=cuda(x), motion_nodes=nn, **geo)
    for want in xs:
        job.step(1)
        got = job.node_values()
        for sl in (slice(0, 3), slice(3, 6)):
            assert np.linalg.norm(got[:, sl] - want[:, sl]) <= 2e-3 * np.linalg.norm(want[:, sl])
    th, _, it = job.motion()
    assert it == 2
    assert np.abs(th - oracle.akima_motion(job.node_values(), cfg.views)).max() < 1e-12
    job.close()
