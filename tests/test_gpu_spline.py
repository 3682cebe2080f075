"""The Akima spline motion model on the GPU (Sec. II-B.1): values and the
reverse-mode VJP against the oracle's spline and its forward-mode
Jacobian, chained with the backprojection VJP through autograd."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _nodes(rng, n):
    return rng.standard_normal((n, 6)) * np.array([3, 3, 3, 0.03, 0.03, 0.03])


@pytest.mark.parametrize("n,V", [(3, 2), (3, 60), (6, 60), (12, 248), (30, 496), (30, 31),
                                 (40, 25), (512, 1500)])
def test_values_and_vjp_match_oracle(n, V):
    from paper_2401_09283_gb300 import bp
    rng = np.random.default_rng(n * 1000 + V)
    nodes = _nodes(rng, n)
    th = bp.bp_akima_motion(torch.as_tensor(nodes, device=DEV), V).cpu().numpy()
    ref = oracle.akima_motion(nodes, V)
    assert np.max(np.abs(th - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))
    g = rng.standard_normal((V, 6))
    got = bp.bp_akima_motion_vjp(torch.as_tensor(nodes, device=DEV),
                                 torch.as_tensor(g, device=DEV)).cpu().numpy()
    want = oracle.akima_motion_vjp(nodes, V, g)
    assert np.max(np.abs(got - want)) <= 1e-10 * (1 + np.max(np.abs(want)))


def test_flat_nodes_degenerate_weights():
    from paper_2401_09283_gb300 import bp
    nodes = np.zeros((9, 6))
    nodes[5:, 0] = [1.0, 2.0, 3.0, 3.5]   # flat stretch then a ramp: zero weight sums
    nodes[:, 1] = np.arange(9) * 0.25      # a line
    V = 100
    th = bp.bp_akima_motion(torch.as_tensor(nodes, device=DEV), V).cpu().numpy()
    assert np.max(np.abs(th - oracle.akima_motion(nodes, V))) < 1e-12
    g = np.random.default_rng(0).standard_normal((V, 6))
    got = bp.bp_akima_motion_vjp(torch.as_tensor(nodes, device=DEV),
                                 torch.as_tensor(g, device=DEV)).cpu().numpy()
    assert np.max(np.abs(got - oracle.akima_motion_vjp(nodes, V, g))) < 1e-10


def test_host_arrays_and_invalid_arguments():
    from paper_2401_09283_gb300 import bp, native as N
    rng = np.random.default_rng(5)
    nodes = _nodes(rng, 8)
    th = bp.bp_akima_motion(torch.as_tensor(nodes), 50)   # host in, host out
    assert np.max(np.abs(th.numpy() - oracle.akima_motion(nodes, 50))) < 1e-12
    for n, V in [(2, 50), (8, 1), (513, 2000)]:
        with pytest.raises(N.BPError):
            bp.bp_akima_motion(torch.zeros((n, 6), dtype=torch.float64, device=DEV), V)


def test_autograd_chain_matches_oracle_spline_jacobian():
    from paper_2401_09283_gb300.autograd import akima_motion
    rng = np.random.default_rng(7)
    n, V = 10, 120
    nodes = torch.as_tensor(_nodes(rng, n), device=DEV).requires_grad_(True)
    w = torch.as_tensor(rng.standard_normal((V, 6)), device=DEV)
    (akima_motion(nodes, V) * w).sum().backward()
    want = oracle.akima_motion_vjp(nodes.detach().cpu().numpy(), V, w.cpu().numpy())
    assert np.max(np.abs(nodes.grad.cpu().numpy() - want)) < 1e-10


def test_spline_model_through_backprojection_matches_oracle():
    """nodes -> Akima theta -> backprojection -> loss, differentiated by the
    autograd chain (spline VJP after the motion VJP), against the oracle's
    Jacobian chain on c1."""
    from cases import scan_case
    from paper_2401_09283_gb300.autograd import akima_motion, backproject
    cfg, P, _, proj, delta = scan_case("c1")
    rng = np.random.default_rng(9)
    x = _nodes(rng, 6) * 0.3
    vw = np.full(cfg.views, cfg.delta_beta)
    nodes = torch.as_tensor(x, device=DEV).requires_grad_(True)
    theta = akima_motion(nodes, cfg.views)
    vol = backproject(torch.as_tensor(proj, device=DEV), theta, torch.as_tensor(P, device=DEV),
                      vol_shape=cfg.vol_shape, spacing=cfg.spacing3, origin=cfg.origin,
                      sid=cfg.sid, view_weight=torch.as_tensor(vw, device=DEV))
    (vol * torch.as_tensor(delta, device=DEV)).sum().backward()
    th = oracle.akima_motion(x, cfg.views)
    Ph = oracle.compose(P, th)
    gP, _ = oracle.bp_vjp(Ph, proj.astype(np.float64), delta.astype(np.float64), cfg.spacing3,
                          cfg.origin, vw, oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid,
                          want_proj=False)
    want = oracle.akima_motion_vjp(x, cfg.views, oracle.chain_motion(P, th, gP))
    got = nodes.grad.cpu().numpy()
    for sl in (slice(0, 3), slice(3, 6)):
        assert np.linalg.norm(got[:, sl] - want[:, sl]) <= 1e-3 * np.linalg.norm(want[:, sl])
