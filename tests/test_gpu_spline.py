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
