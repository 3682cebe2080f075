"""Pins of the oracle's geometry (Eq. 1), chain rule (Eq. 2) and RPE
(Sec. IV-A) against closed forms and finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_09283_gb300 import workloads as W


def test_rigid_identity_and_orthonormal():
    assert np.array_equal(oracle.rigid(np.zeros(6)), np.eye(4))
    rng = np.random.default_rng(0)
    for _ in range(20):
        th = rng.uniform(-1, 1, 6)
        T = oracle.rigid(th)
        R = T[:3, :3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        assert np.array_equal(T[:3, 3], th[:3])
        assert np.array_equal(T[3], [0, 0, 0, 1])


def test_rigid_euler_order_single_axes():
    # R = Rz Ry Rx: a pure rz rotates x towards y (right-handed about z)
    a = 0.3
    T = oracle.rigid([0, 0, 0, 0, 0, a])
    assert np.allclose(T[:3, :3] @ [1, 0, 0], [math.cos(a), math.sin(a), 0], atol=1e-15)
    T = oracle.rigid([0, 0, 0, a, 0, 0])
    assert np.allclose(T[:3, :3] @ [0, 1, 0], [0, math.cos(a), math.sin(a)], atol=1e-15)
    T = oracle.rigid([0, 0, 0, 0, a, 0])
    assert np.allclose(T[:3, :3] @ [0, 0, 1], [math.sin(a), 0, math.cos(a)], atol=1e-15)
    # composition order: Rz(c) Ry(b) Rx(a) applied to e_x differs from Rx Ry Rz
    b, c = 0.4, 0.5
    Rx = oracle.rigid([0, 0, 0, a, 0, 0])[:3, :3]
    Ry = oracle.rigid([0, 0, 0, 0, b, 0])[:3, :3]
    Rz = oracle.rigid([0, 0, 0, 0, 0, c])[:3, :3]
    assert np.allclose(oracle.rigid([0, 0, 0, a, b, c])[:3, :3], Rz @ Ry @ Rx, atol=1e-15)


def test_rigid_grad_matches_central_fd():
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        th = rng.uniform(-0.5, 0.5, 6)
        dT = oracle.rigid_grad(th)
        for m in range(6):
            e = np.zeros(6)
            e[m] = h
            fd = (oracle.rigid(th + e) - oracle.rigid(th - e)) / (2 * h)
            assert np.allclose(dT[m], fd, atol=1e-9), m


def test_compose_identity_is_bitwise():
    P = W.projection_matrices(W.C1)
    assert np.array_equal(oracle.compose(P, None), P)
    assert np.array_equal(oracle.compose(P, np.zeros((P.shape[0], 6))), P)


def test_compose_is_matrix_product():
    P = W.projection_matrices(W.C1)
    th = W.motion_curves(W.C1)
    Ph = oracle.compose(P, th)
    for j in (0, 17, 59):
        ref = P[j] @ oracle.rigid(th[j])
        assert np.allclose(Ph[j], ref, rtol=0, atol=1e-12 * np.abs(P[j]).max())


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c4g"])
def test_nominal_geometry(name):
    cfg = W.CONFIGS[name]
    P = W.projection_matrices(cfg)
    cu, cv = (cfg.nu - 1) / 2, (cfg.nv - 1) / 2
    iso = P @ np.array([0, 0, 0, 1.0])
    assert np.allclose(iso[:, 0] / iso[:, 2], cu, atol=1e-9)
    assert np.allclose(iso[:, 1] / iso[:, 2], cv, atol=1e-9)
    assert np.allclose(iso[:, 2], cfg.sid, atol=1e-9)        # w = depth, mm
    assert np.allclose(np.linalg.norm(P[:, 2, :3], axis=1), 1.0, atol=1e-15)
    C = W.source_positions(P)
    Ch = np.concatenate([C, np.ones((cfg.views, 1))], axis=1)
    assert np.abs(np.einsum("vij,vj->vi", P, Ch)).max() < 1e-6
    assert np.allclose(np.linalg.norm(C[:, :2], axis=1), cfg.sid)
    assert np.allclose(C[:, 2], 0)
    # angular sampling: 200 degrees inclusive
    ang = np.unwrap(np.arctan2(C[:, 1], C[:, 0]))
    assert abs((ang[-1] - ang[0]) - math.radians(cfg.arc_deg)) < 1e-12


def test_chain_rule_against_fd_of_a_linear_functional():
    """dL/dtheta from orc_chain_motion equals FD of L(theta) = <G, P T(theta)>_F."""
    rng = np.random.default_rng(2)
    P = W.projection_matrices(W.C4_GRADCHECK)
    V = P.shape[0]
    th = rng.uniform(-0.1, 0.1, (V, 6))
    G = rng.standard_normal((V, 3, 4))
    g = oracle.chain_motion(P, th, G)
    h = 1e-6
    for j in (0, 5, 11):
        for m in range(6):
            tp, tm = th.copy(), th.copy()
            tp[j, m] += h
            tm[j, m] -= h
            fd = (np.sum(G * oracle.compose(P, tp)) - np.sum(G * oracle.compose(P, tm))) / (2 * h)
            assert abs(fd - g[j, m]) <= 1e-6 * max(1.0, abs(fd)), (j, m, fd, g[j, m])


def test_rpe_zero_and_tz_closed_form():
    cfg = W.C2
    P = W.projection_matrices(cfg)
    pts = W.rpe_points()
    assert pts.shape == (300, 3)
    assert np.allclose(np.sort(np.unique(np.round(np.linalg.norm(pts, axis=1), 9))), [25, 50, 100])
    assert oracle.rpe(P, P, pts, cfg.pitch, cfg.pitch) == 0.0
    s = 0.7
    th = np.zeros((cfg.views, 6))
    th[:, 2] = s
    Pm = oracle.compose(P, th)
    got = oracle.rpe(P, Pm, pts, cfg.pitch, cfg.pitch)
    # a tz shift moves every point's image along v by s*SDD/w mm on the detector
    ph = np.concatenate([pts, np.ones((300, 1))], axis=1)
    depth = np.einsum("vk,pk->vp", P[:, 2, :], ph)
    want = np.mean(s * cfg.sdd / depth)
    assert abs(got - want) < 1e-10 * want


def test_reprojection_error_of_the_package_equals_the_oracle():
    """metrics.reprojection_error (the RPE every reported number uses) against
    the oracle's RPE of Sec. IV-A on moved geometries of two configs."""
    from paper_2401_09283_gb300.metrics import reprojection_error
    pts = W.rpe_points()
    for cfg in (W.C2, W.PAPER):
        P = W.projection_matrices(cfg)
        Pm = oracle.compose(P, W.motion_curves(cfg))
        want = oracle.rpe(P, Pm, pts, cfg.pitch, cfg.pitch)
        got = reprojection_error(P, Pm, pts, cfg.pitch, cfg.pitch)
        assert want > 0.5
        assert abs(got - want) <= 1e-12 * want
        assert reprojection_error(Pm, Pm, pts, cfg.pitch, cfg.pitch) == 0.0
