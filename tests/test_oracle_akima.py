"""Pins of the oracle's Akima spline motion model (Sec. II-B.1): the spline
against scipy's Akima interpolator (an independent library implementation
of Akima's construction), exactness on lines, interpolation of the nodes,
the forward-mode Jacobian against central finite differences, and the
motion-model VJP against finite differences of <g, theta(nodes)>."""
import numpy as np
import pytest

import oracle

scipy_interp = pytest.importorskip("scipy.interpolate")


def test_matches_scipy_akima_on_uneven_knots():
    rng = np.random.default_rng(0)
    for n in (3, 4, 7, 12, 30):
        x = np.cumsum(rng.uniform(0.3, 2.0, n))
        y = rng.standard_normal(n)
        xe = np.linspace(x[0], x[-1], 257)
        ref = scipy_interp.Akima1DInterpolator(x, y)(xe)
        assert np.max(np.abs(oracle.akima_eval(y, xe, x) - ref)) < 1e-12


def test_flat_stretch_uses_the_mean_of_the_two_secants():
    # equal consecutive secants on both sides make the weight denominator 0
    x = np.arange(8.0)
    y = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 2.0, 3.0, 3.5])
    xe = np.linspace(0, 7, 141)
    ref = scipy_interp.Akima1DInterpolator(x, y)(xe)
    assert np.max(np.abs(oracle.akima_eval(y, xe, x) - ref)) < 1e-12


def test_lines_are_reproduced_and_nodes_interpolated():
    x = np.linspace(0, 247, 12)
    y = 0.7 - 0.013 * x
    xe = np.arange(248.0)
    assert np.max(np.abs(oracle.akima_eval(y, xe, x) - (0.7 - 0.013 * xe))) < 1e-12
    rng = np.random.default_rng(1)
    y = rng.standard_normal(12)
    assert np.max(np.abs(oracle.akima_eval(y, x, x) - y)) < 1e-12


def test_jacobian_against_central_differences():
    rng = np.random.default_rng(2)
    n = 9
    x = np.linspace(0, 100, n)
    y = rng.standard_normal(n)
    xe = np.linspace(0, 100, 61)
    J = oracle.akima_jacobian(y, xe, x)
    h = 1e-6
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fd = (oracle.akima_eval(y + e, xe, x) - oracle.akima_eval(y - e, xe, x)) / (2 * h)
        assert np.max(np.abs(fd - J[:, k])) < 1e-7
    # Akima's weights scale with y, so the spline is homogeneous of degree 1
    # in y and Euler's identity J y = spline(y) holds
    assert np.max(np.abs(J @ y - oracle.akima_eval(y, xe, x))) < 1e-12


def test_motion_model_and_its_vjp():
    rng = np.random.default_rng(3)
    V, nn = 60, 7
    nodes = rng.standard_normal((nn, 6)) * np.array([3, 3, 3, 0.03, 0.03, 0.03])
    th = oracle.akima_motion(nodes, V)
    assert th.shape == (V, 6)
    # with 61 views and 7 nodes every 10th view sits on a knot
    V2 = 61
    th2 = oracle.akima_motion(nodes, V2)
    assert np.max(np.abs(th2[::10] - nodes)) < 1e-12
    g = rng.standard_normal((V, 6))
    vjp = oracle.akima_motion_vjp(nodes, V, g)
    h = 1e-6
    for _ in range(5):
        d = rng.standard_normal((nn, 6))
        fd = (np.sum(g * oracle.akima_motion(nodes + h * d, V))
              - np.sum(g * oracle.akima_motion(nodes - h * d, V))) / (2 * h)
        assert abs(fd - np.sum(vjp * d)) < 1e-6 * (1 + abs(fd))
