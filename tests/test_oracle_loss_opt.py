"""Pins of the oracle's sharpness loss and its gradient, the gradient-descent
update of Eq. 6 and the Adam update (closed forms and finite differences)."""
import numpy as np
import pytest

import oracle


def test_sharpness_closed_forms():
    nz, ny, nx = 5, 6, 7
    K = nx * ny * nz
    const = np.full((nz, ny, nx), 3.7)
    L, g = oracle.sharpness(const)
    assert L == 0.0 and np.all(g == 0.0)
    a = 0.3
    ramp = a * np.arange(nx)[None, None, :] * np.ones((nz, ny, nx))
    L, g = oracle.sharpness(ramp)
    assert L == pytest.approx(-(a * a) * (nx - 1) * ny * nz / K, rel=1e-14)
    # dL/dI for a ramp along x: only the two end planes see a net gradient
    want = np.zeros((nz, ny, nx))
    want[:, :, 0] = 2 * a / K
    want[:, :, -1] = -2 * a / K
    assert np.allclose(g, want, atol=1e-15)


def test_sharpness_gradient_fd_and_sum():
    rng = np.random.default_rng(0)
    vol = rng.standard_normal((8, 8, 8))
    L, g = oracle.sharpness(vol)
    assert abs(g.sum()) < 1e-14
    h = 1e-6
    for idx in [(0, 0, 0), (3, 4, 5), (7, 7, 7), (0, 7, 3), (4, 0, 7)]:
        vp, vm = vol.copy(), vol.copy()
        vp[idx] += h
        vm[idx] -= h
        fd = (oracle.sharpness(vp, want_grad=False)[0] - oracle.sharpness(vm, want_grad=False)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8


def test_gd_step_eq6():
    rng = np.random.default_rng(1)
    th = rng.standard_normal((10, 6))
    gr = rng.standard_normal((10, 6))
    s0, t, n = 100.0, 0.97, 7
    out = oracle.gd_step(th, gr, s0, t, n, gauge=False)
    assert np.allclose(out, th - s0 * t ** n * gr, rtol=1e-15, atol=1e-13)
    out = oracle.gd_step(th, gr, s0, t, n, gauge=True)
    raw = th - s0 * t ** n * gr
    assert np.allclose(out, raw - raw.mean(axis=0), atol=1e-12)
    assert np.allclose(out.mean(axis=0), 0, atol=1e-12)


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(2)
    th = rng.standard_normal((4, 6))
    g1 = rng.standard_normal((4, 6))
    lr = 0.01
    z = np.zeros_like(th)
    t1, m1, m2 = oracle.adam_step(th, g1, z, z, lr, 1, gauge=False)
    # first step: m_hat = g, v_hat = g^2 -> a step of lr * g / (|g| + eps)
    assert np.allclose(t1, th - lr * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g1) and np.allclose(m2, 0.001 * g1 * g1)
    g2 = rng.standard_normal((4, 6))
    t2, _, _ = oracle.adam_step(t1, g2, m1, m2, lr, 2, gauge=False)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.9 ** 2)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(t2, t1 - lr * mh / (np.sqrt(vh) + 1e-8), atol=1e-14)


def test_tv_closed_forms():
    nz, ny, nx = 5, 6, 7
    K = nx * ny * nz
    n_int = (nx - 1) * (ny - 1) * (nz - 1)
    eps = 1e-2
    L, g = oracle.tv(np.full((nz, ny, nx), 2.5), eps)
    assert L == pytest.approx(n_int * eps / K, rel=1e-14)
    assert np.all(g == 0.0)
    a = 0.3
    ramp = a * np.arange(nx)[None, None, :] * np.ones((nz, ny, nx))
    L, g = oracle.tv(ramp, eps)
    assert L == pytest.approx(n_int * np.sqrt(a * a + eps * eps) / K, rel=1e-14)
    assert abs(g.sum()) < 1e-14


def test_tv_gradient_fd():
    rng = np.random.default_rng(3)
    vol = rng.standard_normal((8, 8, 8))
    eps = 0.05
    L, g = oracle.tv(vol, eps)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 4, 5), (7, 7, 7), (0, 7, 3), (4, 0, 7), (7, 3, 0)]:
        vp, vm = vol.copy(), vol.copy()
        vp[idx] += h
        vm[idx] -= h
        fd = (oracle.tv(vp, eps, False)[0] - oracle.tv(vm, eps, False)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8
