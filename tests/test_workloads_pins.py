"""Pins of the seeded input generator: closed-form ellipsoid line integrals,
short-scan redundancy weights, the Shepp-Logan ramp, and "FDK of zero motion
reproduces the phantom" (the last one also pins the oracle's Eq. 3 in its FDK
weighting)."""
import math

import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle
from paper_2401_09283_gb300 import workloads as W


def _single(center, axes, rot=None, rho=1.0):
    rot = np.eye(3) if rot is None else rot
    return W.Phantom(np.array([center], float), np.array([axes], float), np.array([rot]),
                     np.array([rho]))


def _ray_P(src, direction):
    """A 3x4 matrix whose pixel (0,0) ray starts at src along direction."""
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    # build an orthonormal frame with d as the principal (third) axis
    a = np.cross(d, [0, 0, 1.0]) if abs(d[2]) < 0.9 else np.cross(d, [1.0, 0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(d, a)
    R = np.stack([a, b, d])
    return np.concatenate([R, (-R @ np.asarray(src, float))[:, None]], axis=1)[None]


def test_sphere_chord_through_centre():
    r = 7.5
    ph = _single([1.0, -2.0, 3.0], [r, r, r], rho=0.6)
    P = _ray_P([1.0 - 100, -2.0, 3.0], [1, 0, 0])
    li = W.line_integrals(ph, P, 1, 1)
    assert abs(float(li[0, 0, 0]) - 0.6 * 2 * r) < 1e-12


def test_line_integrals_match_ray_marching():
    rng = np.random.default_rng(3)
    Q = W._random_rotation(rng)
    ph = _single([2.0, 1.0, -1.0], [20.0, 12.0, 7.0], Q, rho=0.8)
    h = 2e-4
    for _ in range(6):
        src = rng.uniform(-80, 80, 3) + np.array([0, 0, 0])
        src = 100 * src / np.linalg.norm(src)
        target = rng.uniform(-3, 3, 3) + ph.centers[0]
        d = (target - src) / np.linalg.norm(target - src)
        li = float(W.line_integrals(ph, _ray_P(src, d), 1, 1)[0, 0, 0])
        t = np.arange(0.0, 200.0, h) + h / 2
        pts = src[None] + t[:, None] * d[None]
        num = W.phantom_density(ph, pts).sum() * h
        assert abs(li - num) <= 2 * h * 0.8 + 1e-9, (li, num)
        assert li > 0


def test_parker_conjugate_rays_sum_to_one():
    for cfg in (W.C1, W.C2, W.C4):
        w = W.parker_weights(cfg)
        beta = W.view_angles(cfg)
        gam = np.arctan((np.arange(cfg.nu) - (cfg.nu - 1) / 2) * cfg.pitch / cfg.sdd)
        P = W.projection_matrices(cfg)
        C = W.source_positions(P)
        checked = 0
        for j in range(0, cfg.views, 7):
            for a in range(0, cfg.nu, 5):
                g = gam[a]
                bc = beta[j] + math.pi - 2 * g
                if bc > beta[-1] or bc < beta[0]:
                    continue
                # geometric check that (bc, -g) is the conjugate ray: the
                # source at angle bc lies on the in-plane ray of (view j, column a)
                S2 = cfg.sid * np.array([math.cos(bc), math.sin(bc)])
                ray = np.linalg.inv(P[j][:, :3]) @ np.array([a, (cfg.nv - 1) / 2, 1.0])
                dd = ray[:2] / np.linalg.norm(ray[:2])
                rel = S2 - C[j, :2]
                assert abs(rel[0] * dd[1] - rel[1] * dd[0]) < 1e-6 * cfg.sid
                # and the conjugate ray's fan angle is -g: the ray seen from S2
                # makes angle -g with S2's central ray (towards the isocenter)
                back = -dd
                cen = -S2 / np.linalg.norm(S2)
                ang = math.atan2(cen[0] * back[1] - cen[1] * back[0], cen @ back)
                e_u2 = np.array([-math.sin(bc), math.cos(bc)])
                sgn = 1.0 if (back @ e_u2) > 0 else -1.0
                assert abs(sgn * abs(ang) - (-g)) < 1e-9
                wc = W.parker_weight(bc - beta[0], -g, math.radians(cfg.arc_deg))
                assert abs(w[j, a] + float(wc) - 1.0) < 1e-12, (j, a)
                checked += 1
        assert checked > 20
        # the weights vanish at both ends of the scan and are 1 mid-scan
        assert np.abs(w[0]).max() < 1e-12 and np.abs(w[-1]).max() < 1e-12
        assert np.allclose(w[cfg.views // 2], 1.0)


def test_shepp_logan_frequency_response():
    # The Shepp-Logan filter is the ramp |f| times sinc(f tau): with
    # omega = 2 pi f tau the DTFT of tau * h[n] is |sin(omega/2)| / (pi tau).
    # Checked at a few frequencies with a long kernel.
    tau = 0.5
    h = W.shepp_logan_kernel(200000, tau)
    n = np.arange(-200000, 200001)
    for om in (0.3, 1.0, 2.0, math.pi):
        H = tau * np.sum(h * np.cos(om * n))
        want = abs(math.sin(om / 2)) / (math.pi * tau)
        assert abs(H - want) < 1e-4 * want + 1e-5


def test_fdk_filter_is_linear_convolution():
    cfg = W.C4_GRADCHECK
    rng = np.random.default_rng(4)
    raw = torch.as_tensor(rng.standard_normal((2, cfg.nv, cfg.nu)))
    q = W.fdk_filter(raw, cfg, parker=False).numpy()
    tau = cfg.pitch * cfg.sid / cfg.sdd
    h = W.shepp_logan_kernel(cfg.nu - 1, tau)
    a = (np.arange(cfg.nu) - (cfg.nu - 1) / 2) * cfg.pitch
    b = (np.arange(cfg.nv) - (cfg.nv - 1) / 2) * cfg.pitch
    cosw = cfg.sdd / np.sqrt(cfg.sdd ** 2 + a[None] ** 2 + b[:, None] ** 2)
    p = raw.numpy() * cosw[None]
    for vi in range(2):
        for row in (0, 7, cfg.nv - 1):
            ref = np.array([tau * sum(h[cfg.nu - 1 + x - k] * p[vi, row, k] for k in range(cfg.nu))
                            for x in range(cfg.nu)])
            assert np.allclose(q[vi, row], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_fdk_zero_motion_reproduces_phantom():
    cfg = W.C1
    sc = W.make_scan(cfg, motion=False)
    vw = np.full(cfg.views, cfg.delta_beta)
    vol = oracle.bp_forward(sc.P, sc.proj.numpy(), cfg.vol_shape, cfg.spacing3, cfg.origin, vw,
                            oracle.WEIGHT_FDK, cfg.sid)
    ph2 = W.phantom_volume(sc.phantom, cfg, supersample=2)
    ph1 = W.phantom_volume(sc.phantom, cfg)
    z = (np.arange(cfg.n) - (cfg.n - 1) / 2) * cfg.spacing
    central = (np.abs(z) <= 0.25 * cfg.n * cfg.spacing)[:, None, None] & np.ones_like(vol, bool)
    fp = np.ones((7, 7, 7), bool)
    flat = (ndimage.maximum_filter(ph1, footprint=fp) - ndimage.minimum_filter(ph1, footprint=fp)) == 0
    m = flat & central
    assert m.sum() > 10000
    mae = np.abs(vol - ph2)[m].mean()
    rel = np.linalg.norm((vol - ph2)[central]) / np.linalg.norm(ph2[central])
    assert mae <= 0.02 * 1.0, mae
    assert rel <= 0.15, rel
    # the mean density over the central slab is preserved to 1 %
    assert abs(vol[central].mean() - ph2[central].mean()) < 0.01 * ph2[central].mean()


def test_phantom_densities_in_unit_range():
    for cfg in (W.C1, W.C2, W.C4):
        ph = W.head_phantom(cfg)
        assert len(ph.rho) == cfg.n_ellipsoids
        rng = np.random.default_rng(5)
        pts = rng.uniform(-1, 1, (20000, 3)) * ph.axes[0]
        d = W.phantom_density(ph, pts)
        assert d.min() >= -1e-12 and d.max() <= 1.0 + 1e-12


def test_motion_curves_zero_mean_and_amplitude():
    for cfg in (W.C1, W.C2):
        th = W.motion_curves(cfg)
        assert th.shape == (cfg.views, 6)
        assert np.allclose(th.mean(axis=0), 0, atol=1e-12)
        assert np.allclose(np.abs(th[:, :3]).max(axis=0), cfg.trans_mm)
        assert np.allclose(np.abs(th[:, 3:]).max(axis=0), math.radians(cfg.rot_deg))
