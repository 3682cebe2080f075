"""Seeded synthetic workloads: circular cone-beam geometries, ellipsoid head
phantoms, their closed-form line integrals, FDK pre-weighting and ramp
filtering, rigid motion curves and upstream gradients.

This module only produces INPUTS.  It holds none of the arithmetic of the
backprojection, its Jacobian, the motion composition, the loss or the
optimisers, so both the CUDA path and the CPU oracle can be fed from it.

The paper simulates its data from CQ500 head CT volumes with PyroNN (Sec. III);
that dataset is not available here, and closed-form line integrals of seeded
ellipsoid "head" phantoms stand in for it, on the paper's scanner geometry
(source-isocenter 750 mm and source-detector 1200 mm, short scans of 200
degrees as in Sec. IV-D, flat detectors, cosine and Shepp-Logan ramp filter as
in Sec. III).

Detector convention: integer detector coordinates are pixel centres,
(cu, cv) = ((nu-1)/2, (nv-1)/2) is the principal point, the u axis is
horizontal (in the plane of the trajectory, pointing along the source's
direction of travel) and the v axis points along world z.  Every projection
matrix has a unit-norm third row, so w is the depth in mm.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
import torch


# --------------------------------------------------------------------------- configs

@dataclasses.dataclass(frozen=True)
class ScanConfig:
    name: str
    n: int                 # volume edge in voxels (cubic volume)
    spacing: float         # voxel size, mm
    views: int
    arc_deg: float
    sid: float
    sdd: float
    nu: int
    nv: int
    pitch: float           # detector pixel size, mm (du = dv)
    n_ellipsoids: int
    phantom_seed: int
    noise: float           # relative Gaussian noise on line integrals (0 = none)
    knots: int             # spline knots of the true motion
    trans_mm: float        # +- translation amplitude
    rot_deg: float         # +- rotation amplitude
    motion_seed: int
    delta_seed: int

    @property
    def vol_shape(self):
        return (self.n, self.n, self.n)

    @property
    def voxels(self) -> int:
        return self.n ** 3

    @property
    def voxel_views(self) -> int:
        return self.n ** 3 * self.views

    @property
    def origin(self):
        o = -(self.n - 1) / 2.0 * self.spacing
        return (o, o, o)

    @property
    def spacing3(self):
        return (self.spacing,) * 3

    @property
    def delta_beta(self) -> float:
        arc = math.radians(self.arc_deg)
        if self.arc_deg >= 360.0:
            return arc / self.views
        return arc / (self.views - 1)


# Tiny plain-FP32 case (64^3, 60 views, 128x96 detector).
C1 = ScanConfig("c1-64^3x60v-128x96", 64, 1.0, 60, 200.0, 750.0, 1200.0, 128, 96, 1.6,
                10, 1, 0.0, 6, 3.0, 2.0, 1001, 2001)
# Head-size motion estimation (256^3, 248 views, 616x480 detector).
C2 = ScanConfig("c2-256^3x248v-616x480", 256, 1.0, 248, 200.0, 750.0, 1200.0, 616, 480, 0.616,
                30, 2, 0.01, 12, 5.0, 3.0, 1002, 2002)
# Precision form (512^3 at 0.5 mm, 496 views, 1240x960 detector).
C3 = ScanConfig("c3-512^3x496v-1240x960", 512, 0.5, 496, 200.0, 750.0, 1200.0, 1240, 960, 0.308,
                60, 3, 0.0, 6, 3.0, 2.0, 1003, 2003)
# Differentiation form (192^3, 180 views, 320x240 detector).
C4 = ScanConfig("c4-192^3x180v-320x240", 192, 1.33, 180, 200.0, 750.0, 1200.0, 320, 240, 1.30,
                10, 4, 0.0, 6, 3.0, 2.0, 1004, 2004)
# Gradcheck instance of the differentiation form (16^3, 12 views, 32x24).
C4_GRADCHECK = ScanConfig("c4g-16^3x12v-32x24", 16, 4.0, 12, 200.0, 750.0, 1200.0, 32, 24, 6.4,
                          4, 40, 0.0, 6, 3.0, 2.0, 1040, 2040)

# The paper's own motion-estimation setup (Sec. III-IV): 128^3 at 2 mm, 360
# views over the full circle, SID 785 mm, SDD 1200 mm, 500 x 700 detector
# (rows x columns) at 0.64 mm, motion of 10-node splines at 5 mm / 5 deg.
PAPER = ScanConfig("paper-128^3x360v-700x500", 128, 2.0, 360, 360.0, 785.0, 1200.0, 700, 500,
                   0.64, 30, 6, 0.01, 10, 5.0, 5.0, 1006, 2006)

CONFIGS = {"c1": C1, "c2": C2, "c3": C3, "c4": C4, "c4g": C4_GRADCHECK, "paper": PAPER}


def serving_job_config(job_id: int, n: int, views: int) -> ScanConfig:
    """One job of the serving stream: 256 mm field of view at n voxels, a
    detector whose pitch keeps 0.6-1.6 mm pixels and covers 414 mm."""
    vox = 256.0 / n
    pitch = min(max(0.8 * vox * 1.6, 0.6), 1.6)
    nu = int(math.ceil(414.0 / pitch))
    nu = (nu + 7) // 8 * 8
    nv = int(math.ceil(0.75 * nu))
    return ScanConfig("job%d-%d^3x%dv-%dx%d" % (job_id, n, views, nu, nv), n, vox, views, 200.0,
                      750.0, 1200.0, nu, nv, pitch, 30, 5000 + job_id, 0.01, 12, 5.0, 3.0,
                      6000 + job_id, 7000 + job_id)


# ------------------------------------------------------------------------- geometry

def view_angles(cfg: ScanConfig) -> np.ndarray:
    """Source angles beta_j (rad): -arc/2 .. +arc/2 inclusive for short scans,
    evenly over the circle for full scans."""
    arc = math.radians(cfg.arc_deg)
    if cfg.arc_deg >= 360.0:
        return np.arange(cfg.views) * (arc / cfg.views)
    return -arc / 2.0 + np.arange(cfg.views) * cfg.delta_beta


def projection_matrices(cfg: ScanConfig) -> np.ndarray:
    """Calibrated 3x4 matrices of the circular trajectory about world z,
    P_j = K [R_j | -R_j S_j]; shape (V,3,4), float64."""
    cu, cv = (cfg.nu - 1) / 2.0, (cfg.nv - 1) / 2.0
    K = np.array([[cfg.sdd / cfg.pitch, 0.0, cu], [0.0, cfg.sdd / cfg.pitch, cv], [0.0, 0.0, 1.0]])
    out = np.zeros((cfg.views, 3, 4))
    for j, b in enumerate(view_angles(cfg)):
        S = cfg.sid * np.array([math.cos(b), math.sin(b), 0.0])
        e_u = np.array([-math.sin(b), math.cos(b), 0.0])
        e_v = np.array([0.0, 0.0, 1.0])
        e_w = -np.array([math.cos(b), math.sin(b), 0.0])
        R = np.stack([e_u, e_v, e_w])
        out[j] = K @ np.concatenate([R, (-R @ S)[:, None]], axis=1)
    return out


def source_positions(P: np.ndarray) -> np.ndarray:
    """Right null vector of each 3x4 matrix, dehomogenised: C = -M^-1 p4."""
    M = P[:, :, :3]
    p4 = P[:, :, 3]
    return -np.linalg.solve(M, p4[..., None])[..., 0]


# -------------------------------------------------------------------------- phantom

@dataclasses.dataclass
class Phantom:
    centers: np.ndarray   # (E,3) mm
    axes: np.ndarray      # (E,3) semi-axes mm
    rot: np.ndarray       # (E,3,3) columns = ellipsoid axes in world
    rho: np.ndarray       # (E,) additive density


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def head_phantom(cfg: ScanConfig) -> Phantom:
    """Seeded ellipsoid head: skull (rho 1.0), brain (rho -0.8, axes x0.9) and
    n_ellipsoids-2 non-overlapping inner ellipsoids (axes 3-25 % of R,
    rho in [-0.1, 0.3]) so that densities stay in [0, 1]."""
    rng = np.random.default_rng(cfg.phantom_seed)
    R = 0.45 * cfg.n * cfg.spacing
    # keep the skull inside the field of view of the detector
    fov = cfg.sid * math.sin(math.atan(cfg.nu * cfg.pitch / 2.0 / cfg.sdd))
    R = min(R, 0.88 * fov / 0.9)
    skull = np.array([0.70, 0.90, 0.80]) * R
    brain = 0.9 * skull
    centers = [np.zeros(3), np.zeros(3)]
    axes = [skull, brain]
    rots = [np.eye(3), np.eye(3)]
    rho = [1.0, -0.8]
    bounds = []  # (centre, bounding radius) of inner ellipsoids
    tries = 0
    while len(centers) < cfg.n_ellipsoids:
        tries += 1
        if tries > 100000:
            raise RuntimeError("phantom sampling did not converge")
        a = rng.uniform(0.03, 0.25, size=3) * R
        rmax = a.max()
        c = rng.uniform(-1, 1, size=3) * brain
        if np.sum((c / np.maximum(brain - rmax, 1e-9)) ** 2) >= 1.0 or np.any(brain - rmax <= 0):
            continue
        if any(np.linalg.norm(c - c2) < rmax + r2 for c2, r2 in bounds):
            continue
        r = rng.uniform(-0.1, 0.3)
        bounds.append((c, rmax))
        centers.append(c)
        axes.append(a)
        rots.append(_random_rotation(rng))
        rho.append(r)
    return Phantom(np.array(centers), np.array(axes), np.array(rots), np.array(rho))


def phantom_density(ph: Phantom, pts: np.ndarray) -> np.ndarray:
    """Density at world points pts (...,3)."""
    out = np.zeros(pts.shape[:-1])
    for c, a, Q, r in zip(ph.centers, ph.axes, ph.rot, ph.rho):
        local = (pts - c) @ Q / a
        out += r * (np.sum(local * local, axis=-1) <= 1.0)
    return out


def phantom_volume(ph: Phantom, cfg: ScanConfig, supersample: int = 1) -> np.ndarray:
    """Phantom sampled on the reconstruction grid, (nz,ny,nx), averaging
    supersample^3 sub-voxel points per voxel."""
    n, s = cfg.n, cfg.spacing
    o = cfg.origin[0]
    sub = (np.arange(supersample) + 0.5) / supersample - 0.5
    coords = o + (np.arange(n)[:, None] + sub[None, :]).reshape(-1) * s
    acc = np.zeros((n * supersample,) * 3)
    for zi, z in enumerate(coords):
        Y, X = np.meshgrid(coords, coords, indexing="ij")
        pts = np.stack([X, Y, np.full_like(X, z)], axis=-1)
        acc[zi] = phantom_density(ph, pts)
    if supersample > 1:
        acc = acc.reshape(n, supersample, n, supersample, n, supersample).mean(axis=(1, 3, 5))
    return acc


# ---------------------------------------------------------------- line integrals

def line_integrals(ph: Phantom, P: np.ndarray, nu: int, nv: int, device="cpu",
                   dtype=torch.float64, views_per_chunk: int = 8) -> torch.Tensor:
    """Closed-form line integrals sum_e rho_e * chord_e for every pixel of
    every view of the (possibly moved) matrices P (V,3,4).  The ray of pixel
    (u,v) runs from the source C = -M^-1 p4 along M^-1 (u,v,1)."""
    V = P.shape[0]
    Minv = torch.as_tensor(np.linalg.inv(P[:, :, :3]), dtype=torch.float64)
    C = torch.as_tensor(source_positions(P), dtype=torch.float64)
    A = np.einsum("eij,ej->eji", ph.rot, 1.0 / ph.axes)  # A_e = diag(1/a) Q^T
    A = torch.as_tensor(A, dtype=dtype, device=device)
    ctr = torch.as_tensor(ph.centers, dtype=dtype, device=device)
    rho = torch.as_tensor(ph.rho, dtype=dtype, device=device)
    vv, uu = torch.meshgrid(torch.arange(nv, dtype=torch.float64),
                            torch.arange(nu, dtype=torch.float64), indexing="ij")
    pix = torch.stack([uu, vv, torch.ones_like(uu)], dim=-1).reshape(-1, 3)
    out = torch.empty((V, nv, nu), dtype=dtype, device=device)
    for j0 in range(0, V, views_per_chunk):
        j1 = min(V, j0 + views_per_chunk)
        d = torch.einsum("vij,rj->vri", Minv[j0:j1], pix)          # (b,R,3)
        d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
        d = d.to(device=device, dtype=dtype)
        o = C[j0:j1].to(device=device, dtype=dtype)                  # (b,3)
        acc = torch.zeros(d.shape[:2], dtype=dtype, device=device)
        for e in range(A.shape[0]):
            oe = (o - ctr[e]) @ A[e].T                               # (b,3)
            de = d @ A[e].T                                          # (b,R,3)
            qa = (de * de).sum(-1)
            qb = (de * oe[:, None, :]).sum(-1)
            qc = (oe * oe).sum(-1)[:, None] - 1.0
            disc = qb * qb - qa * qc
            acc += rho[e] * 2.0 * torch.sqrt(torch.clamp(disc, min=0.0)) / qa
        out[j0:j1] = acc.reshape(j1 - j0, nv, nu)
    return out


def add_noise(raw: torch.Tensor, rel: float, seed: int) -> torch.Tensor:
    """Additive N(0, sigma^2), sigma = rel * mean of the positive line integrals."""
    if rel <= 0:
        return raw
    pos = raw[raw > 0]
    sigma = rel * float(pos.mean()) if pos.numel() else 0.0
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(tuple(raw.shape)).astype(np.float64) * sigma
    return raw + torch.as_tensor(noise, dtype=raw.dtype, device=raw.device)


# ------------------------------------------------------------------- filtering

def parker_weight(beta_rel, gamma, arc: float):
    """Short-scan redundancy weight w(beta, gamma) for a scan arc pi + 2*delta
    (beta measured from the scan start, gamma the fan angle, positive along
    the detector u axis).  Conjugate rays (beta, gamma) and
    (beta + pi - 2 gamma, -gamma) sum to 1 (Parker's weights generalised to
    over-scan by using delta in place of the maximum fan angle)."""
    B = np.asarray(beta_rel, dtype=np.float64)
    G = np.asarray(gamma, dtype=np.float64)
    delta = (arc - math.pi) / 2.0
    if np.abs(G).max() >= delta:
        raise ValueError("scan arc too short for the fan angle")
    r1 = B < 2 * delta + 2 * G
    r3 = B > math.pi + 2 * G
    with np.errstate(divide="ignore", invalid="ignore"):
        w1 = np.sin(math.pi / 4 * B / (delta + G)) ** 2
        w3 = np.sin(math.pi / 4 * (math.pi + 2 * delta - B) / (delta - G)) ** 2
    w = np.where(r1, w1, np.where(r3, w3, 1.0))
    return np.clip(w, 0.0, 1.0)


def parker_weights(cfg: ScanConfig) -> np.ndarray:
    """Table of parker_weight over (view, detector column), (V, nu); full
    scans get 1/2 everywhere."""
    if cfg.arc_deg >= 360.0:
        return np.full((cfg.views, cfg.nu), 0.5)
    beta = view_angles(cfg) - view_angles(cfg)[0]
    a = (np.arange(cfg.nu) - (cfg.nu - 1) / 2.0) * cfg.pitch
    gamma = np.arctan(a / cfg.sdd)
    return parker_weight(beta[:, None], gamma[None, :], math.radians(cfg.arc_deg))


def shepp_logan_kernel(n_half: int, tau: float) -> np.ndarray:
    """Discrete Shepp-Logan ramp h[n] = -2 / (pi^2 tau^2 (4 n^2 - 1)),
    n = -n_half..n_half (Kak & Slaney)."""
    n = np.arange(-n_half, n_half + 1, dtype=np.float64)
    return -2.0 / (math.pi ** 2 * tau ** 2 * (4.0 * n * n - 1.0))


def fdk_filter(raw: torch.Tensor, cfg: ScanConfig, views: Optional[Sequence[int]] = None,
               parker: bool = True, ext: int = 0) -> torch.Tensor:
    """Cosine weight SDD/sqrt(SDD^2+a^2+b^2), short-scan weights of the rows
    `views` of the scan (all by default), optionally (ext > 0) the rows
    extended by ext pixels per side falling linearly to 0, then the Shepp-Logan ramp along u
    on the detector scaled to the isocenter (tau = pitch*SID/SDD):
    q = tau * (h * p), a linear convolution done by a zero-padded FFT.
    raw (V,nv,nu) -> filtered, same dtype/device."""
    V, nv, nu = raw.shape
    dev, dt = raw.device, raw.dtype
    a = (torch.arange(nu, dtype=torch.float64) - (nu - 1) / 2.0) * cfg.pitch
    b = (torch.arange(nv, dtype=torch.float64) - (nv - 1) / 2.0) * cfg.pitch
    cosw = cfg.sdd / torch.sqrt(cfg.sdd ** 2 + a[None, :] ** 2 + b[:, None] ** 2)
    p = raw * cosw.to(dev, dt)[None]
    if parker:
        rows = parker_weights(cfg)
        rows = rows if views is None else rows[np.asarray(views)]
        p = p * torch.as_tensor(rows, dtype=dt, device=dev)[:, None, :]
    tau = cfg.pitch * cfg.sid / cfg.sdd
    if ext > 0:  # truncation correction: rows extended by linear fall-off to 0
        ramp = 1.0 - torch.arange(1, ext + 1, dtype=p.dtype, device=dev) / ext
        left = p[..., :1] * ramp.flip(0)[None, None, :]
        right = p[..., -1:] * ramp[None, None, :]
        p = torch.cat([left, p, right], dim=-1)
    n = nu + 2 * ext
    L = 1 << int(math.ceil(math.log2(2 * n)))
    h = shepp_logan_kernel(n - 1, tau)
    hk = np.zeros(L)
    hk[: n] = h[n - 1:]                   # m = 0 .. n-1
    hk[L - (n - 1):] = h[: n - 1]         # m = -(n-1) .. -1
    H = torch.fft.rfft(torch.as_tensor(hk, dtype=torch.float64, device=dev))
    out = torch.empty((V, nv, nu), dtype=dt, device=dev)
    for j0 in range(0, V, 16):
        blk = p[j0:j0 + 16].to(torch.float64)
        F = torch.fft.rfft(blk, n=L, dim=-1)
        q = torch.fft.irfft(F * H, n=L, dim=-1)[..., ext:ext + nu] * tau
        out[j0:j0 + 16] = q.to(dt)
    return out


# --------------------------------------------------------------------- motion

def _akima(xk: np.ndarray, yk: np.ndarray, x: np.ndarray) -> np.ndarray:
    from scipy.interpolate import Akima1DInterpolator
    return Akima1DInterpolator(xk, yk)(x)


def motion_curves(cfg: ScanConfig) -> np.ndarray:
    """True per-view motion theta* (V,6) = (tx,ty,tz [mm], rx,ry,rz [rad]):
    one Akima spline per parameter through `knots` evenly spaced knots
    (first and last at the scan ends) with values uniform in [-A, A], made
    zero-mean over the views and rescaled to max |.| = A."""
    rng = np.random.default_rng(cfg.motion_seed)
    t = np.linspace(0.0, 1.0, cfg.views)
    tk = np.linspace(0.0, 1.0, cfg.knots)
    amps = [cfg.trans_mm] * 3 + [math.radians(cfg.rot_deg)] * 3
    out = np.zeros((cfg.views, 6))
    for m, A in enumerate(amps):
        yk = rng.uniform(-A, A, size=cfg.knots)
        c = _akima(tk, yk, t)
        c = c - c.mean()
        mx = np.abs(c).max()
        out[:, m] = c * (A / mx) if mx > 0 else c
    return out


def upstream_gradient(cfg: ScanConfig, dtype=np.float32) -> np.ndarray:
    """Seeded N(0,1) upstream gradient dL/dvol, (nz,ny,nx)."""
    rng = np.random.default_rng(cfg.delta_seed)
    return rng.standard_normal(cfg.vol_shape, dtype=np.float32).astype(dtype)


def rpe_points() -> np.ndarray:
    """300 points: 100 on each sphere of radius 25, 50 and 100 mm about the
    isocenter, on a Fibonacci lattice (Sec. IV-A uses 300 points at three
    radii; their layout is not given)."""
    pts = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for r in (25.0, 50.0, 100.0):
        for i in range(100):
            z = 1.0 - 2.0 * (i + 0.5) / 100.0
            rad = math.sqrt(max(0.0, 1.0 - z * z))
            phi = i * golden
            pts.append([r * rad * math.cos(phi), r * rad * math.sin(phi), r * z])
    return np.array(pts)


# ------------------------------------------------------------------ assembled

@dataclasses.dataclass
class Scan:
    cfg: ScanConfig
    P: np.ndarray            # (V,3,4) calibrated (nominal) matrices
    theta_true: np.ndarray   # (V,6) motion that the data was simulated with
    proj: torch.Tensor       # (V,nv,nu) filtered projections
    phantom: Phantom


def make_scan(cfg: ScanConfig, moved_P: Optional[np.ndarray] = None, *, motion: bool = True,
              device="cpu", dtype=torch.float64, views: Optional[Sequence[int]] = None) -> Scan:
    """Simulate a scan: phantom -> line integrals through the moved geometry
    -> noise -> cosine/short-scan/ramp filtering.

    moved_P: the matrices P_j T(theta*_j) the data is simulated with.  The
    caller composes them (this module holds no motion arithmetic); with
    motion=False the nominal matrices are used and theta* = 0.
    views: optional subset of view indices to simulate (filtered the same way
    as in the full scan)."""
    P = projection_matrices(cfg)
    th = motion_curves(cfg) if motion else np.zeros((cfg.views, 6))
    Pm = P if (moved_P is None or not motion) else moved_P
    if motion and moved_P is None:
        raise ValueError("moved_P is required when motion=True")
    ph = head_phantom(cfg)
    sel = np.arange(cfg.views) if views is None else np.asarray(views)
    raw = line_integrals(ph, Pm[sel], cfg.nu, cfg.nv, device=device, dtype=dtype)
    if cfg.noise > 0:
        raw = add_noise(raw, cfg.noise, cfg.phantom_seed + 100)
    q = fdk_filter(raw, cfg, views=sel)
    return Scan(cfg, P, th, q, ph)
