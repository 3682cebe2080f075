"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the
same seeded inputs.

Tolerances: volumes rel-L2 <= 1e-5 for FP32 data; motion gradients rel-L2
<= 1e-3 per parameter group (translations, rotations); FP16-stored data
rel-L2 <= 2e-3 against the oracle on the FP32 data; BF16 <= 2^-9, its unit
roundoff (derivation beside BF16_STORAGE_TOL in cases.py).
"""
import numpy as np
import pytest
import torch

import oracle
from cases import (BF16_STORAGE_TOL, FP16_STORAGE_TOL, motion_errors, per_view_worst, rel_l2,
                   random_case, scan_case)
from paper_2401_09283_gb300 import bp
from paper_2401_09283_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")
VOL_TOL = 1e-5
GRAD_TOL = 1e-3


def cuda(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def gpu_forward(proj, P, th, vol_shape, spacing, origin, vw=None, weight="fdk", sid=750.0,
                view_scale=None, dtype=torch.float32):
    p = cuda(proj).to(dtype)
    out = bp.bp_forward(p, cuda(P), None if th is None else cuda(th), vol_shape=vol_shape,
                        spacing=spacing, origin=origin,
                        view_weight=None if vw is None else cuda(vw), weight=weight, sid=sid,
                        view_scale=None if view_scale is None else cuda(view_scale))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def gpu_vjp(delta, proj, P, th, spacing, origin, vw=None, weight="fdk", deriv="central",
            sid=750.0, want=(True, True, True), dtype=torch.float32, view_scale=None):
    gm, gP, gD = bp.bp_vjp(cuda(delta), cuda(proj).to(dtype), cuda(P),
                           None if th is None else cuda(th), spacing=spacing, origin=origin,
                           view_weight=None if vw is None else cuda(vw), weight=weight,
                           deriv=deriv, sid=sid,
                           view_scale=None if view_scale is None else cuda(view_scale),
                           want_motion=want[0], want_Phat=want[1], want_proj=want[2])
    torch.cuda.synchronize()
    f = lambda x: None if x is None else x.cpu().numpy()
    return f(gm), f(gP), f(gD)


def motion_rel(g, o):
    return max(rel_l2(g[:, :3], o[:, :3]), rel_l2(g[:, 3:], o[:, 3:]))


# ----------------------------------------------------------------- config 1

@pytest.mark.parametrize("weight", ["fdk", "none"])
def test_c1_forward(weight):
    cfg, P, th, proj, _ = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    mode = oracle.WEIGHT_FDK if weight == "fdk" else oracle.WEIGHT_NONE
    ref = oracle.bp_forward(oracle.compose(P, th), proj.astype(np.float64), cfg.vol_shape,
                            cfg.spacing3, cfg.origin, vw, mode, cfg.sid)
    got = gpu_forward(proj, P, th, cfg.vol_shape, cfg.spacing3, cfg.origin, vw, weight, cfg.sid)
    assert rel_l2(got, ref) <= VOL_TOL


@pytest.mark.parametrize("weight", ["fdk", "none"])
@pytest.mark.parametrize("deriv", ["central", "exact"])
def test_c1_vjp(weight, deriv):
    cfg, P, th, proj, delta = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    mode = oracle.WEIGHT_FDK if weight == "fdk" else oracle.WEIGHT_NONE
    dmode = oracle.DERIV_CENTRAL if deriv == "central" else oracle.DERIV_BILINEAR_EXACT
    Ph = oracle.compose(P, th)
    oP, oD = oracle.bp_vjp(Ph, proj.astype(np.float64), delta.astype(np.float64), cfg.spacing3,
                           cfg.origin, vw, mode, dmode, cfg.sid)
    om = oracle.chain_motion(P, th, oP)
    # all three products: the data VJP runs fused into the motion-VJP kernel
    gm, gP, gD = gpu_vjp(delta, proj, P, th, cfg.spacing3, cfg.origin, vw, weight, deriv, cfg.sid)
    errs = motion_errors(gm, om)
    print("c1 %s %s motion gradient: rel-L2 %.3g / %.3g, worst view %.3g" % ((weight, deriv) + errs))
    assert max(errs[:2]) <= GRAD_TOL
    # The exact derivative of the bilinear interpolant jumps where a sample
    # crosses a pixel boundary; a sample within FP32 rounding (~1e-6 px) of a
    # boundary may take the other side's derivative than the FP64 oracle.
    # Summed over a view's voxels such jumps leave per-view errors of ~1e-2
    # on c1 (group rel-L2 ~1e-4); the paper's CENTRAL derivative is
    # continuous in the sample position and meets the bar per view.
    if deriv == "central":
        assert errs[2] <= GRAD_TOL
    assert rel_l2(gP, oP) <= GRAD_TOL
    assert rel_l2(gD, oD) <= VOL_TOL
    # each product alone: the unfused kernels
    gm2, _, _ = gpu_vjp(delta, proj, P, th, cfg.spacing3, cfg.origin, vw, weight, deriv, cfg.sid,
                        want=(True, False, False))
    # the motion-only kernel sums even and odd voxels of a column separately
    # (packed pairs), the fused one in sequence: same terms, other order
    assert motion_rel(gm2, gm) <= 1e-6
    _, _, gD2 = gpu_vjp(delta, proj, P, th, cfg.spacing3, cfg.origin, vw, weight, deriv, cfg.sid,
                        want=(False, False, True))
    assert rel_l2(gD2, oD) <= VOL_TOL


def test_c1_identity_motion_is_plain_backprojection():
    cfg, P, _, proj, _ = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    a = gpu_forward(proj, P, None, cfg.vol_shape, cfg.spacing3, cfg.origin, vw)
    b = gpu_forward(proj, P, np.zeros((cfg.views, 6)), cfg.vol_shape, cfg.spacing3, cfg.origin, vw)
    assert np.array_equal(a, b)
    ref = oracle.bp_forward(P, proj.astype(np.float64), cfg.vol_shape, cfg.spacing3, cfg.origin,
                            vw, oracle.WEIGHT_FDK, cfg.sid)
    assert rel_l2(a, ref) <= VOL_TOL


def test_deterministic():
    cfg, P, th, proj, delta = scan_case("c1")
    a = gpu_forward(proj, P, th, cfg.vol_shape, cfg.spacing3, cfg.origin)
    b = gpu_forward(proj, P, th, cfg.vol_shape, cfg.spacing3, cfg.origin)
    assert np.array_equal(a, b)
    g1 = gpu_vjp(delta, proj, P, th, cfg.spacing3, cfg.origin, want=(True, True, False))
    g2 = gpu_vjp(delta, proj, P, th, cfg.spacing3, cfg.origin, want=(True, True, False))
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])


# ------------------------------------------------------- ragged and edge cases

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ragged_random(seed):
    cfg, P, th, proj, delta, origin = random_case(seed)
    sp = (cfg.spacing,) * 3
    Ph = oracle.compose(P, th)
    for weight, mode in (("fdk", oracle.WEIGHT_FDK), ("none", oracle.WEIGHT_NONE)):
        ref = oracle.bp_forward(Ph, proj.astype(np.float64), delta.shape, sp, origin, None, mode,
                                cfg.sid)
        got = gpu_forward(proj, P, th, delta.shape, sp, origin, None, weight, cfg.sid)
        assert rel_l2(got, ref) <= VOL_TOL
        for deriv, dm in (("central", oracle.DERIV_CENTRAL), ("exact", oracle.DERIV_BILINEAR_EXACT)):
            oP, oD = oracle.bp_vjp(Ph, proj.astype(np.float64), delta.astype(np.float64), sp,
                                   origin, None, mode, dm, cfg.sid)
            om = oracle.chain_motion(P, th, oP)
            gm, gP, gD = gpu_vjp(delta, proj, P, th, sp, origin, None, weight, deriv, cfg.sid)
            assert motion_rel(gm, om) <= GRAD_TOL
            assert rel_l2(gP, oP) <= GRAD_TOL
            assert rel_l2(gD, oD) <= VOL_TOL


def test_volume_larger_than_detector_field():
    """Voxels projecting off the detector, across its edges and (for a huge
    volume) behind the source plane: EDGE and SKIP tiles."""
    cfg, P, th, _, _, _ = random_case(4, views=5, nu=24, nv=18)
    shape = (23, 70, 70)
    sp = (25.0, 25.0, 25.0)   # 1.75 m wide: corners reach beyond the source circle
    origin = tuple(-(n - 1) / 2.0 * s for n, s in zip(shape[::-1], sp))
    # smooth data: at 13 px per voxel a tile spans hundreds of pixels, where
    # white noise would turn the FP32 position resolution into 1e-5 errors;
    # this case is about the SKIP / EDGE / behind-the-source logic
    vv, uu = np.meshgrid(np.arange(18), np.arange(24), indexing="ij")
    proj = np.stack([np.sin(0.21 * uu + 0.3 * j) * np.cos(0.17 * vv - 0.1 * j) + 0.5
                     for j in range(5)]).astype(np.float32)
    rng = np.random.default_rng(9)
    delta = rng.standard_normal(shape).astype(np.float32)
    Ph = oracle.compose(P, th)
    ref = oracle.bp_forward(Ph, proj.astype(np.float64), shape, sp, origin, None,
                            oracle.WEIGHT_FDK, cfg.sid)
    got = gpu_forward(proj, P, th, shape, sp, origin, None, "fdk", cfg.sid)
    assert rel_l2(got, ref) <= VOL_TOL
    oP, oD = oracle.bp_vjp(Ph, proj.astype(np.float64), delta.astype(np.float64), sp, origin,
                           None, oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid)
    gm, gP, gD = gpu_vjp(delta, proj, P, th, sp, origin, None, "fdk", "central", cfg.sid)
    assert rel_l2(gP, oP) <= GRAD_TOL
    # the data VJP weights the white-noise upstream gradient by detector
    # positions; at 13 px per voxel FP32 resolves them to ~1e-5 px, so this
    # stress geometry gets 1e-4 (a SKIP/EDGE logic error would be O(1))
    assert rel_l2(gD, oD) <= 1e-4


def test_empty_and_degenerate():
    cfg, P, th, proj, delta, origin = random_case(5)
    sp = (cfg.spacing,) * 3
    # no views -> zero volume
    v = bp.bp_forward(cuda(proj[:0]), cuda(P[:0]), None, vol_shape=delta.shape, spacing=sp,
                      origin=origin, weight="fdk", sid=cfg.sid)
    assert float(v.abs().max()) == 0.0
    # empty volume
    v = bp.bp_forward(cuda(proj), cuda(P), cuda(th), vol_shape=(0, 5, 5), spacing=sp,
                      origin=origin, weight="fdk", sid=cfg.sid)
    assert v.numel() == 0
    # volume entirely off the detector (shifted 10 m away)
    far = (1e4, 1e4, 1e4)
    v = gpu_forward(proj, P, th, delta.shape, sp, far, None, "fdk", cfg.sid)
    assert np.abs(v).max() == 0.0
    # one-pixel detector row / column
    proj1 = proj[:, :1, :]
    ref = oracle.bp_forward(oracle.compose(P, th), proj1.astype(np.float64), delta.shape, sp,
                            origin, None, oracle.WEIGHT_NONE, cfg.sid)
    got = gpu_forward(proj1, P, th, delta.shape, sp, origin, None, "none", cfg.sid)
    assert rel_l2(got, ref) <= VOL_TOL or np.abs(ref).max() == 0.0
    # zero upstream gradient -> zero gradients
    gm, gP, gD = gpu_vjp(np.zeros_like(delta), proj, P, th, sp, origin)
    assert np.abs(gm).max() == 0.0 and np.abs(gP).max() == 0.0 and np.abs(gD).max() == 0.0


def test_invalid_arguments_raise():
    cfg, P, th, proj, delta, origin = random_case(6)
    with pytest.raises(RuntimeError):
        bp.bp_forward(cuda(proj), cuda(P), cuda(th), vol_shape=delta.shape, spacing=(0, 1, 1),
                      origin=origin)
    with pytest.raises(TypeError):
        bp.bp_forward(cuda(proj).double(), cuda(P), cuda(th), vol_shape=delta.shape,
                      spacing=(1, 1, 1), origin=origin)


def test_host_buffers_match_device():
    cfg, P, th, proj, delta, origin = random_case(7)
    sp = (cfg.spacing,) * 3
    dev = gpu_forward(proj, P, th, delta.shape, sp, origin)
    host = bp.bp_forward(torch.as_tensor(proj), torch.as_tensor(P), torch.as_tensor(th),
                         vol_shape=delta.shape, spacing=sp, origin=origin, weight="fdk",
                         sid=cfg.sid)
    assert host.device.type == "cpu"
    assert np.array_equal(host.numpy(), dev)
    gm_d, gP_d, gD_d = gpu_vjp(delta, proj, P, th, sp, origin, want=(True, True, False))
    gm_h, gP_h, _ = bp.bp_vjp(torch.as_tensor(delta), torch.as_tensor(proj), torch.as_tensor(P),
                              torch.as_tensor(th), spacing=sp, origin=origin, weight="fdk",
                              sid=cfg.sid, want_Phat=True)
    assert np.array_equal(gm_h.numpy(), gm_d) and np.array_equal(gP_h.numpy(), gP_d)


def test_strided_projections():
    cfg, P, th, proj, delta, origin = random_case(8)
    sp = (cfg.spacing,) * 3
    V, nv, nu = proj.shape
    padded = np.zeros((V, nv + 3, nu + 5), np.float32)
    padded[:, :nv, :nu] = proj
    ref = gpu_forward(proj, P, th, delta.shape, sp, origin)
    # view into a padded buffer through the raw C-ABI descriptor
    import ctypes
    from paper_2401_09283_gb300 import native as N
    buf = cuda(padded)
    out = torch.empty(delta.shape, dtype=torch.float32, device=DEV)
    pd = N.ProjDesc(nu, nv, V, N.F32, nu + 5, (nu + 5) * (nv + 3), None, cfg.sid)
    vd = N.vol_desc(delta.shape, sp, origin)
    ctx = N.context(0)
    Pd, thd = cuda(P), cuda(th)
    rc = N.lib().bp_forward(ctx, buf.data_ptr(), ctypes.byref(pd), Pd.data_ptr(), thd.data_ptr(),
                            None, 1, ctypes.byref(vd), out.data_ptr(), N.stream_of(buf))
    N.check("bp_forward", rc, ctx)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


# ---------------------------------------------------------- reduced precision

@pytest.mark.parametrize("dtype,tol", [(torch.float16, FP16_STORAGE_TOL),
                                       (torch.bfloat16, BF16_STORAGE_TOL)])
def test_c1_half_storage(dtype, tol):
    cfg, P, th, proj, delta = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    # per-view scale; the first and last views are all zero (short-scan weights)
    scale = np.maximum(np.abs(proj).reshape(cfg.views, -1).max(axis=1), 1e-30).astype(np.float32)
    stored = torch.as_tensor(proj / scale[:, None, None]).to(dtype)
    deq = (stored.float().numpy() * scale[:, None, None]).astype(np.float64)
    Ph = oracle.compose(P, th)
    ref32 = oracle.bp_forward(Ph, proj.astype(np.float64), cfg.vol_shape, cfg.spacing3, cfg.origin,
                              vw, oracle.WEIGHT_FDK, cfg.sid)
    refq = oracle.bp_forward(Ph, deq, cfg.vol_shape, cfg.spacing3, cfg.origin, vw,
                             oracle.WEIGHT_FDK, cfg.sid)
    p = stored.to(DEV)
    got = bp.bp_forward(p, cuda(P), cuda(th), vol_shape=cfg.vol_shape, spacing=cfg.spacing3,
                        origin=cfg.origin, view_weight=cuda(vw), weight="fdk", sid=cfg.sid,
                        view_scale=cuda(scale)).cpu().numpy()
    assert rel_l2(got, refq) <= VOL_TOL          # kernel arithmetic on what it stores
    assert rel_l2(got, ref32) <= tol             # storage error against FP32 data
    # motion gradient on the stored data
    oP, _ = oracle.bp_vjp(Ph, deq, delta.astype(np.float64), cfg.spacing3, cfg.origin, vw,
                          oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
    om = oracle.chain_motion(P, th, oP)
    gm, _, _ = bp.bp_vjp(cuda(delta), p, cuda(P), cuda(th), spacing=cfg.spacing3,
                         origin=cfg.origin, view_weight=cuda(vw), weight="fdk", sid=cfg.sid,
                         view_scale=cuda(scale))
    assert motion_rel(gm.cpu().numpy(), om) <= GRAD_TOL


# ------------------------------------------------------ loss, optimisers, compose

def test_compose_matches_oracle():
    cfg, P, th, _, _ = scan_case("c1")
    got = bp.bp_compose(cuda(P), cuda(th)).cpu().numpy()
    ref = oracle.compose(P, th)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(bp.bp_compose(cuda(P), None).cpu().numpy(), P)


def test_sharpness_matches_oracle():
    rng = np.random.default_rng(0)
    vol = rng.standard_normal((13, 17, 19)).astype(np.float32)
    L, g = bp.bp_sharpness(cuda(vol))
    Lo, go = oracle.sharpness(vol.astype(np.float64))
    assert abs(float(L) - Lo) <= 1e-6 * abs(Lo)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-5 * np.abs(go).max()


def test_tv_matches_oracle():
    rng = np.random.default_rng(4)
    vol = rng.standard_normal((13, 17, 19)).astype(np.float32)
    for eps in (1e-3, 0.5):
        L, g = bp.bp_tv(cuda(vol), eps)
        Lo, go = oracle.tv(vol.astype(np.float64), eps)
        assert abs(float(L) - Lo) <= 1e-6 * abs(Lo)
        assert np.abs(g.cpu().numpy() - go).max() <= 1e-5 * np.abs(go).max()


def test_optimisers_match_oracle():
    rng = np.random.default_rng(1)
    th = rng.standard_normal((50, 6))
    gr = rng.standard_normal((50, 6))
    t = cuda(th)
    bp.bp_gd_step(t, cuda(gr), 100.0, 0.97, 3, gauge=True)
    assert np.allclose(t.cpu().numpy(), oracle.gd_step(th, gr, 100.0, 0.97, 3), atol=1e-12)
    t = cuda(th)
    m1 = torch.zeros_like(t)
    m2 = torch.zeros_like(t)
    o_t, o1, o2 = th, np.zeros_like(th), np.zeros_like(th)
    for n in (1, 2, 3):
        g = rng.standard_normal((50, 6))
        bp.bp_adam_step(t, cuda(g), m1, m2, 0.05, n, gauge=True)
        o_t, o1, o2 = oracle.adam_step(o_t, g, o1, o2, 0.05, n)
    assert np.allclose(t.cpu().numpy(), o_t, atol=1e-12)
