"""The z-slab split of one scan through the library on one GPU: the ranks'
slabs (run one after another here) assemble the whole-volume backprojection,
and the sum of their partial motion gradients -- what the all-reduce of the
multi-GPU path computes -- equals the whole-volume VJP and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from cases import motion_errors, rel_l2, scan_case
from paper_2401_09283_gb300 import bp, slab

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEV = torch.device("cuda:0")


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_slabs_assemble_the_whole_volume_and_its_gradient(world):
    cfg, P, th, proj, delta = scan_case("c1")
    vw = np.full(cfg.views, cfg.delta_beta)
    kw = dict(view_weight=cuda(vw), weight="fdk", sid=cfg.sid)
    geo = dict(vol_shape=cfg.vol_shape, spacing=cfg.spacing3, origin=cfg.origin)
    pd, Pd, thd = cuda(proj), cuda(P), cuda(th)
    whole = bp.bp_forward(pd, Pd, thd, **geo, **kw).cpu().numpy()
    parts, gms, gPs = [], [], []
    for r in range(world):
        parts.append(slab.forward_slab(pd, Pd, thd, rank=r, world=world, **geo, **kw).cpu().numpy())
        z0, z1 = slab.slab_range(cfg.n, r, world)
        gm, gP = slab.vjp_slab(cuda(delta[z0:z1]), pd, Pd, thd, rank=r, world=world, reduce=None,
                               **geo, **kw)
        gms.append(gm.cpu().numpy())
        gPs.append(gP.cpu().numpy())
    vol = np.concatenate(parts, axis=0)
    # per-voxel sums; only the tile anchors differ between the two tilings
    assert rel_l2(vol, whole) <= 1e-6
    gm_sum, gP_sum = np.sum(gms, axis=0), np.sum(gPs, axis=0)
    wm, wP, _ = bp.bp_vjp(cuda(delta), pd, Pd, thd, spacing=cfg.spacing3, origin=cfg.origin,
                          want_Phat=True, **kw)
    assert max(motion_errors(gm_sum, wm.cpu().numpy())) <= 1e-5
    assert rel_l2(gP_sum, wP.cpu().numpy()) <= 1e-5
    Ph = oracle.compose(P, th)
    ref = oracle.bp_forward(Ph, proj.astype(np.float64), cfg.vol_shape, cfg.spacing3, cfg.origin,
                            vw, oracle.WEIGHT_FDK, cfg.sid)
    assert rel_l2(vol, ref) <= 1e-5
    oP, _ = oracle.bp_vjp(Ph, proj.astype(np.float64), delta.astype(np.float64), cfg.spacing3,
                          cfg.origin, vw, oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid,
                          want_proj=False)
    assert max(motion_errors(gm_sum, oracle.chain_motion(P, th, oP))) <= 1e-3
