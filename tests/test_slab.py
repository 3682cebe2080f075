"""The z-slab split of one scan on the CPU: the partition of the slices, and
two gloo ranks that each take the oracle's VJP of their own slab and sum the
V x 18 partials with the one all-reduce of `slab.reduce_motion_partials`;
both ranks must end with the oracle's gradient of the whole volume."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2401_09283_gb300 import slab
from paper_2401_09283_gb300 import workloads as W


@pytest.mark.parametrize("nz,world", [(16, 2), (17, 3), (5, 8), (256, 8), (1, 1)])
def test_slab_ranges_partition_the_slices(nz, world):
    ranges = [slab.slab_range(nz, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == nz
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_slab_geometry_moves_the_origin():
    shape, o, (z0, z1) = slab.slab_geometry((17, 5, 6), (1.0, 2.0, 3.0), (-1.0, -2.0, -3.0), 2, 3)
    assert (z0, z1) == (12, 17) and shape == (5, 5, 6)
    assert o == (-1.0, -2.0, -3.0 + 12 * 3.0)
    with pytest.raises(ValueError):
        slab.slab_range(4, 3, 3)


def _case():
    cfg = W.C4_GRADCHECK
    P = W.projection_matrices(cfg)
    th = W.motion_curves(cfg)
    rng = np.random.default_rng(7)
    proj = rng.standard_normal((cfg.views, cfg.nv, cfg.nu))
    delta = rng.standard_normal(cfg.vol_shape)
    return cfg, P, th, proj, delta


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    cfg, P, th, proj, delta = _case()
    shape, o, (z0, z1) = slab.slab_geometry(cfg.vol_shape, cfg.spacing3, cfg.origin, rank, ws)
    vw = np.full(cfg.views, cfg.delta_beta)
    Ph = oracle.compose(P, th)
    gP, _ = oracle.bp_vjp(Ph, proj, delta[z0:z1], cfg.spacing3, o, vw, oracle.WEIGHT_FDK,
                          oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
    gm = oracle.chain_motion(P, th, gP)
    tP, tm = slab.reduce_motion_partials(torch.as_tensor(gP), torch.as_tensor(gm),
                                         slab.allreduce_sum())
    out[rank] = (tP.numpy(), tm.numpy())
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slab_partials_to_the_whole_volume_gradient():
    ws, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    cfg, P, th, proj, delta = _case()
    vw = np.full(cfg.views, cfg.delta_beta)
    Ph = oracle.compose(P, th)
    wP, _ = oracle.bp_vjp(Ph, proj, delta, cfg.spacing3, cfg.origin, vw, oracle.WEIGHT_FDK,
                          oracle.DERIV_CENTRAL, cfg.sid, want_proj=False)
    wm = oracle.chain_motion(P, th, wP)
    for r in range(ws):
        gP, gm = out[r]
        assert np.allclose(gP, wP, rtol=1e-10, atol=1e-10 * np.abs(wP).max())
        assert np.allclose(gm, wm, rtol=1e-10, atol=1e-10 * np.abs(wm).max())
    assert np.array_equal(out[0][1], out[1][1])  # every rank steps with the same gradient
