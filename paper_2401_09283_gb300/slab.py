"""One scan across several GPUs: the volume split into z-slabs.

Each rank owns a contiguous range of volume slices.  The backprojection of
Eq. 3 is per voxel, so a rank backprojects its slab from the full projection
stack with no communication.  The motion Jacobian of Eqs. 4-5 is a sum over
voxels, per view: each rank's bp_vjp on its slab gives a partial dL/dPhat
(V x 12) and, through the chain of Eq. 2 -- linear in dL/dPhat -- a partial
dL/dtheta (V x 6).  One all-reduce (sum) of those V x 18 float64 values gives
every rank the gradient of the whole volume, so the optimiser step that
follows is identical on every rank.  dL/dproj is not reduced here: the
detector rows that two slabs touch overlap, and a rank that needs it sums
the ranks' images itself.

The collective is torch.distributed's all_reduce (NCCL for CUDA tensors,
gloo for CPU tensors); nothing else crosses ranks.  Plain NCCL: no cluster
multicast or other single-GPU-only transfer is used on this path.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch

from . import bp


def slab_range(nz: int, rank: int, world: int) -> Tuple[int, int]:
    """Slices [z0, z1) of rank `rank` among `world`: contiguous, sizes differ
    by at most one, lower ranks first."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(int(nz), int(world))
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def slab_geometry(vol_shape, spacing, origin, rank: int, world: int):
    """(slab shape (nz_r, ny, nx), slab origin, (z0, z1)) of a rank: the
    slab's first slice sits z0 voxels above the volume's."""
    nz, ny, nx = (int(n) for n in vol_shape)
    z0, z1 = slab_range(nz, rank, world)
    o = (float(origin[0]), float(origin[1]), float(origin[2]) + z0 * float(spacing[2]))
    return (z1 - z0, ny, nx), o, (z0, z1)


def forward_slab(proj, P, motion=None, *, vol_shape, spacing, origin, rank: int, world: int,
                 **kw) -> torch.Tensor:
    """This rank's slab of bp_forward (no communication)."""
    shape, o, _ = slab_geometry(vol_shape, spacing, origin, rank, world)
    return bp.bp_forward(proj, P, motion, vol_shape=shape, spacing=spacing, origin=o, **kw)


def allreduce_sum(group=None) -> Callable[[torch.Tensor], None]:
    """In-place sum over the ranks of `group` (torch.distributed)."""
    import torch.distributed as dist

    def f(t: torch.Tensor) -> None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return f


def reduce_motion_partials(dL_dPhat: torch.Tensor, dL_dmotion: torch.Tensor,
                           reduce: Optional[Callable[[torch.Tensor], None]]):
    """Sum the per-rank partial gradients with ONE collective: dL/dPhat
    (V,3,4) and dL/dmotion (V,6) float64 travel in one V x 18 buffer.
    `reduce` sums a tensor in place over the ranks (None: a single rank)."""
    V = dL_dPhat.shape[0]
    buf = torch.cat([dL_dPhat.reshape(V, 12), dL_dmotion.reshape(V, 6)], dim=1).contiguous()
    if reduce is not None:
        reduce(buf)
    return buf[:, :12].reshape(V, 3, 4).clone(), buf[:, 12:].clone()


def vjp_slab(dL_dvol_slab, proj, P, motion=None, *, vol_shape, spacing, origin, rank: int,
             world: int, reduce: Optional[Callable[[torch.Tensor], None]] = None, **kw):
    """Motion gradient of the whole volume from this rank's slab of dL/dvol:
    the slab's bp_vjp (Eqs. 4-5, chained by Eq. 2), then one all-reduce of
    the V x 18 partial sums.  Returns (dL/dmotion (V,6), dL/dPhat (V,3,4)),
    equal on every rank."""
    shape, o, _ = slab_geometry(vol_shape, spacing, origin, rank, world)
    if tuple(dL_dvol_slab.shape) != shape:
        raise ValueError("dL/dvol slab has shape %s, rank %d owns %s"
                         % (tuple(dL_dvol_slab.shape), rank, shape))
    gm, gP, _ = bp.bp_vjp(dL_dvol_slab, proj, P, motion, spacing=spacing, origin=o,
                          want_motion=True, want_Phat=True, want_proj=False, **kw)
    gP, gm = reduce_motion_partials(gP, gm, reduce)
    return gm, gP
