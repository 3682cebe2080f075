"""bp_sharpness_noalloc: the allocation-free entry point, for callers that
cannot allocate device memory during a call (graph capture, pooled or
real-time hosts).  It must give the oracle's sharpness loss and gradient,
and what bp_sharpness gives: the gradient bit for bit (same per-voxel
arithmetic), the loss up to the order of its FP64 sums.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before it.  It also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2401_09283_gb300 import bp, native  # noqa: E402

DEV = torch.device("cuda:0")


def noalloc(vol, want_grad=True):
    loss = torch.empty((), dtype=torch.float64, device=DEV)
    grad = torch.empty_like(vol) if want_grad else None
    vd = native.vol_desc(vol.shape, (1, 1, 1), (0, 0, 0))
    rc = native.lib().bp_sharpness_noalloc(vol.data_ptr(), ctypes.byref(vd), loss.data_ptr(),
                                           None if grad is None else grad.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == native.BP_OK, native.STATUS.get(rc, rc)
    return loss, grad


def test_noalloc_matches_bp_sharpness_on_two_calls():
    torch.cuda.set_device(DEV)
    rng = np.random.default_rng(11)
    # a larger volume first, then a smaller one: the second call must not see
    # partial sums left over from the first
    shapes = [(37, 53, 61), (13, 17, 19)]
    for shape in shapes:
        vol = torch.as_tensor(rng.standard_normal(shape).astype(np.float32), device=DEV)
        L_ref, g_ref = bp.bp_sharpness(vol)
        L, g = noalloc(vol)
        torch.cuda.synchronize()
        gr, gg = g_ref.cpu().numpy(), g.cpu().numpy()
        assert np.array_equal(gg, gr)
        assert abs(float(L) - float(L_ref)) <= 1e-12 * abs(float(L_ref))
        # against the FP64 oracle: the kernels round each difference to FP32
        # (relative 2^-24, squared in FP64) and sum the six differences of
        # the gradient in FP32
        Lo, go = oracle.sharpness(vol.cpu().numpy().astype(np.float64))
        assert abs(float(L) - Lo) <= 1e-6 * abs(Lo)
        assert np.abs(gg - go).max() <= 1e-5 * np.abs(go).max()


def test_noalloc_rejects_bad_sizes_and_host_memory():
    torch.cuda.set_device(DEV)
    vol = torch.zeros((4, 4, 4), dtype=torch.float32, device=DEV)
    loss = torch.empty((), dtype=torch.float64, device=DEV)
    big = native.vol_desc((513, 512, 512), (1, 1, 1), (0, 0, 0))
    rc = native.lib().bp_sharpness_noalloc(vol.data_ptr(), ctypes.byref(big), loss.data_ptr(),
                                           None, None)
    assert rc == -4  # BP_ERR_UNSUPPORTED: above the 512^3 limit
    host = torch.zeros((4, 4, 4), dtype=torch.float32)
    vd = native.vol_desc((4, 4, 4), (1, 1, 1), (0, 0, 0))
    rc = native.lib().bp_sharpness_noalloc(host.data_ptr(), ctypes.byref(vd), loss.data_ptr(),
                                           None, None)
    assert rc == -1  # BP_ERR_INVALID_ARG: device memory only
