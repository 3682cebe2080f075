"""FDK preprocessing on the GPU (bp_fdk_filter) against the oracle's direct
convolution (c1, short scan; a full scan; with and without the truncation
extension) and against the FFT input generator at full c2 size."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2401_09283_gb300.workloads as W
from cases import rel_l2

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("name,views,nv,nu,ext", [("c1", 60, 96, 128, 0), ("paper", 9, 13, 70, 0),
                                                   ("c1", 5, 7, 37, 0), ("c1", 60, 96, 128, 13),
                                                   ("paper", 9, 13, 70, 7), ("c1", 4, 6, 20, 1)])
def test_matches_oracle(name, views, nv, nu, ext):
    from paper_2401_09283_gb300 import bp
    cfg = W.CONFIGS[name]
    raw = np.random.default_rng(views + nu).standard_normal((views, nv, nu)).astype(np.float32)
    geo = dict(pitch=cfg.pitch, sid=cfg.sid, sdd=cfg.sdd, arc=math.radians(cfg.arc_deg))
    want = oracle.fdk_filter(raw, ext=ext, **geo)
    got = bp.bp_fdk_filter(torch.as_tensor(raw, device=DEV), ext=ext, **geo).cpu().numpy()
    assert rel_l2(got, want) <= 1e-6
    # host arrays give the device result
    host = bp.bp_fdk_filter(torch.as_tensor(raw), ext=ext, **geo).numpy()
    assert np.array_equal(host, got)


def test_full_size_c2_against_fft_generator():
    from paper_2401_09283_gb300 import bp
    cfg = W.C2
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    raw = torch.rand((cfg.views, cfg.nv, cfg.nu), device=DEV, generator=g)
    want = W.fdk_filter(raw.double(), cfg).cpu().numpy()
    got = bp.bp_fdk_filter(raw, pitch=cfg.pitch, sid=cfg.sid, sdd=cfg.sdd,
                           arc=math.radians(cfg.arc_deg)).cpu().numpy()
    assert rel_l2(got, want) <= 1e-6


def test_invalid_arguments():
    from paper_2401_09283_gb300 import bp, native as N
    raw = torch.zeros((4, 5, 16), device=DEV)
    with pytest.raises(N.BPError):
        bp.bp_fdk_filter(raw, pitch=1.0, sid=750.0, sdd=1200.0, arc=math.radians(150.0))
    with pytest.raises(N.BPError):
        bp.bp_fdk_filter(torch.zeros((1, 1, 8193), device=DEV), pitch=1.0, sid=750.0, sdd=1200.0,
                         arc=2 * math.pi)
    with pytest.raises(N.BPError):
        bp.bp_fdk_filter(torch.zeros((1, 1, 8000), device=DEV), pitch=1.0, sid=750.0, sdd=1200.0,
                         arc=2 * math.pi, ext=100)
