"""FDK preprocessing on the GPU (bp_fdk_filter) against the oracle's direct
convolution (c1, short scan; a full scan) and against the FFT input generator
at full c2 size."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2401_09283_gb300.workloads as W
from cases import rel_l2

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("name,views,nv,nu", [("c1", 60, 96, 128), ("paper", 9, 13, 70),
                                               ("c1", 5, 7, 37)])
def test_matches_oracle(name, views, nv, nu):
    from paper_2401_09283_gb300 import bp
    cfg = W.CONFIGS[name]
    raw = np.random.default_rng(views + nu).standard_normal((views, nv, nu)).astype(np.float32)
    want = oracle.fdk_filter(raw, cfg.pitch, cfg.sid, cfg.sdd, math.radians(cfg.arc_deg))
    got = bp.bp_fdk_filter(torch.as_tensor(raw, device=DEV), pitch=cfg.pitch, sid=cfg.sid,
                           sdd=cfg.sdd, arc=math.radians(cfg.arc_deg)).cpu().numpy()
    assert rel_l2(got, want) <= 1e-6
    # host arrays give the device result
    host = bp.bp_fdk_filter(torch.as_tensor(raw), pitch=cfg.pitch, sid=cfg.sid, sdd=cfg.sdd,
                            arc=math.radians(cfg.arc_deg)).numpy()
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
