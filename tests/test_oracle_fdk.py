"""Pins of the oracle's FDK preprocessing (direct convolution): against the
input generator's independent FFT implementation, the ramp's impulse response
in closed form, the cosine weight at the principal point, and Parker's
conjugate-ray identity."""
import math

import numpy as np
import torch

import oracle
import paper_2401_09283_gb300.workloads as W


def test_matches_fft_generator_short_and_full_scan():
    rng = np.random.default_rng(0)
    for cfg in (W.C1, W.PAPER):
        small = W.ScanConfig(**{**cfg.__dict__, "views": 7, "nu": 40, "nv": 9})
        raw = rng.standard_normal((7, 9, 40))
        want = W.fdk_filter(torch.as_tensor(raw), small).numpy()
        # the generator spreads short-scan views over the arc like the geometry
        got = oracle.fdk_filter(raw, small.pitch, small.sid, small.sdd, math.radians(small.arc_deg))
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
        # with the truncation correction (rows extended by 10 % per side)
        want = W.fdk_filter(torch.as_tensor(raw), small, ext=4).numpy()
        got = oracle.fdk_filter(raw, small.pitch, small.sid, small.sdd,
                                math.radians(small.arc_deg), ext=4)
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_ramp_impulse_response_closed_form():
    nu, nv, pitch, sid, sdd = 33, 1, 1.0, 750.0, 1200.0
    raw = np.zeros((1, nv, nu))
    raw[0, 0, 16] = 1.0
    q = oracle.fdk_filter(raw, pitch, sid, sdd, 2 * math.pi)   # full scan: weight 1/2
    tau = pitch * sid / sdd
    x = 0.0
    c = sdd / math.sqrt(sdd * sdd + x * x)   # principal column, single row at y = 0
    n = np.arange(nu) - 16
    want = 0.5 * c * tau * (-2.0 / (math.pi ** 2 * tau ** 2 * (4.0 * n * n - 1.0)))
    assert np.max(np.abs(q[0, 0] - want)) <= 1e-12 * np.max(np.abs(want))


def test_parker_conjugate_rays_sum_to_one():
    arc = math.radians(200.0)
    rng = np.random.default_rng(1)
    for _ in range(200):
        g = rng.uniform(-0.15, 0.15)
        delta = (arc - math.pi) / 2
        b = rng.uniform(0, 2 * delta + 2 * g)  # so that the conjugate beta + pi - 2g <= arc
        s = oracle.parker(b, g, arc) + oracle.parker(b + math.pi - 2 * g, -g, arc)
        assert abs(s - 1.0) < 1e-12
    assert oracle.parker(0.0, 0.0, arc) == 0.0


def test_truncation_extension_is_a_linear_fall_off():
    """A row that is constant c after weighting (full scan, one row at the
    principal point, tiny pitch so the cosine weight is ~1) filtered with the
    extension equals the filter of the explicitly extended row: c on the
    detector and c (1 - m/E) on extension pixel m."""
    nu, E, pitch, sid, sdd = 24, 5, 1e-3, 750.0, 1200.0
    raw = np.full((1, 1, nu), 2.0)
    got = oracle.fdk_filter(raw, pitch, sid, sdd, 2 * math.pi, ext=E)
    tau = pitch * sid / sdd
    x = (np.arange(nu) - 0.5 * (nu - 1)) * pitch
    row = 0.5 * 2.0 * sdd / np.sqrt(sdd ** 2 + x ** 2)
    m = np.arange(1, E + 1)
    ext = np.concatenate([row[0] * (1 - m / E)[::-1], row, row[-1] * (1 - m / E)])
    n = np.arange(-(nu + 2 * E - 1), nu + 2 * E)
    h = -2.0 / (math.pi ** 2 * tau ** 2 * (4.0 * n * n - 1.0))
    full = np.convolve(ext, h)                       # index i + j
    want = tau * full[(nu + 2 * E - 1) + E: (nu + 2 * E - 1) + E + nu]
    assert np.max(np.abs(got[0, 0] - want)) <= 1e-10 * np.max(np.abs(want))
    # without the extension the result differs (the edges see the cut)
    assert np.max(np.abs(oracle.fdk_filter(raw, pitch, sid, sdd, 2 * math.pi) - got)) > 1e-3
