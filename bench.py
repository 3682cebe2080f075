#!/usr/bin/env python
"""Benchmark of the motion-compensated backprojection hot path on GB300.

One step = one pass of the whole hot path over the head-size workload
(256^3 voxels at 1 mm, 248 views over 200 degrees, 616x480 detector, FP32,
FDK weights, seeded 30-ellipsoid phantom with 1 % noise and 12-knot motion):
  compose (Eq. 1) -> backprojection (Eq. 3) -> sharpness loss and dL/dvol ->
  gradient images + motion VJP (Eqs. 4-5) -> FP64 per-view reduction and
  chain rule (Eq. 2) -> data VJP (adjoint of Eq. 3) -> Adam update.
The metric counts voxel-view updates: every step makes three passes over the
N^3 x V voxel-view pairs (forward, motion VJP, data VJP).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torchrun: each rank runs an independent replica (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-view updates/s (fwd+VJP)"
UNIT = "voxel-view updates/s"
PASSES = 3          # forward, motion VJP, data VJP
SM_MAX_MHZ = 2070.0  # GB300 maximum SM clock (roofline peak)

# Algorithmic cost per voxel-view update of each pass (minimal FP32 lane
# operations and gathered/scattered samples), used for the ALU/LSU roofline.
PASS_COST = {
    "forward": {"fp32": 16, "samples": 4},      # FDK weighting
    "vjp_motion": {"fp32": 38, "samples": 12},  # CENTRAL g_u, g_v + FDK value
    "vjp_proj": {"fp32": 12, "samples": 4},
    "vjp_fused": {"fp32": 50, "samples": 16},   # motion and data VJP in one pass
}


# DRAM bytes (read + write) per launch of each kernel on the c2 workload:
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of the
# current kernels at full c2 size (one launch each; the capture and its
# command are kept with the profiles).  "vjp_fused" is the fused VJP kernel
# plus the block-image combine kernel (3.644e9 + 1.747e9); the block image's
# memset (1.17 GB written) is not a kernel of ours and not included.
# Reported as the roofline's "traffic" for c2 only; it must be re-captured
# whenever one of these kernels changes.
NCU_TRAFFIC_C2 = {"forward": 0.4639e9, "vjp_fused": 5.3908e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="c2")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--quick", action="store_true", help="skip clocks/e2e/cpu legs (profiling)")
    ap.add_argument("--me-iters", type=int, default=100, help="motion-estimation leg iterations")
    ap.add_argument("--serving", type=int, default=16, help="jobs of the serving leg (0 = skip)")
    ap.add_argument("--serving-repeats", type=int, default=3,
                    help="runs of each serving form (spread of jobs/s)")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the 512^3 precision form (FP32/FP16/BF16 storage)")
    ap.add_argument("--paper-iters", type=int, default=100,
                    help="iterations of the paper-setup leg (0 = skip)")
    return ap.parse_args()


def job_throughput(ms_local, units_per_step, steps, ws, device):
    """Whole-job throughput of N independent replicas (weak scaling): the
    slowest rank's time (max over ranks, one all-reduce of a scalar) and the
    units all ranks processed divided by it.  Returns (ms, units/s)."""
    import torch
    ms = float(ms_local)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t)
    return ms, units_per_step * ws * steps / (ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def roofline_peak(kernel, sms):
    c = PASS_COST[kernel]
    f = SM_MAX_MHZ * 1e6
    r_fp32 = sms * 128 * f / c["fp32"]
    r_lsu = sms * 32 * f / c["samples"]
    return min(r_fp32, r_lsu), r_fp32, r_lsu


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        loaded = [s for s in sm if s > 0]
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------- workload

def make_inputs(cfg, device):
    import torch

    import paper_2401_09283_gb300.workloads as W
    from paper_2401_09283_gb300 import bp
    P = W.projection_matrices(cfg)
    th_true = W.motion_curves(cfg)
    Pd = torch.as_tensor(P, device=device)
    Pm = bp.bp_compose(Pd, torch.as_tensor(th_true, device=device)).cpu().numpy()
    ph = W.head_phantom(cfg)
    raw = W.line_integrals(ph, Pm, cfg.nu, cfg.nv, device=device, dtype=torch.float32,
                           views_per_chunk=32)
    raw = W.add_noise(raw, cfg.noise, cfg.phantom_seed + 100) if cfg.noise > 0 else raw
    proj = W.fdk_filter(raw, cfg).to(torch.float32).contiguous()
    del raw
    return P, th_true, proj


def run_ours(args):
    import torch

    import paper_2401_09283_gb300.workloads as W
    from paper_2401_09283_gb300 import bp, native

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = W.CONFIGS[args.config]
    P, th_true, proj = make_inputs(cfg, dev)
    V = cfg.views
    Pd = torch.as_tensor(P, device=dev)
    vw = torch.full((V,), cfg.delta_beta, dtype=torch.float64, device=dev)
    theta = torch.zeros((V, 6), dtype=torch.float64, device=dev)
    m1 = torch.zeros_like(theta)
    m2 = torch.zeros_like(theta)
    vol = torch.empty(cfg.vol_shape, dtype=torch.float32, device=dev)
    dvol = torch.empty_like(vol)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    g_th = torch.empty_like(theta)
    g_P = torch.empty((V, 3, 4), dtype=torch.float64, device=dev)
    g_D = torch.empty_like(proj)
    geo = dict(spacing=cfg.spacing3, origin=cfg.origin, weight="fdk", sid=cfg.sid)
    lr = 1e-3
    it = [0]

    def step():
        it[0] += 1
        bp.bp_forward(proj, Pd, theta, vol_shape=cfg.vol_shape, view_weight=vw, out=vol, **geo)
        bp.bp_sharpness(vol, loss_out=loss, grad_out=dvol)
        bp.bp_vjp(dvol, proj, Pd, theta, view_weight=vw, deriv="central", want_Phat=True,
                  want_proj=True, out_motion=g_th, out_Phat=g_P, out_proj=g_D, **geo)
        bp.bp_adam_step(theta, g_th, m1, m2, lr, it[0])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier = (lambda: torch.distributed.barrier()) if ws > 1 else (lambda: None)
    clocks = None if args.quick else ClockSampler(local)
    native.set_timing(True, local)
    launches0 = native.launch_count(local)
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.4)
    s = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    ms_total = e0.elapsed_time(e1)
    launches = native.launch_count(local) - launches0
    ktimes = native.kernel_times(local)
    native.set_timing(False, local)
    updates_step = PASSES * cfg.voxel_views
    ms_total, value = job_throughput(ms_total, updates_step, args.steps, ws, dev)
    ms_step = ms_total / args.steps

    # roofline of the dominant kernel
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    dom = max(PASS_COST, key=lambda k: ktimes[k][0])
    k_ms, k_n = ktimes[dom]
    achieved = cfg.voxel_views / ((k_ms / k_n) / 1e3)
    peak, r_fp32, r_lsu = roofline_peak(dom, sms)
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gupdate/s", "frac": achieved / peak,
            "traffic": NCU_TRAFFIC_C2.get(dom) if cfg.name == W.C2.name else None,
            "traffic_unit": "bytes per launch (ncu dram__bytes_read+write; vjp_fused: VJP "
                            "kernel + block-image combine)",
            "peak_basis": "min(FP32 issue %.0f, LSU %.0f) Gupdate/s at %d SMs x %.0f MHz"
                          % (r_fp32 / 1e9, r_lsu / 1e9, sms, SM_MAX_MHZ)}
    kernels = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else None, "launches": v[1],
                   "share": v[0] / max(1e-9, sum(x[0] for x in ktimes.values()))}
               for k, v in ktimes.items() if v[1]}
    for k in PASS_COST:
        if ktimes[k][1]:
            kernels[k]["Gupdate_per_s"] = cfg.voxel_views / (ktimes[k][0] / ktimes[k][1] / 1e3) / 1e9
            kernels[k]["roofline_frac"] = (kernels[k]["Gupdate_per_s"] * 1e9) / roofline_peak(k, sms)[0]

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(cfg, ws),
           "gpu_launches": launches, "roofline": roof, "kernels": kernels,
           "loss_last": float(loss)}
    if clk:
        out["clocks"] = clk
    if not args.quick:
        out["probes"] = probe_leg(local, sms, clk)

    if not args.no_e2e and not args.quick:
        out["e2e"] = e2e_leg(args, cfg, P, proj, vw, geo, dev)
    if not args.quick and args.me_iters > 0:
        out["motion_estimation"] = motion_estimation_leg(args, cfg, P, th_true, proj, vw, dev)
    if not args.quick and args.paper_iters > 0 and rank == 0:
        out["paper_setup"] = paper_setup_leg(args, dev)
    if not args.quick and not args.no_c3 and rank == 0:
        out["precision_form"] = precision_leg(args, dev)
    if not args.quick and args.serving > 0 and rank == 0:
        out["serving"] = serving_leg(args, local)
    if ws > 1:
        torch.distributed.barrier()
    if rank == 0 and not args.no_cpu and not args.quick and ws == 1:
        out["cpu_baseline"] = cpu_baseline(cfg, P, proj, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def probe_leg(device, sms, clk):
    """Measured throughputs behind the roofline's denominators (bp_probe):
    FP32 FMA lane operations per clock per SM with scalar FFMA and with the
    packed f32x2 FMA the kernels use (a packed instruction counts two lane
    operations), against the 128 lanes per SM per clock of the ALU roofline;
    and FP32 atomic adds per second in L2, coalesced and in the data VJP's
    scattered pattern (the data VJP is the adjoint scatter of Eq. 3: four
    atomic adds per sample unless merged)."""
    from paper_2401_09283_gb300 import native
    mhz = (clk or {}).get("sm_mhz") or SM_MAX_MHZ
    vals = {k: native.probe(i, device) for i, k in enumerate(
        ("ffma_lane_ops_per_s", "ffma2_lane_ops_per_s", "red_coalesced_per_s",
         "red_scatter_2x2_per_s"))}
    per_clk = lambda v: v / (sms * mhz * 1e6)
    vals["ffma_lane_ops_per_clk_per_sm"] = per_clk(vals["ffma_lane_ops_per_s"])
    vals["ffma2_lane_ops_per_clk_per_sm"] = per_clk(vals["ffma2_lane_ops_per_s"])
    vals["roofline_lanes_per_clk_per_sm"] = 128
    vals["clock_mhz_used"] = mhz
    return vals


def motion_estimation_leg(args, cfg, P, th_true, proj, vw, dev):
    """Config-2 motion estimation through the job API (device-resident state,
    one CUDA graph per iteration): time per iteration and RPE before/after,
    with the configured sharpness loss and with total variation."""
    import torch

    import paper_2401_09283_gb300.workloads as W
    from paper_2401_09283_gb300 import bp
    from paper_2401_09283_gb300.job import MotionJob
    from paper_2401_09283_gb300.metrics import reprojection_error
    Pd = torch.as_tensor(P, device=dev)
    pts = W.rpe_points()
    true = bp.bp_compose(Pd, torch.as_tensor(th_true, device=dev)).cpu().numpy()
    out = {"iters": args.me_iters, "optimizer": "adam", "lr_mm": 0.05, "lr_rad": 5e-4,
           "rpe_before_mm": reprojection_error(P, true, pts, cfg.pitch, cfg.pitch)}
    geo = dict(vol_shape=cfg.vol_shape, spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid)
    for loss, nodes in (("sharpness", 0), ("tv", 0), ("tv", 30)):
        name = loss if nodes == 0 else "%s_akima%d" % (loss, nodes)
        job = MotionJob(proj, Pd, view_weight=vw, optimizer="adam", lr=0.05, lr_rot=5e-4,
                        max_iters=args.me_iters, loss=loss, motion_nodes=nodes, **geo)
        s = torch.cuda.current_stream(dev)
        job.step(2, s.cuda_stream)  # capture + warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        job.step(args.me_iters - 2, s.cuda_stream)
        e1.record(s)
        th, hist, it = job.motion()
        ms = e0.elapsed_time(e1) / (args.me_iters - 2)
        job.close()
        est = bp.bp_compose(Pd, torch.as_tensor(th, device=dev)).cpu().numpy()
        out[name] = {"ms_per_iter": ms, "iters_done": it,
                     "rpe_after_mm": reprojection_error(est, true, pts, cfg.pitch, cfg.pitch),
                     "loss_first": float(hist[0]), "loss_last": float(hist[it - 1])}
    out["jobs_per_s"] = 1000.0 / (out["sharpness"]["ms_per_iter"] * args.me_iters)
    return out


def serving_leg(args, device):
    """Config 5: a seeded Poisson stream of motion-estimation jobs (volumes
    128-384^3, 120-496 views, 50 iterations each) served with FP16
    projections by batches of resident jobs (two batch lanes: small and large
    jobs on priority streams),
    against the same jobs one at a time in plain FP32; jobs/s, p50/p99
    latency and the final reprojection error of each form, best of
    `serving_repeats` runs with every run's jobs/s listed, plus one run of the
    served FP16 form without batching (per-job graphs on streams)."""
    from paper_2401_09283_gb300 import serving as S
    return S.compare(n_jobs=args.serving, rate=4.0, seed=5, slots=4, opt=S.OptConfig(iters=50),
                     repeats=max(1, args.serving_repeats), device=device)


def paper_setup_leg(args, dev):
    """The paper's own motion-estimation setup (128^3 at 2 mm, 360 views over
    2 pi, 500 x 700 detector, SID 785 mm): 100 iterations of the decaying
    gradient step of Eq. 6 (t = 0.97) on the 30-node Akima spline model, as a
    job (one CUDA graph per iteration), beside Adam.  The paper's s0 = 100
    belongs to its learned metric's scale; here s0 is set so that the first
    step moves the largest translation node by a fixed length (mm) and the
    largest rotation node by the same number of degrees.
    Reports the wall time of the 100 iterations beside the paper's "under two
    minutes" on an A40 (context only: other loss, other GPU)."""
    import torch

    import paper_2401_09283_gb300.workloads as W
    from paper_2401_09283_gb300 import bp
    from paper_2401_09283_gb300.job import MotionJob
    from paper_2401_09283_gb300.metrics import reprojection_error
    cfg = W.PAPER
    P, th_true, proj = make_inputs(cfg, dev)
    V, nn, iters = cfg.views, 30, args.paper_iters
    Pd = torch.as_tensor(P, device=dev)
    vw = torch.full((V,), cfg.delta_beta, dtype=torch.float64, device=dev)
    pts = W.rpe_points()
    true = bp.bp_compose(Pd, torch.as_tensor(th_true, device=dev)).cpu().numpy()
    geo = dict(spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid)
    out = {"config": cfg.name, "iters": iters, "optimizer": "gd (Eq. 6, t = 0.97) and adam",
           "motion_model": "Akima, %d nodes" % nn,
           "rpe_before_mm": reprojection_error(P, true, pts, cfg.pitch, cfg.pitch),
           "paper_context": "under 2 min for 100 iterations on an NVIDIA A40 (learned metric)"}
    zeros = torch.zeros((nn, 6), dtype=torch.float64, device=dev)
    th0 = torch.zeros((V, 6), dtype=torch.float64, device=dev)
    # (name, loss, optimiser, first-step size in mm and deg for GD / Adam lr in mm and rad)
    runs = (("sharpness_gd", "sharpness", "gd", 0.1, 0.1),
            ("tv_gd", "tv", "gd", 0.05, 0.05),
            ("sharpness_adam", "sharpness", "adam", 0.05, 5e-4))
    for name, loss, opt, a, b in runs:
        if opt == "gd":
            vol = bp.bp_forward(proj, Pd, th0, vol_shape=cfg.vol_shape, view_weight=vw, **geo)
            L, dvol = bp.bp_sharpness(vol) if loss == "sharpness" else bp.bp_tv(vol, 1e-3)
            gth, _, _ = bp.bp_vjp(dvol, proj, Pd, th0, view_weight=vw, **geo)
            g0 = bp.bp_akima_motion_vjp(zeros, gth).abs()
            lr, lr_rot = a / float(g0[:, :3].max()), math.radians(b) / float(g0[:, 3:].max())
        else:
            lr, lr_rot = a, b
        job = MotionJob(proj, Pd, view_weight=vw, optimizer=opt, lr=lr, lr_rot=lr_rot, decay=0.97,
                        max_iters=iters, loss=loss, motion_nodes=nn, vol_shape=cfg.vol_shape,
                        **geo)
        s = torch.cuda.current_stream(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        job.step(iters, s.cuda_stream)
        th, hist, it = job.motion()
        wall = time.perf_counter() - t0
        job.close()
        est = bp.bp_compose(Pd, torch.as_tensor(th, device=dev)).cpu().numpy()
        out[name] = {"wall_s": wall, "ms_per_iter": 1e3 * wall / iters, "iters_done": it,
                     "rpe_after_mm": reprojection_error(est, true, pts, cfg.pitch, cfg.pitch),
                     "loss_first": float(hist[0]), "loss_last": float(hist[it - 1])}
    return out


def precision_leg(args, dev):
    """The precision form at full size (512^3 at 0.5 mm, 496 views,
    1240 x 960): forward and motion VJP with the projections stored in FP32,
    FP16 and BF16 (per-view scale), FP32 interpolation and accumulation.
    Throughput only; the errors against the FP64 oracle on a sampled
    sub-block come from the parity tests."""
    import torch

    import paper_2401_09283_gb300.workloads as W
    from paper_2401_09283_gb300 import bp
    cfg = W.C3
    P, th_true, proj = make_inputs(cfg, dev)
    V = cfg.views
    Pd = torch.as_tensor(P, device=dev)
    vw = torch.full((V,), cfg.delta_beta, dtype=torch.float64, device=dev)
    th = torch.as_tensor(th_true, device=dev)
    geo = dict(spacing=cfg.spacing3, origin=cfg.origin, weight="fdk", sid=cfg.sid)
    vol = torch.empty(cfg.vol_shape, dtype=torch.float32, device=dev)
    scale = proj.abs().reshape(V, -1).amax(dim=1).clamp_min(1e-30).float()
    forms = {"f32": (proj, None), "f16": ((proj / scale[:, None, None]).half(), scale),
             "bf16": ((proj / scale[:, None, None]).to(torch.bfloat16), scale)}
    out = {"config": cfg.name, "voxel_views": cfg.voxel_views}
    dvol = None
    for name, (q, sc) in forms.items():
        def fwd():
            bp.bp_forward(q, Pd, th, vol_shape=cfg.vol_shape, view_weight=vw, view_scale=sc,
                          out=vol, **geo)
        fwd()
        if dvol is None:
            _, dvol = bp.bp_sharpness(vol)
        g = torch.empty((V, 6), dtype=torch.float64, device=dev)

        def vjp():
            bp.bp_vjp(dvol, q, Pd, th, view_weight=vw, view_scale=sc, out_motion=g, **geo)
        res = {}
        for label, f, reps in (("forward", fwd, 5), ("vjp_motion", vjp, 3)):
            f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[label] = {"ms": ms, "Gupdate_per_s": cfg.voxel_views / (ms / 1e3) / 1e9}
        out[name] = res
    del forms, proj
    torch.cuda.empty_cache()
    return out


def e2e_leg(args, cfg, P, proj, vw, geo, dev):
    """Same step through the C-ABI with host buffers: projections, matrices,
    motion and optimiser state in pinned host memory, copied in by the
    library every call; the results -- loss, dL/dtheta, dL/dPhat, dL/dproj
    and the updated motion and Adam state -- copied back to the host.  Only
    the volume and dL/dvol, intermediates of the step, stay on the device."""
    import torch

    from paper_2401_09283_gb300 import bp
    V = cfg.views
    proj_h = proj.cpu().pin_memory()
    P_h = torch.as_tensor(P).pin_memory()
    vw_h = vw.cpu().pin_memory()
    th_h = torch.zeros((V, 6), dtype=torch.float64).pin_memory()
    m1_h = torch.zeros_like(th_h).pin_memory()
    m2_h = torch.zeros_like(th_h).pin_memory()
    g_th = torch.empty_like(th_h).pin_memory()
    g_P = torch.empty((V, 3, 4), dtype=torch.float64).pin_memory()
    loss_h = torch.empty((), dtype=torch.float64).pin_memory()
    vol = torch.empty(cfg.vol_shape, dtype=torch.float32, device=dev)
    dvol = torch.empty_like(vol)
    g_D = torch.empty(proj.shape, dtype=torch.float32).pin_memory()
    it = [0]

    def step():
        it[0] += 1
        bp.bp_forward(proj_h, P_h, th_h, vol_shape=cfg.vol_shape, view_weight=vw_h, out=vol, **geo)
        bp.bp_sharpness(vol, loss_out=loss_h, grad_out=dvol)
        bp.bp_vjp(dvol, proj_h, P_h, th_h, view_weight=vw_h, deriv="central", want_Phat=True,
                  want_proj=True, out_motion=g_th, out_Phat=g_P, out_proj=g_D, **geo)
        bp.bp_adam_step(th_h, g_th, m1_h, m2_h, 1e-3, it[0])

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    n = max(1, args.e2e_steps)
    t0 = time.perf_counter()
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    pb = proj.numel() * 4
    small_in = (V * 12 + V * 6 + V) * 8
    h2d = 2 * (pb + small_in) + 3 * V * 6 * 8            # fwd + vjp copies, adam state in
    # loss, dL/dtheta, dL/dPhat, dL/dproj, adam state out
    d2h = 8 + (V * 6 + V * 12) * 8 + g_D.numel() * 4 + 3 * V * 6 * 8
    return {"value": PASSES * cfg.voxel_views * n / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt / n * 1e3, "steps": n}


# ----------------------------------------------------------- oracle (CPU) leg

def oracle_sample(cfg, P, proj_np, seconds):
    """Time the FP64 oracle on a bounded sample of the workload: a 64^3
    sub-block at the volume centre and a strided subset of the views, the
    three passes of a step (forward, motion VJP, data VJP), repeated with
    more views until about `seconds` of CPU work."""
    import oracle
    rng = np.random.default_rng(0)
    vw_all = np.full(cfg.views, cfg.delta_beta)
    th = np.zeros((cfg.views, 6))
    avail = np.flatnonzero(np.abs(proj_np).reshape(cfg.views, -1).max(axis=1) > 0)
    n, nviews = 32, 8
    while True:
        n = min(n, cfg.n)
        off = (cfg.n - n) // 2
        origin = tuple(o + off * cfg.spacing for o in cfg.origin)
        delta = rng.standard_normal((n, n, n))
        sel = avail[np.linspace(0, len(avail) - 1, min(nviews, len(avail))).astype(int)]
        Ph = oracle.compose(P[sel], th[sel])
        pj = proj_np[sel].astype(np.float64)
        t0 = time.perf_counter()
        oracle.bp_forward(Ph, pj, (n, n, n), cfg.spacing3, origin, vw_all[sel],
                          oracle.WEIGHT_FDK, cfg.sid)
        gP, gD = oracle.bp_vjp(Ph, pj, delta, cfg.spacing3, origin, vw_all[sel],
                               oracle.WEIGHT_FDK, oracle.DERIV_CENTRAL, cfg.sid)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.5 or (nviews >= len(avail) and n >= cfg.n):
            break
        grow = max(2.0, seconds / max(dt, 1e-3))
        if nviews < len(avail):
            nviews = int(nviews * grow)
        else:
            n = int(n * grow ** (1.0 / 3.0)) + 1
    updates = PASSES * n ** 3 * len(sel)
    return {"value": updates / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d^3 central sub-block x %d of %d views, forward + motion VJP + data VJP "
                      "(%.1f s)" % (n, len(sel), cfg.views, dt)}


def cpu_baseline(cfg, P, proj, seconds):
    """The oracle on all host cores, plus a single-threaded sample beside it."""
    import oracle
    pj = proj.cpu().numpy()
    out = oracle_sample(cfg, P, pj, seconds)
    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        one = oracle_sample(cfg, P, pj, max(1.0, seconds / 4))
    finally:
        oracle.set_num_threads(cores)
    out["single_thread"] = {"value": one["value"], "sample": one["sample"]}
    return out


def workload_config(cfg, ws):
    """The `config` of both arms' JSON lines."""
    proj_mb = cfg.views * cfg.nv * cfg.nu * 4 / 1e6
    vol_mb = 2 * cfg.voxels * 4 / 1e6
    return {"workload": cfg.name, "volume": list(cfg.vol_shape), "voxel_mm": cfg.spacing,
            "views": cfg.views, "detector": [cfg.nv, cfg.nu], "weight": "fdk", "deriv": "central",
            "updates_per_step": "3*N^3*V (forward, motion VJP, data VJP)",
            "l2": "inputs larger than L2 (projections %.0f MB + volumes %.0f MB)" % (proj_mb, vol_mb),
            "parallelism": "replicas" if ws > 1 else "single"}


def run_reference(args):
    """The oracle as the reference arm, on the host cores of rank 0."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import torch

    import paper_2401_09283_gb300.workloads as W
    from oracle import build as OB
    OB.build_oracle()
    cfg = W.CONFIGS[args.config]
    P = W.projection_matrices(cfg)
    # the oracle's inputs: the same filtered projections, simulated on the CPU
    # for the views the sample uses (moved geometry composed by the oracle)
    import oracle
    th_true = W.motion_curves(cfg)
    Pm = oracle.compose(P, th_true)
    nsel = 64
    sel = np.linspace(0, cfg.views - 1, nsel).astype(int)
    ph = W.head_phantom(cfg)
    raw = W.line_integrals(ph, Pm[sel], cfg.nu, cfg.nv, dtype=torch.float64)
    proj_sel = W.fdk_filter(raw, cfg, views=sel).numpy().astype(np.float32)
    proj_np = np.zeros((cfg.views, cfg.nv, cfg.nu), np.float32)
    proj_np[sel] = proj_sel
    vals = []
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps))
    if args.warmup:
        oracle_sample(cfg, P, proj_np, 0.5)
    res = None
    for _ in range(args.steps):
        res = oracle_sample(cfg, P, proj_np, per_step)
        vals.append(res["value"])
    value = float(np.median(vals))
    res["value"] = value
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(cfg, ws),
           "cpu_baseline": res,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
