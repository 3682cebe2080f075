"""Serving: continuous batching of motion-estimation jobs on one GPU.

Requests arrive over time (Poisson arrivals).  A request is admitted as soon
as a slot is free and its device memory fits the HBM budget (the job API's
admission check); admitted jobs keep all their state on the device and
replay their captured iteration graph in chunks on priority streams (oldest
job first, the others back-filling the SMs it leaves idle), so the kernels of
concurrent jobs overlap on the GPU.  A finished job is read
back and freed with the stream-ordered allocator (no device-wide
synchronisation), and the next waiting request takes its slot.

The baseline serves the same requests one at a time, in arrival order, each
alone on the GPU.

Usage: python -m paper_2401_09283_gb300.serving [--jobs 64] [--rate 4] ...
prints one JSON line with jobs/s and p50/p99 latency of both forms.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import json
import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import bp
from . import native as N
from . import workloads as W
from .job import MotionJob
from .metrics import reprojection_error


@dataclasses.dataclass
class Request:
    job_id: int
    arrival: float            # seconds after the start of the stream
    cfg: W.ScanConfig
    proj: torch.Tensor        # pinned host tensor (V, nv, nu), float16 or float32
    scale: Optional[torch.Tensor]
    P: np.ndarray
    theta_true: np.ndarray


@dataclasses.dataclass
class Result:
    job_id: int
    arrival: float
    admitted: float
    finished: float
    theta: np.ndarray
    loss: np.ndarray
    rpe: float

    @property
    def latency(self):
        return self.finished - self.arrival


def make_requests(n_jobs=64, rate=4.0, seed=5, dtype="fp16", sizes=(128, 192, 256, 384),
                  views=(120, 248, 496), device=0) -> List[Request]:
    """Seeded job stream: Poisson arrivals at `rate` jobs/s, volume edge and
    view count drawn uniformly, scans simulated on the device (closed-form
    ellipsoid line integrals through the moved geometry, 1 % noise) and
    filtered by the library (bp_fdk_filter), kept in pinned host memory as
    the client's data."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    arrivals -= arrivals[0]
    out = []
    dev = torch.device("cuda", device)
    for i in range(n_jobs):
        n = int(rng.choice(sizes))
        v = int(rng.choice(views))
        cfg = W.serving_job_config(i, n, v)
        P = W.projection_matrices(cfg)
        th = W.motion_curves(cfg)
        Pm = bp.bp_compose(torch.as_tensor(P, device=dev), torch.as_tensor(th, device=dev))
        raw = W.line_integrals(W.head_phantom(cfg), Pm.cpu().numpy(), cfg.nu, cfg.nv, device=dev,
                               dtype=torch.float32, views_per_chunk=32)
        raw = W.add_noise(raw, cfg.noise, cfg.phantom_seed + 100)
        q = bp.bp_fdk_filter(raw.float().contiguous(), pitch=cfg.pitch, sid=cfg.sid, sdd=cfg.sdd,
                             arc=math.radians(cfg.arc_deg))
        if dtype == "fp16":
            scale = q.abs().reshape(v, -1).amax(dim=1).clamp_min(1e-30)
            stored = (q / scale[:, None, None]).half()
            out.append(Request(i, float(arrivals[i]), cfg, stored.cpu().pin_memory(),
                               scale.cpu().pin_memory(), P, th))
        else:
            out.append(Request(i, float(arrivals[i]), cfg, q.cpu().pin_memory(), None, P, th))
        del raw, q
    torch.cuda.synchronize(dev)
    return out


@dataclasses.dataclass
class OptConfig:
    iters: int = 50
    lr: float = 0.05
    lr_rot: float = 5e-4
    loss: str = "sharpness"
    tv_eps: float = 1e-3


def _create(req: Request, opt: OptConfig, device):
    cfg = req.cfg
    vw = torch.full((cfg.views,), cfg.delta_beta, dtype=torch.float64)
    return MotionJob(req.proj, torch.as_tensor(req.P), vol_shape=cfg.vol_shape,
                     spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid, view_weight=vw,
                     weight="fdk", deriv="central", optimizer="adam", lr=opt.lr,
                     lr_rot=opt.lr_rot, max_iters=opt.iters, view_scale=req.scale, device=device,
                     loss=opt.loss, tv_eps=opt.tv_eps)


def _rpe(req: Request, theta: np.ndarray, device) -> float:
    cfg = req.cfg
    dev = torch.device("cuda", device)
    Pd = torch.as_tensor(req.P, device=dev)
    est = bp.bp_compose(Pd, torch.as_tensor(theta, device=dev)).cpu().numpy()
    true = bp.bp_compose(Pd, torch.as_tensor(req.theta_true, device=dev)).cpu().numpy()
    return reprojection_error(est, true, W.rpe_points(), cfg.pitch, cfg.pitch)


class Server:
    """Continuous-batching server: up to `slots` jobs resident at once,
    admission by free HBM (or an explicit budget), FIFO with back-fill.

    Every resident job advances in chunks of `chunk` iterations.  Chunks go to
    the stream of the job's rank among the resident jobs: the oldest job on
    the highest-priority stream, the next on the next one, and so on.  The
    block scheduler then serves the oldest job first and hands the other jobs
    only the SMs it leaves idle (the tails of its kernels), so the head job
    runs almost as if alone while the others fill its gaps.  When the head
    finishes, the next job's later chunks move to the top stream (motion_step
    orders a job's work across streams)."""

    def __init__(self, device=0, slots=4, opt: OptConfig = OptConfig(), hbm_budget=0, chunk=5):
        self.device = device
        self.slots = slots
        self.opt = opt
        self.hbm_budget = hbm_budget
        self.chunk = chunk
        self.max_resident_bytes = 0
        self.max_concurrent = 0

    def _streams(self, dev):
        # lower numbers are higher priorities: rank 0 gets the greatest
        least, greatest = torch.cuda.Stream.priority_range()
        return [torch.cuda.Stream(dev, priority=min(greatest + k, least))
                for k in range(self.slots)]

    def run(self, requests: List[Request]) -> List[Result]:
        dev = torch.device("cuda", self.device)
        torch.cuda.set_device(dev)
        ctx = N.context(self.device)
        N.check("bp_ctx_set_hbm_budget", N.lib().bp_ctx_set_hbm_budget(ctx, int(self.hbm_budget)),
                ctx)
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = []  # admission order: dicts req, job, left, events, admitted
        results = []
        streams = self._streams(dev)
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission: FIFO while a slot is free and the job fits in memory
            while waiting and len(active) < self.slots:
                try:
                    job = _create(waiting[0], self.opt, self.device)
                except RuntimeError as e:
                    if "BP_ERR_OOM" in str(e):
                        break
                    raise
                req = waiting.popleft()
                active.append(dict(req=req, job=job, left=self.opt.iters, events=[],
                                   admitted=time.perf_counter() - t0))
                resident = sum(a["job"].nbytes for a in active)
                self.max_resident_bytes = max(self.max_resident_bytes, resident)
                self.max_concurrent = max(self.max_concurrent, len(active))
            progressed = False
            for rank, a in enumerate(list(active)):
                a["events"] = [ev for ev in a["events"] if not ev.query()]
                # keep two chunks queued per job, on the stream of its rank
                while a["left"] > 0 and len(a["events"]) < 2:
                    s = streams[rank]
                    n = min(self.chunk, a["left"])
                    a["job"].step(n, s.cuda_stream)
                    ev = torch.cuda.Event()
                    ev.record(s)
                    a["events"].append(ev)
                    a["left"] -= n
                    progressed = True
                if a["left"] == 0 and not a["events"]:
                    th, hist, _ = a["job"].motion()
                    fin = time.perf_counter() - t0
                    a["job"].close()
                    active.remove(a)
                    results.append(Result(a["req"].job_id, a["req"].arrival, a["admitted"], fin,
                                          th, hist, float("nan")))
                    progressed = True
            if not progressed:
                if not active and not waiting and pending:
                    time.sleep(max(0.0, min(0.005, pending[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        N.lib().bp_ctx_set_hbm_budget(ctx, 0)
        by_id = {r.job_id: r for r in requests}
        for r in results:
            r.rpe = _rpe(by_id[r.job_id], r.theta, self.device)
        return sorted(results, key=lambda r: r.job_id)


def run_sequential(requests: List[Request], opt: OptConfig = OptConfig(), device=0) -> List[Result]:
    """One job at a time in arrival order, each alone on the GPU."""
    dev = torch.device("cuda", device)
    torch.cuda.set_device(dev)
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        adm = time.perf_counter() - t0
        job = _create(req, opt, device)
        job.step(opt.iters)
        th, hist, _ = job.motion()
        fin = time.perf_counter() - t0
        job.close()
        results.append(Result(req.job_id, req.arrival, adm, fin, th, hist, float("nan")))
    for r, req in zip(results, sorted(requests, key=lambda r: r.arrival)):
        r.rpe = _rpe(req, r.theta, device)
    return sorted(results, key=lambda r: r.job_id)


def _rpe_initial(req: Request) -> float:
    return reprojection_error(req.P, _moved(req), W.rpe_points(), req.cfg.pitch, req.cfg.pitch)


def _moved(req: Request):
    dev = torch.device("cuda", torch.cuda.current_device())
    Pd = torch.as_tensor(req.P, device=dev)
    return bp.bp_compose(Pd, torch.as_tensor(req.theta_true, device=dev)).cpu().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--loss", default="sharpness")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--sizes", default="128,192,256,384")
    ap.add_argument("--views", default="120,248,496")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--served-dtype", default="fp16", choices=["fp16", "fp32"])
    args = ap.parse_args()
    sizes = tuple(int(x) for x in args.sizes.split(","))
    views = tuple(int(x) for x in args.views.split(","))
    opt = OptConfig(iters=args.iters, loss=args.loss)
    req16 = make_requests(args.jobs, args.rate, args.seed, args.served_dtype, sizes, views)
    served = Server(slots=args.slots, opt=opt)
    res16 = served.run(req16)
    out = {"served_" + args.served_dtype: summarize(res16, req16, served)}
    if not args.no_baseline:
        req32 = make_requests(args.jobs, args.rate, args.seed, "fp32", sizes, views)
        res32 = run_sequential(req32, opt)
        out["sequential_fp32"] = summarize(res32, req32, None)
    out["config"] = {"jobs": args.jobs, "rate_per_s": args.rate, "slots": args.slots,
                     "iters": args.iters, "loss": args.loss, "sizes": sizes, "views": views}
    print(json.dumps(out))


def summarize(results, requests, server):
    lat = np.array([r.latency for r in results])
    first = min(r.arrival for r in requests)
    last = max(r.finished for r in results)
    out = {"jobs": len(results), "jobs_per_s": len(results) / (last - first),
           "makespan_s": last - first, "latency_p50_s": float(np.percentile(lat, 50)),
           "latency_p99_s": float(np.percentile(lat, 99)), "latency_mean_s": float(lat.mean()),
           "rpe_mean_mm": float(np.mean([r.rpe for r in results])),
           "rpe_initial_mean_mm": float(np.mean([_rpe_initial(q) for q in requests]))}
    if server is not None:
        out["max_concurrent_jobs"] = server.max_concurrent
        out["max_resident_gb"] = server.max_resident_bytes / 1e9
    return out


if __name__ == "__main__":
    main()
