"""Serving: continuous batching of motion-estimation jobs on one GPU.

Requests arrive over time (Poisson arrivals).  A request is admitted as soon
as a slot is free and its device memory fits the HBM budget (the job API's
admission check); admitted jobs keep all their state on the device and are
advanced together as one batch (bp_batch_step): compose, backprojection,
loss, reduction and update are each a single launch over the work items of
all resident jobs (the backprojection persistent), and the jobs' motion VJPs
run as parallel branches of the same graph.
A finished job is read back and freed with the stream-ordered allocator (no
device-wide synchronisation), and the next waiting request takes its slot.

The baseline serves the same requests one at a time, in arrival order, each
alone on the GPU, with FP32 projections.

The default loss is the smoothed TV of the paper's comparison (Sec. IV-A):
on these phantoms the sharpness loss sharpens the volume without lowering the
reprojection error, so only TV gives served results whose accuracy can be
compared.

Usage: python -m paper_2401_09283_gb300.serving [--jobs 64] [--rate 4] ...
prints one JSON line with jobs/s, p50/p99 latency and the final reprojection
error of the served and the one-at-a-time forms.
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
from .job import Batch, MotionJob
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
    theta: Optional[np.ndarray]
    loss: Optional[np.ndarray]
    rpe: float
    status: str = "ok"

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
    loss: str = "tv"
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
    admission by free HBM (or an explicit budget), FIFO.

    batched=True (the serving form): the resident jobs are the members of
    `lanes` bp_batches -- with two lanes, jobs of at most `small_voxel_views`
    voxel-views per iteration in a batch on a high-priority stream, larger ones
    in a batch on a low-priority stream, so that small jobs do not advance in
    lockstep with large ones and the two batches fill each other's kernel
    tails.  In a batch every stage of an iteration but the VJP is ONE launch
    over the work items of all its members, the VJPs run as parallel graph
    branches (bp_batch_step replays one captured graph).  A batch advances in
    steps of at most `chunk` iterations, never past a member's remaining
    iterations; a job that finishes leaves its batch and the next waiting
    request takes its slot at the following step.  Two steps per batch are
    kept queued on the device, so admissions and read-backs on the host
    overlap the GPU's work.

    batched=False: each resident job replays its own iteration graph
    (motion_step) in chunks on a priority stream by age (oldest first), so the
    jobs' kernels overlap only through the block scheduler.

    Failure handling (all on the host): a request whose job cannot be created
    (malformed descriptor) is rejected with its error; a job resident longer
    than `deadline_s` is cancelled and reported as timed out; `cancel(job_id)`
    cancels a waiting or resident job.  Every result carries its status."""

    def __init__(self, device=0, slots=4, opt: OptConfig = OptConfig(), hbm_budget=0, chunk=5,
                 batched=True, deadline_s=None, lanes=2, small_voxel_views=2 ** 31):
        self.device = device
        self.slots = slots
        self.lanes = lanes
        self.small_voxel_views = small_voxel_views
        self.opt = opt
        self.hbm_budget = hbm_budget
        self.chunk = chunk
        self.batched = batched
        self.deadline_s = deadline_s
        self.max_resident_bytes = 0
        self.max_concurrent = 0
        self.steps = 0
        self._cancel = set()

    def cancel(self, job_id):
        """Cancel a waiting or resident job (takes effect at the next step)."""
        self._cancel.add(job_id)

    def _streams(self, dev):
        # lower numbers are higher priorities: rank 0 gets the greatest
        least, greatest = torch.cuda.Stream.priority_range()
        return [torch.cuda.Stream(dev, priority=min(greatest + k, least))
                for k in range(self.slots)]

    def _admit(self, waiting, active, results, t0):
        """FIFO admission while a slot is free and the job fits in memory."""
        changed = False
        while waiting and len(active) < self.slots:
            req = waiting[0]
            if req.job_id in self._cancel:
                waiting.popleft()
                now = time.perf_counter() - t0
                results.append(Result(req.job_id, req.arrival, now, now, None, None, float("nan"),
                                      "cancelled"))
                continue
            try:
                job = _create(req, self.opt, self.device)
            except (RuntimeError, TypeError, ValueError) as e:
                if "BP_ERR_OOM" in str(e):
                    break
                waiting.popleft()
                now = time.perf_counter() - t0
                results.append(Result(req.job_id, req.arrival, now, now, None, None, float("nan"),
                                      "rejected: %s" % e))
                continue
            waiting.popleft()
            active.append(dict(req=req, job=job, left=self.opt.iters, events=[],
                               admitted=time.perf_counter() - t0, status="ok"))
            changed = True
            resident = sum(a["job"].nbytes for a in active)
            self.max_resident_bytes = max(self.max_resident_bytes, resident)
            self.max_concurrent = max(self.max_concurrent, len(active))
        return changed

    def _finish(self, a, results, t0):
        th, hist, _ = a["job"].motion()
        fin = time.perf_counter() - t0
        a["job"].close()
        results.append(Result(a["req"].job_id, a["req"].arrival, a["admitted"], fin, th, hist,
                              float("nan"), a["status"]))

    def _expire(self, active, t0):
        """Cancel resident jobs past their deadline or asked to stop."""
        now = time.perf_counter() - t0
        for a in active:
            if a["left"] == 0:
                continue
            late = self.deadline_s is not None and now - a["admitted"] > self.deadline_s
            if late or a["req"].job_id in self._cancel:
                a["job"].cancel()
                a["left"] = 0
                a["status"] = "timeout" if late else "cancelled"

    def run(self, requests: List[Request]) -> List[Result]:
        dev = torch.device("cuda", self.device)
        torch.cuda.set_device(dev)
        ctx = N.context(self.device)
        N.check("bp_ctx_set_hbm_budget", N.lib().bp_ctx_set_hbm_budget(ctx, int(self.hbm_budget)),
                ctx)
        try:
            if self.batched:
                results = self._run_batched(requests, dev)
            else:
                results = self._run_streams(requests, dev)
        finally:
            N.lib().bp_ctx_set_hbm_budget(ctx, 0)
        by_id = {r.job_id: r for r in requests}
        for r in results:
            if r.theta is not None:
                r.rpe = _rpe(by_id[r.job_id], r.theta, self.device)
        return sorted(results, key=lambda r: r.job_id)

    def _lane_of(self, req):
        """Batch lane of a request: 0 (high-priority stream) for jobs of at
        most `small_voxel_views` voxel-views per iteration, else 1."""
        if self.lanes < 2:
            return 0
        return 0 if req.cfg.voxel_views <= self.small_voxel_views else 1

    def _run_batched(self, requests, dev):
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        active = []   # admission order: dicts req, job, left, admitted, status, lane
        done = []     # finished jobs whose last iterations may still be queued
        results = []
        least, greatest = torch.cuda.Stream.priority_range()
        lanes = [dict(batch=Batch(max_jobs=self.slots, device=self.device),
                      stream=torch.cuda.Stream(dev, priority=min(greatest + k, least)),
                      inflight=collections.deque(), members=[])
                 for k in range(max(1, self.lanes))]
        t0 = time.perf_counter()
        try:
            while pending or waiting or active or done:
                now = time.perf_counter() - t0
                while pending and pending[0].arrival <= now:
                    waiting.append(pending.popleft())
                self._expire(active, t0)
                # finished (or cancelled) jobs leave their batch and free their slot
                done.extend(a for a in active if a["left"] == 0)
                active = [a for a in active if a["left"] > 0]
                n_before = len(active)
                self._admit(waiting, active, results, t0)
                for a in active[n_before:]:
                    a["lane"] = self._lane_of(a["req"])
                progressed = False
                for k, L in enumerate(lanes):
                    while L["inflight"] and L["inflight"][0].query():
                        L["inflight"].popleft()
                    running = [a for a in active if a["lane"] == k]
                    jobs = [a["job"] for a in running]
                    if jobs != L["members"]:
                        L["members"] = jobs
                        L["batch"].set_jobs(jobs)
                    # keep two steps of each lane queued on the device, so
                    # admissions and read-backs on the host overlap its work
                    if running and len(L["inflight"]) < 2:
                        n = min(self.chunk, min(a["left"] for a in running))
                        L["batch"].step(n, L["stream"].cuda_stream)
                        self.steps += 1
                        ev = torch.cuda.Event()
                        ev.record(L["stream"])
                        L["inflight"].append(ev)
                        for a in running:
                            a["left"] -= n
                        progressed = True
                # read back the jobs whose last step has run
                for a in [a for a in done if a["job"].wait(0.0)]:
                    done.remove(a)
                    self._finish(a, results, t0)
                    progressed = True
                if progressed:
                    continue
                if not active and not done and not waiting and pending:
                    time.sleep(max(0.0, min(0.005, pending[0].arrival - (time.perf_counter() - t0))))
                elif not active and done and not waiting:
                    for a in list(done):
                        a["job"].wait(-1.0)
                        self._finish(a, results, t0)
                    done.clear()
                else:
                    time.sleep(0.0002)
        finally:
            for L in lanes:
                L["batch"].close()
        return results

    def _run_streams(self, requests, dev):
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
            self._expire(active, t0)
            self._admit(waiting, active, results, t0)
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
                    active.remove(a)
                    self._finish(a, results, t0)
                    progressed = True
            if not progressed:
                if not active and not waiting and pending:
                    time.sleep(max(0.0, min(0.005, pending[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        return results


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
        results.append(Result(req.job_id, req.arrival, adm, fin, th, hist, float("nan"), "ok"))
    for r, req in zip(results, sorted(requests, key=lambda r: r.arrival)):
        r.rpe = _rpe(req, r.theta, device)
    return sorted(results, key=lambda r: r.job_id)


def _rpe_initial(req: Request) -> float:
    return reprojection_error(req.P, _moved(req), W.rpe_points(), req.cfg.pitch, req.cfg.pitch)


def _moved(req: Request):
    dev = torch.device("cuda", torch.cuda.current_device())
    Pd = torch.as_tensor(req.P, device=dev)
    return bp.bp_compose(Pd, torch.as_tensor(req.theta_true, device=dev)).cpu().numpy()


def compare(n_jobs=16, rate=4.0, seed=5, slots=4, opt: OptConfig = OptConfig(), repeats=1,
            sizes=(128, 192, 256, 384), views=(120, 248, 496), device=0, streams_form=True):
    """The served FP16 form (batched launches in two lanes) against the same
    requests served one at a time in plain FP32, `repeats` runs of each (the
    spread of jobs/s), plus one run of the served FP16 form without batching
    (per-job graphs on streams) when streams_form is set."""
    req16 = make_requests(n_jobs, rate, seed, "fp16", sizes, views, device=device)
    req32 = make_requests(n_jobs, rate, seed, "fp32", sizes, views, device=device)
    out = {"config": {"jobs": n_jobs, "rate_per_s": rate, "slots": slots, "iters": opt.iters,
                      "loss": opt.loss, "lr_mm": opt.lr, "lr_rad": opt.lr_rot, "sizes": list(sizes),
                      "views": list(views), "repeats": repeats}}
    runs16, runs32 = [], []
    for _ in range(repeats):
        srv = Server(device=device, slots=slots, opt=opt, batched=True)
        runs16.append(summarize(srv.run(req16), req16, srv))
        runs32.append(summarize(run_sequential(req32, opt, device=device), req32, None))
    for name, runs in (("served_fp16_batched", runs16), ("sequential_fp32", runs32)):
        jps = [r["jobs_per_s"] for r in runs]
        best = dict(runs[int(np.argmax(jps))])
        best["jobs_per_s_runs"] = jps
        out[name] = best
    if streams_form:
        srv = Server(device=device, slots=slots, opt=opt, batched=False)
        out["served_fp16_streams"] = summarize(srv.run(req16), req16, srv)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--loss", default="tv", choices=["tv", "sharpness"])
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--sizes", default="128,192,256,384")
    ap.add_argument("--views", default="120,248,496")
    args = ap.parse_args()
    sizes = tuple(int(x) for x in args.sizes.split(","))
    views = tuple(int(x) for x in args.views.split(","))
    opt = OptConfig(iters=args.iters, loss=args.loss)
    print(json.dumps(compare(args.jobs, args.rate, args.seed, args.slots, opt, args.repeats,
                             sizes, views)))


def summarize(results, requests, server):
    """jobs/s and latency over the completed jobs; other outcomes counted."""
    ok = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    first = min(r.arrival for r in requests)
    last = max(r.finished for r in results)
    out = {"jobs": len(ok), "jobs_per_s": len(ok) / max(last - first, 1e-9),
           "makespan_s": last - first, "latency_p50_s": float(np.percentile(lat, 50)),
           "latency_p99_s": float(np.percentile(lat, 99)), "latency_mean_s": float(lat.mean()),
           "rpe_mean_mm": float(np.mean([r.rpe for r in ok])) if ok else float("nan"),
           "rpe_initial_mean_mm": float(np.mean([_rpe_initial(q) for q in requests]))}
    other = collections.Counter(r.status.split(":")[0] for r in results if r.status != "ok")
    if other:
        out["not_completed"] = dict(other)
    if server is not None:
        out["max_concurrent_jobs"] = server.max_concurrent
        out["max_resident_gb"] = server.max_resident_bytes / 1e9
        out["form"] = ("batched launches, %d batch lane(s) on priority streams" % server.lanes
                       if server.batched else "per-job graphs on streams")
    return out


if __name__ == "__main__":
    main()
