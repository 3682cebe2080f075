"""Serving (continuous batching with batched persistent launches): every job
gives the same result alone and in the mix, in either server form; a batch
whose members change between steps advances each member exactly as
motion_step would; admission by an HBM budget serialises jobs that do not fit
together; cancellation, a deadline, a bounded wait and malformed requests are
handled on the host."""
import dataclasses

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_09283_gb300 import native as N  # noqa: E402
from paper_2401_09283_gb300.job import Batch, MotionJob  # noqa: E402
from paper_2401_09283_gb300.serving import (OptConfig, Server, _create, make_requests,  # noqa: E402
                                            run_sequential)


def small_requests(n=4, seed=11):
    # all requests arrive at once: the first admissions fill every slot
    return make_requests(n_jobs=n, rate=1e6, seed=seed, dtype="fp16", sizes=(32, 48),
                         views=(24, 40))


@pytest.mark.parametrize("batched", [True, False])
def test_results_same_alone_and_in_the_mix(batched):
    reqs = small_requests()
    opt = OptConfig(iters=6)
    server = Server(slots=4, opt=opt, batched=batched)
    mixed = server.run(reqs)
    assert server.max_concurrent >= 2          # jobs did run concurrently
    alone = run_sequential(reqs, opt)
    for a, b in zip(mixed, alone):
        assert a.job_id == b.job_id and a.status == "ok"
        assert np.isfinite(a.theta).all()
        # deterministic kernels: identical alone and in the mix
        assert np.array_equal(a.theta, b.theta), a.job_id
        assert np.array_equal(a.loss, b.loss)


def test_batch_members_change_between_steps():
    """Three jobs in a batch whose member set changes from step to step: each
    ends bit for bit where motion_step alone takes it after the same number
    of iterations."""
    reqs = small_requests(3, seed=12)
    opt = OptConfig(iters=12)
    jobs = [_create(r, opt, 0) for r in reqs]
    batch = Batch(max_jobs=4)
    plan = [((0, 1), 3), ((0, 1, 2), 2), ((2,), 4), ((1, 2), 1), ((0,), 5)]
    total = [0, 0, 0]
    s = torch.cuda.current_stream().cuda_stream
    for members, n in plan:
        batch.set_jobs([jobs[k] for k in members])
        assert batch.size == len(members)
        batch.step(n, s)
        for k in members:
            total[k] += n
    got = [j.motion() for j in jobs]
    batch.close()
    for k, r in enumerate(reqs):
        assert jobs[k].iterations_queued == total[k]
        ref = _create(r, opt, 0)
        ref.step(total[k])
        th, hist, it = ref.motion()
        assert it == total[k] == got[k][2]
        assert np.array_equal(got[k][0], th), k
        assert np.array_equal(got[k][1], hist), k
        ref.close()
        jobs[k].close()


def test_batch_rejects_mixed_or_unsupported_members():
    r16 = small_requests(1, seed=13)[0]
    r32 = make_requests(n_jobs=1, rate=50.0, seed=13, dtype="fp32", sizes=(32,), views=(24,))[0]
    opt = OptConfig(iters=2)
    a, b = _create(r16, opt, 0), _create(r32, opt, 0)
    batch = Batch(max_jobs=2)
    with pytest.raises(N.BPError, match="BP_ERR_INVALID_ARG"):
        batch.set_jobs([a, b])                 # FP16 and FP32 members
    with pytest.raises(N.BPError, match="BP_ERR_INVALID_ARG"):
        batch.set_jobs([a, a])                 # listed twice
    cfg = r16.cfg
    spl = MotionJob(r16.proj, torch.as_tensor(r16.P), vol_shape=cfg.vol_shape,
                    spacing=cfg.spacing3, origin=cfg.origin, sid=cfg.sid, view_scale=r16.scale,
                    motion_nodes=4, max_iters=2)
    with pytest.raises(N.BPError, match="BP_ERR_UNSUPPORTED"):
        batch.set_jobs([spl])                  # spline motion model
    batch.set_jobs([a])
    with pytest.raises(N.BPError, match="BP_ERR_INVALID_ARG"):
        a.step(1)                              # a member is advanced by its batch only
    batch.close()
    for j in (a, b, spl):
        j.close()


def test_cancelled_job_stops_and_leaves_the_batch():
    reqs = small_requests(2, seed=14)
    opt = OptConfig(iters=8)
    a, b = (_create(r, opt, 0) for r in reqs)
    batch = Batch(max_jobs=2)
    batch.set_jobs([a, b])
    batch.step(2)
    a.cancel()
    batch.step(3)                              # a is dropped before this step
    assert batch.size == 1
    assert a.iterations_queued == 2 and b.iterations_queued == 5
    with pytest.raises(N.BPError, match="BP_ERR_CANCELLED"):
        batch.set_jobs([a, b])
    with pytest.raises(N.BPError, match="BP_ERR_CANCELLED"):
        a.step(1)
    _, _, it = a.motion()                      # its state stays readable
    assert it == 2
    batch.close()
    a.close()
    b.close()


def test_wait_times_out_on_a_slow_job():
    """A job given far more queued work than the wait allows: bp_job_wait
    returns BP_ERR_TIMEOUT (nothing is stopped), then completes."""
    req = make_requests(n_jobs=1, rate=50.0, seed=15, dtype="fp16", sizes=(128,), views=(248,))[0]
    opt = OptConfig(iters=400)
    job = _create(req, opt, 0)
    job.step(400)
    assert job.wait(1.0) is False
    assert job.wait(-1.0) is True
    _, _, it = job.motion()
    assert it == 400
    job.close()


def test_server_rejects_malformed_requests_cancels_and_times_out():
    reqs = small_requests(4, seed=16)
    bad = dataclasses.replace(reqs[1], proj=reqs[1].proj[:0])   # no views: malformed
    reqs = [reqs[0], bad, reqs[2], reqs[3]]
    opt = OptConfig(iters=6)
    server = Server(slots=2, opt=opt)
    server.cancel(reqs[2].job_id)
    res = {r.job_id: r for r in server.run(reqs)}
    assert res[bad.job_id].status.startswith("rejected") and "BP_ERR_INVALID_ARG" in res[bad.job_id].status
    assert res[reqs[2].job_id].status == "cancelled"
    assert res[reqs[0].job_id].status == "ok" and res[reqs[3].job_id].status == "ok"
    ref = run_sequential([reqs[0], reqs[3]], opt)
    assert np.array_equal(res[reqs[0].job_id].theta, ref[0].theta)
    late = Server(slots=2, opt=OptConfig(iters=2000), deadline_s=0.0)
    out = late.run(small_requests(2, seed=17))
    assert all(r.status == "timeout" for r in out)


def test_admission_by_hbm_budget():
    reqs = small_requests()
    opt = OptConfig(iters=4)
    sizes = [MotionJob.bytes_for(r.proj.shape, 1, r.cfg.vol_shape, "central", opt.iters)
             for r in reqs]
    budget = 2 * min(sizes) - 1       # any job fits alone, no two fit together
    assert budget >= max(sizes)
    server = Server(slots=4, opt=opt, hbm_budget=budget)
    res = server.run(reqs)
    assert server.max_concurrent == 1
    assert len(res) == len(reqs)
    ref = Server(slots=4, opt=opt).run(reqs)
    for a, b in zip(res, ref):
        assert np.array_equal(a.theta, b.theta)
