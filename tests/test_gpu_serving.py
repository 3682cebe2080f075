"""Serving (continuous batching): every job gives the same result alone and
in the mix, and admission by an HBM budget serialises jobs that do not fit
together."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2401_09283_gb300.job import MotionJob  # noqa: E402
from paper_2401_09283_gb300.serving import OptConfig, Server, make_requests, run_sequential  # noqa: E402


def small_requests():
    return make_requests(n_jobs=4, rate=50.0, seed=11, dtype="fp16", sizes=(32, 48),
                         views=(24, 40))


def test_results_same_alone_and_in_the_mix():
    reqs = small_requests()
    opt = OptConfig(iters=6)
    server = Server(slots=4, opt=opt)
    mixed = server.run(reqs)
    assert server.max_concurrent >= 2          # jobs did run concurrently
    alone = run_sequential(reqs, opt)
    for a, b in zip(mixed, alone):
        assert a.job_id == b.job_id
        assert np.isfinite(a.theta).all()
        # deterministic kernels: identical alone and in the mix
        assert np.array_equal(a.theta, b.theta), a.job_id
        assert np.array_equal(a.loss, b.loss)


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
