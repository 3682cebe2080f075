"""Host-side logic of the serving layer (no GPU): the batch lanes."""
import types

from paper_2401_09283_gb300 import serving as S
from paper_2401_09283_gb300 import workloads as W


def _req(job_id, n, views, arrival=0.0):
    return types.SimpleNamespace(job_id=job_id, arrival=arrival,
                                 cfg=W.serving_job_config(job_id, n, views))


def test_two_lanes_split_jobs_by_iteration_size():
    srv = S.Server(device=0, slots=4, batched=True)
    small = [_req(0, 128, 496), _req(1, 192, 248), _req(2, 256, 120)]
    large = [_req(3, 256, 248), _req(4, 384, 120), _req(5, 384, 496)]
    assert [srv._lane_of(r) for r in small] == [0, 0, 0]
    assert [srv._lane_of(r) for r in large] == [1, 1, 1]
    # the threshold is the request's voxel-views per iteration
    for r in small:
        assert r.cfg.voxel_views <= srv.small_voxel_views
    for r in large:
        assert r.cfg.voxel_views > srv.small_voxel_views


def test_one_lane_puts_every_job_in_one_batch():
    srv = S.Server(device=0, slots=4, batched=True, lanes=1)
    assert {srv._lane_of(_req(i, n, v)) for i, (n, v) in enumerate(
        ((128, 120), (256, 248), (384, 496)))} == {0}
