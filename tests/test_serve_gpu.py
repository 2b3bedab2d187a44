"""Serving pattern: continuous batching of render requests of different
scenes and resolutions.  Each result is the same alone and in the mix
(bit-identical: the batched forward runs the same per-tile computation, and
a batch of one request runs the single-view calls)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402
from paper_2505_05587_gb300 import serve as SV  # noqa: E402

RES = [(64, 48), (96, 64), (128, 96), (80, 80)]


def _setup(n_jobs=40, rate=2000.0):
    scenes = [B.GaussianTensors.from_scene(synth.cluster_scene(20 + k, n, 3))
              for k, n in enumerate((3000, 8000, 20000))]
    reqs = synth.request_stream(7, n_jobs, rate, len(scenes), RES)
    jobs = [SV.Job(k, r.arrival_s - reqs[0].arrival_s, r.scene, r.camera) for k, r in enumerate(reqs)]
    return scenes, jobs


def _alone(scenes, job, st):
    g = scenes[job.scene]
    vb = PL.ViewBuffers.alloc(g.n, job.cam, st)
    PL.render(g, vb)
    torch.cuda.synchronize()
    return vb.image


@pytest.mark.parametrize("realtime", [False, True])
def test_each_result_same_alone_and_in_the_mix(realtime):
    scenes, jobs = _setup()
    st = synth.Settings()
    server = SV.RenderServer(scenes, st, max_batch=6, n_slots=3, keep_images=True)
    out = server.run(jobs, realtime=realtime)
    assert out["requests"] == len(jobs) and out["batches"] < len(jobs)
    for j in jobs:
        assert torch.equal(server.images[j.idx], _alone(scenes, j, st)), j.idx
    assert out["p99_ms"] >= out["p50_ms"] > 0
    # batches of one request take the single-view calls, larger ones the batched pass
    assert out["batched_requests"] > out.get("single_view_batches", 0)
    if realtime:                                  # requests arriving one at a time: both paths ran
        assert out.get("single_view_batches", 0) > 0


def test_admission_waits_for_memory_and_completes():
    scenes, jobs = _setup(24)
    st = synth.Settings()
    one = SV.RenderServer(scenes, st, max_batch=1, n_slots=1)
    need = max(one._batch_bytes([j], one._capacity([j])) for j in jobs)
    server = SV.RenderServer(scenes, st, max_batch=4, n_slots=4, hbm_budget=int(1.5 * need), keep_images=True)
    out = server.run(jobs, realtime=False)
    assert out["requests"] == len(jobs)
    assert out.get("admission_waits", 0) > 0
    for j in jobs[:6]:
        assert torch.equal(server.images[j.idx], _alone(scenes, j, st))


def test_capacity_underestimate_is_rerun_not_truncated():
    scenes, jobs = _setup(8)
    st = synth.Settings()
    server = SV.RenderServer(scenes, st, max_batch=4, n_slots=2, keep_images=True)
    for j in jobs:
        server.m_est[(j.scene, j.cam.width, j.cam.height)] = 16     # far too small
    out = server.run(jobs, realtime=False)
    assert out.get("reruns", 0) > 0
    for j in jobs:
        assert torch.equal(server.images[j.idx], _alone(scenes, j, st))
