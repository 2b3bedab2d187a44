"""Host logic of the render server's continuous batching, on the CPU: the
scheduler runs against a fake launcher (no GPU), so the tests can make a
batch overflow its instance capacity, hold completions back, or shrink the
memory budget, and check what the scheduler does about it: batch sizes, the
admission waits, the reruns with grown estimates, and a latency for every
request."""
import collections
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2505_05587_gb300 import serve as SV  # noqa: E402


class _Event:
    def __init__(self, clock, done_after):
        self.clock, self.done_after = clock, done_after

    def query(self):
        self.clock[0] += 1
        return self.clock[0] >= self.done_after


def _server(n_scenes=3, max_batch=3, n_slots=2, budget=10_000, bytes_per_job=1_000, true_M=None, delay=2):
    srv = SV.RenderServer.__new__(SV.RenderServer)
    srv.scenes = [types.SimpleNamespace(n=1_000 * (k + 1)) for k in range(n_scenes)]
    srv.st = None
    srv.single_path = True
    srv.max_batch, srv.n_slots, srv.batch_depth = max_batch, n_slots, 0
    srv.keep_images = False
    srv.budget = budget
    srv.in_use = 0
    srv.m_est = {}
    srv.images = {}
    srv.stats = collections.Counter()
    clock = [0]
    launched = []

    def batch_bytes(jobs, capacity):
        return bytes_per_job * len(jobs)

    def launch(jobs, slot, capacity=None):
        capacity = capacity or srv._capacity(jobs)
        nbytes = srv._batch_bytes(jobs, capacity)
        srv.in_use += nbytes
        srv.stats["batches"] += 1
        srv.stats["batched_requests"] += len(jobs)
        M = sum((true_M or {}).get(j.scene, 10) for j in jobs)
        launched.append((tuple(j.idx for j in jobs), slot, capacity, M))
        host = types.SimpleNamespace(item=lambda M=M: M)
        return SV._Batch(list(jobs), slot, _Event(clock, clock[0] + delay), None, None, None, host, capacity, nbytes,
                         [0] * (len(jobs) + 1))

    srv._batch_bytes = batch_bytes
    srv._launch = launch
    return srv, launched


def _jobs(n, n_scenes=3):
    cam = types.SimpleNamespace(width=64, height=48)
    return [SV.Job(k, 0.0, k % n_scenes, cam) for k in range(n)]


@pytest.fixture(autouse=True)
def _no_device_sync(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def test_every_request_served_once_in_batches_of_at_most_max_batch():
    srv, launched = _server()
    out = srv.run(_jobs(20), realtime=False)
    assert out["requests"] == 20
    served = [i for ids, *_ in launched for i in ids]
    assert sorted(served) == list(range(20))
    assert all(1 <= len(ids) <= 3 for ids, *_ in launched)
    assert srv.in_use == 0                          # every batch's memory returned
    assert {slot for _, slot, _, _ in launched} <= {0, 1}


def test_admission_waits_for_memory_when_the_budget_is_full():
    # two requests' worth of budget: a second batch waits until the first completes
    srv, launched = _server(budget=2_000, bytes_per_job=1_000, max_batch=2, n_slots=2)
    out = srv.run(_jobs(8), realtime=False)
    assert out["requests"] == 8
    assert srv.stats["admission_waits"] > 0
    assert all(len(ids) <= 2 for ids, *_ in launched)
    assert srv.in_use == 0


def test_capacity_overflow_reruns_the_batch_with_grown_estimates():
    # scene 0's requests need far more instances than the first estimate
    srv, launched = _server(true_M={0: 50_000, 1: 10, 2: 10})
    out = srv.run(_jobs(6), realtime=False)
    assert out["requests"] == 6
    assert srv.stats["reruns"] >= 1
    reruns = [(ids, cap, M) for ids, _, cap, M in launched if M <= cap]
    overflowed = [(ids, cap, M) for ids, _, cap, M in launched if M > cap]
    assert overflowed and reruns
    # a rerun of an overflowed batch holds its instances
    first_over = overflowed[0]
    assert any(ids == first_over[0] and cap >= first_over[2] for ids, cap, _ in reruns)
    # the overflowed batch's estimates grew to hold at least what it needed
    ids, cap, M = first_over
    scenes = {i % 3 for i in ids}
    assert sum(srv.m_est[(sc, 64, 48)] for sc in scenes) >= M
    assert srv.in_use == 0


def test_latency_is_completion_minus_arrival_for_every_request():
    srv, _ = _server()
    jobs = _jobs(9)
    out = srv.run(jobs, realtime=False)
    assert out["requests"] == 9 and out["p50_ms"] >= 0.0 and out["max_ms"] >= out["p99_ms"] >= out["p50_ms"]
