"""Render serving with continuous batching.

Scene Gaussians stay resident on the device.  Requests (scene, camera,
resolution) arrive over time; a host scheduler forms batches of the requests
that have arrived, up to `max_batch`, whenever a stream slot is free and the
batch's memory fits the HBM budget (admission by free device memory), and
launches each batch as ONE forward pass (``render_batch_fwd``: projection of
every request's scene, one binning and depth sort, one persistent compositing
kernel over the tiles of all its views).  A batch of one request (what a
lightly loaded server mostly sees) takes the single-view calls instead
(project, bin_sort, render_fwd with the tile schedule) on its slot's
grow-only buffers, with no host synchronisation between them; the image is
the same bits either way.  Batches in flight on different streams overlap
on the device; completions are detected with events and their memory is
returned to the budget.  Latency = completion - arrival.

``serve_one_per_launch`` is the baseline: each request alone, one launch
sequence at a time, in arrival order.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B


@dataclass
class Job:
    idx: int
    arrival: float      # seconds from the start of the run
    scene: int
    cam: object


@dataclass
class _SlotView:
    """Grow-only single-view buffers of one stream slot."""
    proj: B.ProjBuffers
    bins: B.BinBuffers
    sort_ws: torch.Tensor
    image: torch.Tensor     # [P, 3] f32
    final_T: torch.Tensor   # [P] f32
    n_contrib: torch.Tensor  # [P] i32
    n: int
    tiles: int


@dataclass
class _Batch:
    jobs: list
    stream: int                 # slot index
    event: torch.cuda.Event
    images: torch.Tensor
    ws: torch.Tensor
    count: torch.Tensor
    count_host: torch.Tensor
    capacity: int
    nbytes: int
    pix_off: list


class RenderServer:
    def __init__(self, scenes: list[B.GaussianTensors], st, max_batch: int = 8, n_slots: int = 4,
                 hbm_budget: int | None = None, batch_depth: int = 0, keep_images: bool = False,
                 single_path: bool = True):
        self.scenes, self.st = scenes, st
        self.single_path = single_path
        self.slot_view: list = [None] * n_slots
        self.max_batch, self.n_slots, self.batch_depth = max_batch, n_slots, batch_depth
        self.keep_images = keep_images
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(hbm_budget if hbm_budget is not None else 0.5 * free)
        self.in_use = 0
        self.streams = [torch.cuda.Stream() for _ in range(n_slots)]
        self.slot_ws = [None] * n_slots          # grow-only workspaces, one per stream slot
        self.slot_img = [None] * n_slots
        self.slot_cnt = [torch.zeros(1, dtype=torch.int32, device="cuda") for _ in range(n_slots)]
        self.m_est: dict = {}            # (scene, w, h) -> instance estimate
        self.images: dict = {}
        self.stats = collections.Counter()

    def _est(self, j) -> int:
        return self.m_est.get((j.scene, j.cam.width, j.cam.height), 4 * self.scenes[j.scene].n)

    def _capacity(self, jobs) -> int:
        return int(sum(self._est(j) for j in jobs)) + 4096

    def _batch_bytes(self, jobs, capacity) -> int:
        scenes = [self.scenes[j.scene] for j in jobs]
        cams = [j.cam for j in jobs]
        ws = B.render_batch_workspace_size(scenes, cams, self.st, capacity)
        return ws + 12 * sum(c.width * c.height for c in cams)

    def _view(self, slot, n, capacity, T, P) -> _SlotView:
        v = self.slot_view[slot]
        if v is None or v.n < n or v.bins.capacity < capacity or v.tiles < T or v.final_T.shape[0] < P:
            n2 = max(n, v.n if v else 0)
            cap2 = max(capacity, v.bins.capacity if v else 0)
            T2 = max(T, v.tiles if v else 0)
            P2 = max(P, v.final_T.shape[0] if v else 0)
            v = _SlotView(B.ProjBuffers.alloc(n2), B.BinBuffers.alloc(cap2, T2),
                          B.workspace(B.bin_sort_workspace_size(n2, cap2, T2)),
                          torch.empty(P2, 3, device="cuda"), torch.empty(P2, device="cuda"),
                          torch.empty(P2, dtype=torch.int32, device="cuda"), n2, T2)
            self.slot_view[slot] = v
        return v

    def _launch_single(self, job, slot, capacity) -> _Batch:
        stream = self.streams[slot]
        g, cam = self.scenes[job.scene], job.cam
        P = cam.width * cam.height
        T = B.num_tiles(cam, self.st)
        with torch.cuda.stream(stream):
            v = self._view(slot, g.n, capacity, T, P)
            img, fT, nc = v.image[:P], v.final_T[:P], v.n_contrib[:P]
            B.project(g, cam, self.st, v.proj, stream)
            B.bin_sort(v.proj, g.n, cam, self.st, v.bins, v.sort_ws, stream)
            B.render_fwd(v.proj, v.bins, cam, self.st, img, fT, nc, stream)
            count_host = torch.empty(1, dtype=torch.int32, pin_memory=True)
            count_host.copy_(v.bins.count, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        nbytes = self._batch_bytes([job], capacity)
        self.in_use += nbytes
        self.stats["batches"] += 1
        self.stats["batched_requests"] += 1
        self.stats["single_view_batches"] += 1
        return _Batch([job], slot, ev, img, v.sort_ws, v.bins.count, count_host, v.bins.capacity, nbytes, [0, P])

    def _launch(self, jobs, slot, capacity=None) -> _Batch:
        stream = self.streams[slot]
        capacity = capacity or self._capacity(jobs)
        if len(jobs) == 1 and self.single_path:
            return self._launch_single(jobs[0], slot, capacity)
        scenes = [self.scenes[j.scene] for j in jobs]
        cams = [j.cam for j in jobs]
        nbytes = self._batch_bytes(jobs, capacity)
        P = sum(c.width * c.height for c in cams)
        wsb = B.render_batch_workspace_size(scenes, cams, self.st, capacity)
        with torch.cuda.stream(stream):
            if self.slot_ws[slot] is None or self.slot_ws[slot].numel() < wsb:
                self.slot_ws[slot] = B.workspace(int(wsb * 1.25))
            if self.slot_img[slot] is None or self.slot_img[slot].shape[0] < P:
                self.slot_img[slot] = torch.empty(int(P * 1.25), 3, device="cuda")
            ws, images, count = self.slot_ws[slot], self.slot_img[slot][:P], self.slot_cnt[slot]
            B.render_batch_fwd(scenes, cams, self.st, self.batch_depth, images, count, capacity, ws, stream)
            count_host = torch.empty(1, dtype=torch.int32, pin_memory=True)
            count_host.copy_(count, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        offs = np.cumsum([0] + [c.width * c.height for c in cams]).tolist()
        self.in_use += nbytes
        self.stats["batches"] += 1
        self.stats["batched_requests"] += len(jobs)
        return _Batch(jobs, slot, ev, images, ws, count, count_host, capacity, nbytes, offs)

    def _finish(self, b: _Batch, now: float, lat: dict) -> _Batch | None:
        self.in_use -= b.nbytes
        M = B.check_count(int(b.count_host.item()))
        if M > b.capacity:                       # instance capacity too small: rerun with room
            self.stats["reruns"] += 1
            ests = [self._est(j) for j in b.jobs]
            for j, e in zip(b.jobs, ests):       # estimates only grow
                self.m_est[(j.scene, j.cam.width, j.cam.height)] = int(1.5 * e * M / max(sum(ests), 1)) + 1024
            return self._launch(b.jobs, b.stream, int(M * 1.1) + 4096)
        for k, j in enumerate(b.jobs):
            lat[j.idx] = now - j.arrival
            if self.keep_images:
                self.images[j.idx] = b.images[b.pix_off[k]:b.pix_off[k + 1]].reshape(j.cam.height, j.cam.width,
                                                                                      3).clone()
        return None

    def run(self, jobs: list[Job], realtime: bool = True) -> dict:
        """Serves the jobs (sorted by arrival); realtime=False releases every
        job at t=0 (saturation)."""
        jobs = sorted(jobs, key=lambda j: j.arrival)
        if not realtime:
            jobs = [Job(j.idx, 0.0, j.scene, j.cam) for j in jobs]
        pending = collections.deque()
        free_slots = list(range(self.n_slots))
        inflight: dict = {}
        lat: dict = {}
        nxt = 0
        t0 = time.perf_counter()
        while len(lat) < len(jobs):
            now = time.perf_counter() - t0
            while nxt < len(jobs) and jobs[nxt].arrival <= now:
                pending.append(jobs[nxt])
                nxt += 1
            # completions
            for slot, b in list(inflight.items()):
                if b.event.query():
                    again = self._finish(b, time.perf_counter() - t0, lat)
                    if again is not None:
                        inflight[slot] = again
                    else:
                        del inflight[slot]
                        free_slots.append(slot)
            # admissions: fill free slots with batches that fit the budget
            while free_slots and pending:
                take = []
                while pending and len(take) < self.max_batch:
                    cand = take + [pending[0]]
                    cap = self._capacity(cand)
                    if take and self.in_use + self._batch_bytes(cand, cap) > self.budget:
                        break
                    take.append(pending.popleft())
                if not take:
                    break
                if self.in_use + self._batch_bytes(take, self._capacity(take)) > self.budget and inflight:
                    pending.extendleft(reversed(take))     # wait for memory to free up
                    self.stats["admission_waits"] += 1
                    break
                slot = free_slots.pop()
                inflight[slot] = self._launch(take, slot)
            if not inflight and not pending and nxt < len(jobs):
                _wait_until(t0 + jobs[nxt].arrival, 0.002)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return _summary(jobs, lat, wall, dict(self.stats))


def serve_one_per_launch(scenes: list[B.GaussianTensors], st, jobs: list[Job], realtime: bool = True,
                         keep_images: bool = False) -> dict:
    """Baseline: every request alone, one launch sequence after the other."""
    from . import pipeline as PL
    jobs = sorted(jobs, key=lambda j: j.arrival)
    if not realtime:
        jobs = [Job(j.idx, 0.0, j.scene, j.cam) for j in jobs]
    views = {}
    lat, images = {}, {}
    t0 = time.perf_counter()
    for j in jobs:
        _wait_until(t0 + j.arrival)
        key = (j.scene, j.cam.width, j.cam.height)
        g = scenes[j.scene]
        if key not in views:
            views[key] = PL.ViewBuffers.alloc(g.n, j.cam, st, walk=False)     # a forward-only render
        vb = views[key]
        vb.cam = j.cam
        PL.project_and_sort(g, vb)             # reads back M (a sync) as a per-request launch sequence does
        B.render_fwd(vb.proj, vb.bins, j.cam, st, vb.image, vb.final_T, vb.n_contrib)
        torch.cuda.synchronize()
        lat[j.idx] = time.perf_counter() - t0 - j.arrival
        if keep_images:
            images[j.idx] = vb.image.clone()
    wall = time.perf_counter() - t0
    out = _summary(jobs, lat, wall, {})
    if keep_images:
        out["images"] = images
    return out


def _wait_until(t: float, at_most: float = float("inf")):
    """Waits until perf_counter() reaches t, or for at most `at_most` seconds:
    sleeps, then spins the last 0.3 ms (a sleep overshoots by tens of us)."""
    end = min(t, time.perf_counter() + at_most)
    left = end - time.perf_counter()
    if left > 4e-4:
        time.sleep(left - 3e-4)
    while time.perf_counter() < end:
        pass


def _summary(jobs, lat, wall, stats) -> dict:
    l = np.array([lat[j.idx] for j in jobs]) * 1e3
    return {"requests": len(jobs), "wall_s": round(wall, 4), "frames_per_s": round(len(jobs) / wall, 2),
            "p50_ms": round(float(np.percentile(l, 50)), 3), "p99_ms": round(float(np.percentile(l, 99)), 3),
            "mean_ms": round(float(l.mean()), 3), "max_ms": round(float(l.max()), 3), **stats}


def serving_requests(seed: int = 3, n_requests: int = 4000, rate_hz: float = 200.0, n_scenes: int = 6):
    import synth
    reqs = synth.request_stream(seed, n_requests, rate_hz, n_scenes)
    return [Job(k, r.arrival_s - reqs[0].arrival_s, r.scene, r.camera) for k, r in enumerate(reqs)]


def resident_scenes(sizes=(100_000, 300_000, 1_000_000, 1_000_000, 2_000_000, 3_000_000)):
    import synth
    return [B.GaussianTensors.from_scene(synth.cluster_scene(10 + k, n, 3)) for k, n in enumerate(sizes)]


def run_serving(n_requests: int = 4000, rate_hz: float = 200.0) -> dict:
    import synth
    st = synth.Settings()
    scenes = resident_scenes()
    jobs = serving_requests(3, n_requests, rate_hz, len(scenes))
    warm = jobs[:200]
    server = RenderServer(scenes, st)
    server.run(warm, realtime=False)               # warm-up: workspaces and instance estimates
    serve_one_per_launch(scenes, st, warm, realtime=False)
    out = {"workload": f"render serving: {n_requests} requests, Poisson {rate_hz:g} req/s, 6 resident scenes "
                       "(100k, 300k, 1M, 1M, 2M, 3M Gaussians, SH3), 640x480 / 1237x822 / 1920x1080"}
    server.stats.clear()
    out["continuous_batching_realtime"] = server.run(jobs, realtime=True)
    out["one_per_launch_realtime"] = serve_one_per_launch(scenes, st, jobs, realtime=True)
    sat = jobs[:1000]
    server.stats.clear()
    out["continuous_batching_saturated"] = server.run(sat, realtime=False)
    out["one_per_launch_saturated"] = serve_one_per_launch(scenes, st, sat, realtime=False)
    return out


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(run_serving(int(sys.argv[1]) if len(sys.argv) > 1 else 4000)))
