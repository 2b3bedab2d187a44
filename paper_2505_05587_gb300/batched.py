"""Batched densification step: several views of uneven resolution in one pass.

One ``render_views_with_splitting`` call (projection of all (view, Gaussian)
pairs, one binning and depth sort, persistent forward and backward kernels,
L1 loss, projection adjoint summed over views) followed by ``densify_split``,
captured once into a CUDA graph and replayed.  The tile shape and the staging
batch depth are chosen by a small autotuner that times every candidate on the
actual workload.

For comparison ``PlainDensifyStep`` runs the same step one view per launch
sequence (project, bin_sort, render_fwd, l1, render_bwd per view).
"""
from __future__ import annotations

import dataclasses
import time

import torch

from . import binding as B
from . import pipeline as PL

TILE_SHAPES = [(16, 16), (16, 8), (8, 8), (32, 8)]
BATCH_DEPTHS = [64, 128, 256]


def concat_images(images: list[torch.Tensor]) -> torch.Tensor:
    """[H_v, W_v, 3] images -> the concatenated [sum H_v W_v, 3] layout."""
    return torch.cat([im.reshape(-1, 3) for im in images], 0).contiguous()


class BatchedDensifyStep:
    def __init__(self, g: B.GaussianTensors, cams, targets: torch.Tensor, st, batch: int = 0,
                 capacity: int | None = None, eps_split: float = 0.0, step_scale: float = 1.0):
        self.g, self.cams, self.targets, self.st, self.batch = g, cams, targets, st, batch
        self.eps_split, self.step_scale = eps_split, step_scale
        dev = g.means.device
        self.P = sum(c.width * c.height for c in cams)
        self.images = torch.empty(self.P, 3, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.grads = g.zeros_like()
        self.S = torch.zeros(g.n, 6, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.db = PL.DensifyBuffers.alloc(g)
        self.graph = None
        self._set_capacity(capacity if capacity is not None else 4 * g.n * len(cams))

    def _set_capacity(self, cap: int):
        self.capacity = int(cap)
        nbytes = B.render_views_workspace_size(self.g.n, self.cams, self.st, self.capacity)
        self.ws = B.workspace(nbytes, self.g.means.device)
        self.graph = None

    def run_eager(self, stream=None):
        B.clear(self.loss, stream)          # the projection adjoint writes the gradients and S (reset)
        B.render_views_with_splitting(self.g, self.cams, self.st, self.batch, self.targets, self.images, self.loss,
                                      self.grads, False, self.S, self.count, self.capacity, self.ws, stream,
                                      reset_S=True)
        db = self.db
        B.densify_split(self.g, self.S, 1.0, self.eps_split, self.step_scale, None, 0.0, db.out, db.capacity,
                        db.n_out, db.parent, db.lam, db.v, db.split_ws, stream)

    def fit_capacity(self):
        """Runs once eagerly and grows the instance capacity until it holds M."""
        while True:
            self.run_eager()
            M = B.check_count(int(self.count.item()))
            if M <= self.capacity:
                return M
            self._set_capacity(int(M * 1.1) + 4096)

    def capture(self):
        """Captures the step (zeroing, batched render/backward, densify) in a CUDA graph."""
        self.fit_capacity()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run_eager()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run_eager()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


class PlainDensifyStep:
    """The same step with one launch sequence per view."""

    def __init__(self, g: B.GaussianTensors, cams, targets: list[torch.Tensor], st, eps_split: float = 0.0,
                 step_scale: float = 1.0):
        self.g, self.cams, self.targets, self.st = g, cams, targets, st
        self.eps_split, self.step_scale = eps_split, step_scale
        self.views = [PL.ViewBuffers.alloc(g.n, c, st, device=g.means.device) for c in cams]
        self.db = PL.DensifyBuffers.alloc(g)
        for vb in self.views:          # size the instance buffers once
            PL.project_and_sort(g, vb)

    def run(self, stream=None):
        PL.fused_iteration(self.g, self.views, self.targets, self.db, eps_split=self.eps_split,
                           step_scale=self.step_scale, stream=stream, check_capacity=False)


def time_fn(fn, reps: int = 5, warmup: int = 2) -> float:
    """Mean device milliseconds per call (CUDA events on the current stream)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(g: B.GaussianTensors, cams, targets: torch.Tensor, st, reps: int = 3, shapes=None, batches=None,
             log=None):
    """Times every (tile shape, batch depth) candidate on the workload and
    returns the fastest as (settings, batch, table)."""
    table = []
    best = None
    for (tw, th) in (shapes or TILE_SHAPES):
        st_c = dataclasses.replace(st, tile_w=tw, tile_h=th)
        step = None
        for b in (batches or BATCH_DEPTHS):
            if step is None:
                step = BatchedDensifyStep(g, cams, targets, st_c, batch=b)
                step.fit_capacity()
            else:
                step.batch = b
            ms = time_fn(step.run_eager, reps=reps, warmup=1)
            table.append({"tile": f"{tw}x{th}", "batch": b, "ms": round(ms, 4)})
            if log:
                log(table[-1])
            if best is None or ms < best[2]:
                best = (st_c, b, ms)
        del step
        torch.cuda.empty_cache()
    return best[0], best[1], table


def run_ring_densify(n: int = 3_000_000, steps: int = 20, warmup: int = 3, tune: bool = True) -> dict:
    """Batched densification step on the ring of 8 uneven views: 3M Gaussians
    (cluster mixture, SH3).  Times the autotuned, graph-captured batched step
    against the one-view-per-launch form of the same step."""
    import synth
    scene = synth.cluster_scene(0, n, 3)
    cams = synth.ring_cameras(6.0)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    tgs = [torch.as_tensor(synth.target_image(10 + k, c.height, c.width)).cuda() for k, c in enumerate(cams)]
    targets = concat_images(tgs)
    del scene
    table = []
    if tune:
        st_best, batch, table = autotune(g, cams, targets, st, reps=3)
    else:
        st_best, batch = st, 256
    step = BatchedDensifyStep(g, cams, targets, st_best, batch=batch)
    step.capture()
    ms_graph = time_fn(step.replay, reps=steps, warmup=warmup)
    ms_eager = time_fn(step.run_eager, reps=steps, warmup=warmup)
    M = int(step.count.item())
    n_out = int(step.db.n_out.item())
    del step
    torch.cuda.empty_cache()
    plain = PlainDensifyStep(g, cams, tgs, st_best)
    ms_plain = time_fn(plain.run, reps=steps, warmup=warmup)
    return {"workload": "batched densification step: 3M Gaussians (cluster mixture, SH3), 8 ring views "
                        "1957x1091, 1600x1060, 1237x822, 980x545 x2, 800x600 x3",
            "gaussians": n, "views": len(cams), "pixels": sum(c.width * c.height for c in cams),
            "tile": f"{st_best.tile_w}x{st_best.tile_h}", "batch": batch, "instances_M": M, "n_out": n_out,
            "ms_batched_graph": round(ms_graph, 4), "ms_batched_eager": round(ms_eager, 4),
            "ms_one_view_per_launch": round(ms_plain, 4), "speedup_vs_plain": round(ms_plain / ms_graph, 3),
            "autotune": table}


def run_eager_steps(steps: int = 3, n: int = 3_000_000, tile=(16, 16), batch: int = 128, views: int = 8) -> dict:
    """A few eager batched steps on the ring workload with a fixed tile shape
    and batch depth (no tuning, no graph), over its first `views` views: the
    command a per-launch profile of the batched step runs."""
    import synth
    scene = synth.cluster_scene(0, n, 3)
    cams = synth.ring_cameras(6.0)[:views]
    st = dataclasses.replace(synth.Settings(), tile_w=tile[0], tile_h=tile[1])
    g = B.GaussianTensors.from_scene(scene)
    del scene
    tgs = [torch.as_tensor(synth.target_image(10 + k, c.height, c.width)).cuda() for k, c in enumerate(cams)]
    step = BatchedDensifyStep(g, cams, concat_images(tgs), st, batch=batch)
    M = step.fit_capacity()
    ms = time_fn(step.run_eager, reps=steps, warmup=0)
    return {"steps": steps, "instances_M": M, "ms_eager": round(ms, 4)}


if __name__ == "__main__":
    import json
    import sys
    if len(sys.argv) > 2 and sys.argv[1] == "--eager":        # --eager STEPS [VIEWS [GAUSSIANS]]
        print(json.dumps(run_eager_steps(int(sys.argv[2]), views=int(sys.argv[3]) if len(sys.argv) > 3 else 8,
                                         n=int(sys.argv[4]) if len(sys.argv) > 4 else 3_000_000)))
    else:
        print(json.dumps(run_ring_densify(int(sys.argv[1]) if len(sys.argv) > 1 else 3_000_000)))
