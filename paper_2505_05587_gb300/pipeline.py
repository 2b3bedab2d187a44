"""Buffers and the fused densification iteration on one GPU.

Every step runs in libsteepgs through the binding; this module only owns the
device buffers (allocated once, reused across iterations) and orders the
calls on one stream:

    project -> bin_sort -> render_fwd -> l1_loss_grad (or ssim_l1_loss_grad)
            -> render_bwd_with_splitting (S += P^T(...)P per view)
            -> densify_split (lambda_min, v_min, split, compaction)

The instance count M is data dependent.  Buffers are sized with headroom; when
a view needs more, the pipeline reads M back once, grows the buffers and
re-runs the sort (never silently truncates).

FusedIterationGraph captures one fused iteration as a CUDA graph: the ~35
launches of an iteration then replay without host work between them (every
library call is capture-safe: no allocation, no synchronisation, no host
read-back inside a call).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import binding as B


def as_stream(stream) -> torch.cuda.Stream:
    """A torch stream for the `stream` argument of the calls: None is the
    current stream, an int a raw cudaStream_t."""
    if stream is None:
        return torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream
    return torch.cuda.ExternalStream(int(stream))


@dataclass
class ViewBuffers:
    """Per-view buffers: projection, bins, image maps and the L1 gradient."""
    cam: object
    st: object
    n: int
    proj: B.ProjBuffers
    bins: B.BinBuffers
    image: torch.Tensor
    final_T: torch.Tensor
    n_contrib: torch.Tensor
    dL: torch.Tensor
    sort_ws: torch.Tensor
    with_keys: bool = False
    ssim_ws: torch.Tensor | None = None

    def loss_grad(self, target, n_views: int, loss, lambda_dssim: float | None, stream=None):
        """dL/dimage of this view into self.dL, loss accumulated: L1, or with
        lambda_dssim set, (1 - lambda) L1 + lambda (1 - SSIM)."""
        if lambda_dssim is None:
            B.l1_loss_grad(self.image, target, n_views, self.dL, loss, stream)
            return
        if self.ssim_ws is None:
            H, W = self.cam.height, self.cam.width
            self.ssim_ws = B.workspace(B.ssim_l1_workspace_size(H, W), self.image.device)
        B.ssim_l1_loss_grad(self.image, target, n_views, lambda_dssim, self.dL, loss, self.ssim_ws, stream)

    @staticmethod
    def alloc(n: int, cam, st, capacity: int | None = None, with_keys=False, device="cuda",
              walk: bool = True) -> "ViewBuffers":
        """walk: room for the forward pass's walk lists (the backward pass then
        visits only the entries each warp composited)."""
        T = B.num_tiles(cam, st)
        cap = capacity if capacity is not None else max(4 * n, 1024)
        H, W = cam.height, cam.width
        f = dict(device=device, dtype=torch.float32)
        ww = st.tile_w * st.tile_h // 32 if walk else 0
        return ViewBuffers(cam, st, n, B.ProjBuffers.alloc(n, device),
                           B.BinBuffers.alloc(cap, T, with_keys, device, walk_warps=ww),
                           torch.empty(H, W, 3, **f), torch.empty(H, W, **f),
                           torch.empty(H, W, device=device, dtype=torch.int32), torch.empty(H, W, 3, **f),
                           B.workspace(B.bin_sort_workspace_size(n, cap, T), device), with_keys)

    def grow(self, capacity: int):
        T = B.num_tiles(self.cam, self.st)
        dev = self.image.device
        self.bins = B.BinBuffers.alloc(capacity, T, self.with_keys, dev, walk_warps=self.bins.walk_warps)
        self.sort_ws = B.workspace(B.bin_sort_workspace_size(self.n, capacity, T), dev)


def project_and_sort(g: B.GaussianTensors, vb: ViewBuffers, stream=None, check_capacity=True) -> int | None:
    """Runs project + bin_sort; grows the instance buffers when M exceeds them.
    Returns M when it was read back (check_capacity=True), else None."""
    B.project(g, vb.cam, vb.st, vb.proj, stream)
    B.bin_sort(vb.proj, g.n, vb.cam, vb.st, vb.bins, vb.sort_ws, stream)
    if not check_capacity:
        return None
    as_stream(stream).synchronize()          # the count is read on the host after the sort finishes
    M = B.check_count(int(vb.bins.count.item()))
    if M > vb.bins.capacity:
        vb.grow(int(M * 1.25) + 1024)
        B.bin_sort(vb.proj, g.n, vb.cam, vb.st, vb.bins, vb.sort_ws, stream)
    return M


def render(g: B.GaussianTensors, vb: ViewBuffers, stream=None):
    project_and_sort(g, vb, stream)
    B.render_fwd(vb.proj, vb.bins, vb.cam, vb.st, vb.image, vb.final_T, vb.n_contrib, stream)
    return vb.image


@dataclass
class DensifyBuffers:
    """Accumulators and outputs of the densification step."""
    grads: B.GaussianTensors
    S: torch.Tensor
    bwd_ws: torch.Tensor
    loss: torch.Tensor
    out: B.GaussianTensors
    parent: torch.Tensor
    lam: torch.Tensor
    v: torch.Tensor
    n_out: torch.Tensor
    split_ws: torch.Tensor
    capacity: int
    S_po: torch.Tensor | None = None     # [N,3] position-opacity block when dim_theta = 4 or 7
    S_ls: torch.Tensor | None = None     # [N,18] log-scale blocks (theta = (p, l, o)) when dim_theta = 7

    @staticmethod
    def alloc(g: B.GaussianTensors, capacity: int | None = None, dim_theta: int = 3) -> "DensifyBuffers":
        """dim_theta = 3: splitting matrices over the position (the paper's
        experiments); 4: over (position, opacity); 7: over (position,
        log-scales, opacity)."""
        if dim_theta not in (3, 4, 7):
            raise ValueError("dim_theta must be 3, 4 or 7")
        n = g.n
        dev = g.means.device
        cap = capacity if capacity is not None else 2 * n
        return DensifyBuffers(g.zeros_like(), torch.zeros(n, 6, device=dev),
                              B.workspace(B.render_bwd_workspace_size(n), dev), torch.zeros(1, device=dev),
                              B.GaussianTensors.empty(cap, g.sh_degree, dev),
                              torch.empty(cap, device=dev, dtype=torch.int32), torch.empty(n, device=dev),
                              torch.empty(n, dim_theta, device=dev), torch.zeros(1, device=dev, dtype=torch.int32),
                              B.workspace(B.densify_split_workspace_size(n), dev), cap,
                              torch.zeros(n, 3, device=dev) if dim_theta > 3 else None,
                              torch.zeros(n, 18, device=dev) if dim_theta == 7 else None)

    def zero_(self, grads: bool = True, S: bool = True, stream=None):
        """Resets the accumulators with library memsets on `stream` (default
        the current one).  The gradients need no reset when the first backward
        call of an iteration overwrites them, nor the splitting matrices when
        it resets them (reset_S)."""
        ts = [self.loss]
        if grads:
            ts += list(self.grads.tensors())
        if S:
            ts += [t for t in (self.S, self.S_po, self.S_ls) if t is not None]
        for t in ts:
            B.clear(t, stream)


def fused_iteration(g: B.GaussianTensors, views: list[ViewBuffers], targets: list[torch.Tensor],
                    db: DensifyBuffers, T_split: float = 1.0, eps_split: float = 0.0, step_scale: float = 1.0,
                    grad_norm=None, eps_grad: float = 0.0, stream=None, check_capacity=True, max_splits: int = 0,
                    lambda_dssim: float | None = None):
    """One fused fwd+bwd+splitting iteration over the views (Algorithm 1 with
    the split step taken right after accumulation).  lambda_dssim set: the loss
    has the SSIM term, (1 - lambda) L1 + lambda (1 - SSIM)."""
    db.zero_(grads=False, S=False, stream=stream)    # the loss; the first backward writes grads and S
    V = len(views)
    for k, (vb, tgt) in enumerate(zip(views, targets)):
        project_and_sort(g, vb, stream, check_capacity)
        if lambda_dssim is None:                    # L1: the loss is fused into the forward kernel
            B.render_fwd_l1(vb.proj, vb.bins, vb.cam, vb.st, tgt, V, vb.image, vb.final_T, vb.n_contrib, vb.dL,
                            db.loss, stream)
        else:
            B.render_fwd(vb.proj, vb.bins, vb.cam, vb.st, vb.image, vb.final_T, vb.n_contrib, stream)
            vb.loss_grad(tgt, V, db.loss, lambda_dssim, stream)
        # the first view overwrites the gradients and starts the splitting
        # matrices' accumulation; later views add to both
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, vb.cam, vb.st, vb.final_T, vb.n_contrib, vb.dL,
                                    db.grads, db.S, db.bwd_ws, stream, accumulate=k > 0, S_po=db.S_po,
                                    S_ls=db.S_ls, reset_S=k == 0)
    B.densify_split(g, db.S, 1.0 / T_split, eps_split, step_scale, grad_norm, eps_grad, db.out, db.capacity,
                    db.n_out, db.parent, db.lam, db.v, db.split_ws, stream, max_splits=max_splits, S_po=db.S_po,
                    S_ls=db.S_ls)


class FusedIterationGraph:
    """fused_iteration captured once as a CUDA graph.

    The scene size, the views, the buffers and the scalar arguments are fixed
    at capture; the VALUES in the parameter, target and gradient buffers may
    change between replays (the graph reads and writes the same device
    memory).  One eager iteration first sizes the instance buffers.  When the
    parameters move, a view may need more instances than its buffers hold:
    the sort then writes nothing out of bounds but the iteration is not valid,
    so replay(check=True) reads the counts back and raises; grow the buffers
    (an eager fused_iteration does) and capture again."""

    def __init__(self, g: B.GaussianTensors, views: list[ViewBuffers], targets: list[torch.Tensor],
                 db: DensifyBuffers, **kw):
        kw.pop("stream", None)
        kw.pop("check_capacity", None)
        self.views = views
        fused_iteration(g, views, targets, db, check_capacity=True, **kw)
        torch.cuda.synchronize()
        self.stream = torch.cuda.Stream(device=g.means.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            fused_iteration(g, views, targets, db, stream=self.stream, check_capacity=False, **kw)

    def replay(self, check: bool = False):
        """Launches the captured iteration on the current stream."""
        self.graph.replay()
        if check:
            for vb in self.views:
                M = B.check_count(int(vb.bins.count.item()))
                if M > vb.bins.capacity:
                    raise RuntimeError(f"a view needs {M} instances, its buffers hold {vb.bins.capacity}: "
                                       "run fused_iteration eagerly to grow them and capture again")


class PrefetchedIterations:
    """Fused iterations fed from page-locked host memory with the inputs of
    iteration k + 1 copied (on a copy stream) while iteration k computes: two
    device copies of the parameters and the targets, one captured graph for
    each, and events that order every copy after the last iteration that read
    its buffers and every iteration after its own copy.  The views' and the
    densification buffers are shared (the iterations run in order on one
    stream); each iteration's loss and split count are read back to host.

    run(host_params, host_targets, k_steps) -> (loss[k], n_out[k]) host arrays;
    host_params / host_targets: per iteration, or one set reused."""

    def __init__(self, g: B.GaussianTensors, views: list[ViewBuffers], targets: list[torch.Tensor],
                 db: DensifyBuffers, **kw):
        self.sets = [(g, targets)]
        g2 = B.GaussianTensors(*[t.clone() for t in g.tensors()], g.sh_degree)
        self.sets.append((g2, [t.clone() for t in targets]))
        self.graphs = [FusedIterationGraph(gs, views, ts, db, **kw) for gs, ts in self.sets]
        self.db = db
        dev = g.means.device
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.copied = [torch.cuda.Event(), torch.cuda.Event()]
        self.done = [torch.cuda.Event(), torch.cuda.Event()]
        self.loss_host = torch.empty(2, dtype=torch.float32).pin_memory()
        self.nout_host = torch.empty(2, dtype=torch.int32).pin_memory()

    def _copy(self, s: int, params_host, targets_host, after_done: bool):
        gs, ts = self.sets[s]
        with torch.cuda.stream(self.copy_stream):
            if after_done:
                self.copy_stream.wait_event(self.done[s])       # the buffers' last reader finished
            for dst, src in zip(gs.tensors(), params_host):
                dst.copy_(src, non_blocking=True)
            for dst, src in zip(ts, targets_host):
                dst.copy_(src, non_blocking=True)
            self.copied[s].record(self.copy_stream)

    def run(self, host_params, host_targets, k_steps: int, stream=None):
        """Issues k_steps iterations; returns the pinned per-iteration loss and
        split count arrays (valid once `stream` has been synchronised)."""
        stream = as_stream(stream)
        per_step = isinstance(host_params[0], (list, tuple))
        pick = (lambda seq, k: seq[k]) if per_step else (lambda seq, k: seq)
        loss = torch.empty(k_steps, dtype=torch.float32).pin_memory()
        nout = torch.empty(k_steps, dtype=torch.int32).pin_memory()
        self._copy(0, pick(host_params, 0), pick(host_targets, 0), after_done=False)
        for k in range(k_steps):
            s = k & 1
            if k + 1 < k_steps:
                self._copy(1 - s, pick(host_params, k + 1), pick(host_targets, k + 1), after_done=k >= 1)
            stream.wait_event(self.copied[s])
            with torch.cuda.stream(stream):
                self.graphs[s].replay()
                loss[k:k + 1].copy_(self.db.loss, non_blocking=True)
                nout[k:k + 1].copy_(self.db.n_out, non_blocking=True)
            self.done[s].record(stream)
        return loss, nout
