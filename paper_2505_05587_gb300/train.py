"""Differentiable rendering through libsteepgs and the SteepGS training loop.

``RasterizeWithSplitting`` is a ``torch.autograd.Function`` whose forward is
project + bin_sort + render_fwd and whose backward is the hand-written adjoint
``render_bwd_with_splitting`` (transmittance recomputed back to front; no
per-pixel Gaussian lists are stored).  As a side effect the backward adds the
view's splitting matrices to a persistent accumulator (Algorithm 1:
S <- S + dl/dsigma Hess sigma at every step).

``SteepGSTrainer`` runs Algorithm 1: Adam steps (a library kernel) with the
splitting matrices and gradients accumulated every step, and every T_split
steps from `start` on, the steepest-density-control split: lambda_min, v_min
of S / (steps accumulated), offspring p +- eps v_min with opacity o/2.
Offspring get zeroed Adam moments; S and G are reset after each split.
The trainer's state between steps can be saved and restored (``save``,
``restore``, ``run(first_step=...)``).
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass, field

import torch

from . import binding as B
from . import pipeline as PL


@dataclass
class RenderContext:
    """Per-view state shared by the forward and backward of one render."""
    view: PL.ViewBuffers
    S: torch.Tensor            # [N,6] splitting-matrix accumulator (added to in backward)
    bwd_ws: torch.Tensor
    sh_degree: int
    S_po: torch.Tensor | None = None   # [N,3] position-opacity block (theta = (p, o) or (p, l, o))
    S_ls: torch.Tensor | None = None   # [N,18] log-scale blocks (theta = (p, l, o))


class RasterizeWithSplitting(torch.autograd.Function):
    """image = render(means, log_scales, quats, opacity_logit, sh) for one view."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, rc: RenderContext):
        g = B.GaussianTensors(means.detach().contiguous(), log_scales.detach().contiguous(),
                              quats.detach().contiguous(), opacity_logit.detach().contiguous(),
                              sh.detach().contiguous(), rc.sh_degree)
        vb = rc.view
        PL.project_and_sort(g, vb)
        B.render_fwd(vb.proj, vb.bins, vb.cam, vb.st, vb.image, vb.final_T, vb.n_contrib)
        ctx.g = g
        ctx.rc = rc
        return vb.image.clone()

    @staticmethod
    def backward(ctx, dL_dimage):
        g, rc = ctx.g, ctx.rc
        vb = rc.view
        grads = B.GaussianTensors.empty(g.n, g.sh_degree, g.means.device)
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, vb.cam, vb.st, vb.final_T, vb.n_contrib,
                                    dL_dimage.contiguous(), grads, rc.S, rc.bwd_ws, accumulate=False, S_po=rc.S_po,
                                    S_ls=rc.S_ls)
        return grads.means, grads.log_scales, grads.quats, grads.opacity_logit, grads.sh, None


def render(params: list[torch.Tensor], rc: RenderContext) -> torch.Tensor:
    return RasterizeWithSplitting.apply(*params, rc)


@dataclass
class TrainConfig:
    lr: float = 1e-3
    steps: int = 2000
    T_split: int = 100
    start: int = 500
    eps_split: float = -1e-6
    step_scale: float = 1.0
    eps_grad: float | None = None      # compactest gate ||G_bar|| <= eps_grad when set
    max_splits: int = 0                # increment budget per densification (0: none)
    dim_theta: int = 3                 # splitting over the position (3), (position, opacity) (4) or
    #                                    (position, log-scales, opacity) (7)
    lambda_dssim: float | None = None  # loss (1 - l) L1 + l (1 - SSIM) when set, else L1
    log_every: int = 10
    graphs: bool = True                # each training step replayed as captured CUDA graphs (else autograd)


def densify_due(t: int, cfg: TrainConfig) -> bool:
    """Whether step t (1-based) ends with a densification: every T_split steps
    from step `start` on (Section 5, implementation details: every 100 steps
    from the 500th)."""
    return t >= cfg.start and t % cfg.T_split == 0


class SteepGSTrainer:
    """Algorithm 1 on one GPU: one view per step (cycled), L1 loss, Adam.

    With cfg.graphs (the default) a step is two captured CUDA graphs per view:
    (projection, binning) and (forward with the loss, backward with the
    splitting accumulators, Adam on every parameter, the device step count);
    between them the view's instance count is read back, and when it
    outgrows the buffers they grow and the graphs are captured again, so no
    step runs on truncated lists.  The graphs are captured again after every
    densification (the number of Gaussians changes).  Without graphs a step
    runs through the autograd Function above."""

    def __init__(self, g: B.GaussianTensors, cams, targets: list[torch.Tensor], st, cfg: TrainConfig):
        self.cams, self.targets, self.st, self.cfg = cams, targets, st, cfg
        self.sh_degree = g.sh_degree
        self.params = [t.clone().requires_grad_(True) for t in g.tensors()]
        self.log: list[dict] = []
        self._alloc(g.n)
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.adam_t = 0
        self.step_graphs = None

    def _alloc(self, n: int):
        dev = self.params[0].device
        self.views = [PL.ViewBuffers.alloc(n, c, self.st, device=dev) for c in self.cams]
        self.S = torch.zeros(n, 6, device=dev)
        self.S_po = torch.zeros(n, 3, device=dev) if self.cfg.dim_theta > 3 else None
        self.S_ls = torch.zeros(n, 18, device=dev) if self.cfg.dim_theta == 7 else None
        self.G = torch.zeros(n, 3, device=dev)
        self.n_accum = 0
        self.bwd_ws = B.workspace(B.render_bwd_workspace_size(n), dev)
        self.dL = [torch.empty_like(t) for t in self.targets]
        self.loss = torch.zeros(1, device=dev)
        if self.cfg.lambda_dssim is not None and not hasattr(self, "ssim_ws"):
            H = max(c.height for c in self.cams)
            W = max(c.width for c in self.cams)
            self.ssim_ws = B.workspace(B.ssim_l1_workspace_size(H, W), dev)

    @property
    def n(self) -> int:
        return int(self.params[0].shape[0])

    def gaussians(self) -> B.GaussianTensors:
        return B.GaussianTensors(*[p.detach() for p in self.params], self.sh_degree)

    def _capture(self):
        """Captures the (projection, binning) and (forward, loss, backward,
        Adam) graphs of every view for the current buffers."""
        cfg = self.cfg
        dev = self.params[0].device
        g = self.gaussians()
        self.grads = B.GaussianTensors.empty(g.n, self.sh_degree, dev)
        self.d_step = torch.full((1,), self.adam_t, dtype=torch.int32, device=dev)
        for vb in self.views:                       # size the instance buffers (no side effects)
            PL.project_and_sort(g, vb)
        torch.cuda.synchronize()
        cs = torch.cuda.Stream(device=dev)
        self.step_graphs = []
        for k, vb in enumerate(self.views):
            ga, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(ga, stream=cs):
                PL.project_and_sort(g, vb, cs, check_capacity=False)
            with torch.cuda.graph(gb, stream=cs):
                B.clear(self.loss, cs)
                if cfg.lambda_dssim is None:
                    B.render_fwd_l1(vb.proj, vb.bins, vb.cam, vb.st, self.targets[k], 1, vb.image, vb.final_T,
                                    vb.n_contrib, self.dL[k], self.loss, cs)
                else:
                    B.render_fwd(vb.proj, vb.bins, vb.cam, vb.st, vb.image, vb.final_T, vb.n_contrib, cs)
                    B.ssim_l1_loss_grad(vb.image, self.targets[k], 1, cfg.lambda_dssim, self.dL[k], self.loss,
                                        self.ssim_ws, cs)
                B.render_bwd_with_splitting(g, vb.proj, vb.bins, vb.cam, vb.st, vb.final_T, vb.n_contrib, self.dL[k],
                                            self.grads, self.S, self.bwd_ws, cs, accumulate=False, S_po=self.S_po,
                                            S_ls=self.S_ls)
                self.d_step.add_(1)
                for i, (p, gr) in enumerate(zip(self.params, self.grads.tensors())):
                    B.adam_step_dev(p.data, gr, self.m[i], self.v[i], cfg.lr, self.d_step,
                                    grad_accum=self.G if i == 0 else None, stream=cs)
            self.step_graphs.append((ga, gb))

    def _graph_step(self, k: int):
        if self.step_graphs is None:
            self._capture()
        ga, gb = self.step_graphs[k]
        vb = self.views[k]
        ga.replay()
        M = B.check_count(int(vb.bins.count.item()))
        if M > vb.bins.capacity:                    # grow, capture again, redo the binning
            vb.grow(int(M * 1.25) + 1024)
            self.step_graphs = None
            self._capture()
            ga, gb = self.step_graphs[k]
            ga.replay()
        gb.replay()

    def step(self, t: int) -> float | None:
        k = t % len(self.cams)
        if self.cfg.graphs:
            self._graph_step(k)
            self.adam_t += 1
            self.n_accum += 1
            loss = None
            if t % self.cfg.log_every == 0 or t == 1:
                loss = float(self.loss.item())
                self.log.append({"step": t, "loss": loss, "gaussians": self.n})
            if densify_due(t, self.cfg):
                self.densify(t)
            return loss
        rc = RenderContext(self.views[k], self.S, self.bwd_ws, self.sh_degree, self.S_po, self.S_ls)
        image = render(self.params, rc)
        B.clear(self.loss)
        if self.cfg.lambda_dssim is None:
            B.l1_loss_grad(image.detach(), self.targets[k], 1, self.dL[k], self.loss)
        else:
            B.ssim_l1_loss_grad(image.detach(), self.targets[k], 1, self.cfg.lambda_dssim, self.dL[k], self.loss,
                                self.ssim_ws)
        for p in self.params:
            p.grad = None
        image.backward(self.dL[k])
        self.adam_t += 1
        for i, p in enumerate(self.params):
            B.adam_step(p.data, p.grad, self.m[i], self.v[i], self.cfg.lr, self.adam_t,
                        grad_accum=self.G if i == 0 else None)
        self.n_accum += 1
        loss = None
        if t % self.cfg.log_every == 0 or t == 1:
            loss = float(self.loss.item())
            self.log.append({"step": t, "loss": loss, "gaussians": self.n})
        if densify_due(t, self.cfg):
            self.densify(t)
        return loss

    def densify(self, t: int):
        cfg = self.cfg
        g = self.gaussians()
        n = g.n
        dev = g.means.device
        out = B.GaussianTensors.empty(2 * n, self.sh_degree, dev)
        parent = torch.empty(2 * n, dtype=torch.int32, device=dev)
        n_out = torch.zeros(1, dtype=torch.int32, device=dev)
        lam = torch.empty(n, device=dev)
        vmin = torch.empty(n, cfg.dim_theta, device=dev)
        ws = B.workspace(B.densify_split_workspace_size(n), dev)
        gn = None
        if cfg.eps_grad is not None:
            gn = (self.G / max(self.n_accum, 1)).norm(dim=1).contiguous()
        B.densify_split(g, self.S, 1.0 / max(self.n_accum, 1), cfg.eps_split, cfg.step_scale, gn,
                        cfg.eps_grad or 0.0, out, 2 * n, n_out, parent, lam, vmin, ws, max_splits=cfg.max_splits,
                        S_po=self.S_po, S_ls=self.S_ls)
        n2 = int(n_out.item())
        split = n2 - n
        par = parent[:n2].long()
        flagged_parents = par[n:]
        # Adam moments follow their rows; both offspring of a split start from zero
        for i, old in enumerate(self.params):
            new = getattr(out, ("means", "log_scales", "quats", "opacity_logit", "sh")[i])[:n2]
            m_new, v_new = self.m[i][par], self.v[i][par]
            m_new[flagged_parents] = 0
            v_new[flagged_parents] = 0
            m_new[n:] = 0
            v_new[n:] = 0
            self.params[i] = new.clone().requires_grad_(True)
            self.m[i], self.v[i] = m_new.contiguous(), v_new.contiguous()
        self.log.append({"step": t, "densify": True, "split": split, "gaussians": n2,
                         "lambda_min_min": float(lam.min().item()) if n else 0.0})
        self._alloc(n2)
        self.step_graphs = None                     # captured again for the new buffers

    # -- checkpoint / resume ------------------------------------------------
    # The state between two steps of Algorithm 1: the Gaussians, their Adam
    # moments and step count, the splitting-matrix and gradient accumulators
    # with the number of steps they hold, and the log.  The loop draws no
    # random numbers, so this is all a resumed run needs.
    _FIELDS = ("params", "m", "v")

    def state_dict(self) -> dict:
        c = lambda t: None if t is None else t.detach().clone()    # noqa: E731
        return {"params": [c(p) for p in self.params], "m": [c(t) for t in self.m], "v": [c(t) for t in self.v],
                "adam_t": self.adam_t, "S": c(self.S), "S_po": c(self.S_po), "S_ls": c(self.S_ls),
                "G": c(self.G), "n_accum": self.n_accum, "log": [dict(r) for r in self.log],
                "sh_degree": self.sh_degree, "dim_theta": self.cfg.dim_theta}

    def load_state_dict(self, sd: dict):
        if sd["sh_degree"] != self.sh_degree or sd["dim_theta"] != self.cfg.dim_theta:
            raise ValueError("checkpoint: SH degree or dim Theta differs from this trainer's")
        dev = self.params[0].device
        self.params = [p.to(dev).clone().requires_grad_(True) for p in sd["params"]]
        self._alloc(self.n)
        self.m = [t.to(dev).clone() for t in sd["m"]]
        self.v = [t.to(dev).clone() for t in sd["v"]]
        self.adam_t = int(sd["adam_t"])
        for name in ("S", "S_po", "S_ls", "G"):
            if sd[name] is not None:
                getattr(self, name).copy_(sd[name].to(dev))
        self.n_accum = int(sd["n_accum"])
        self.log = [dict(r) for r in sd["log"]]
        self.step_graphs = None                     # captured again for these buffers

    def save(self, path: str, step: int):
        """Checkpoint after `step` (1-based) steps."""
        torch.save({"step": int(step), "state": self.state_dict()}, path)

    def restore(self, path: str) -> int:
        """Loads a checkpoint; returns the number of steps it holds (resume at
        that step + 1)."""
        ck = torch.load(path, map_location=self.params[0].device, weights_only=False)
        self.load_state_dict(ck["state"])
        return int(ck["step"])

    def run(self, steps: int | None = None, log_path: str | None = None, first_step: int = 1,
            checkpoint_path: str | None = None, checkpoint_every: int = 0):
        """Steps first_step .. steps (1-based; first_step > 1 after restore);
        with checkpoint_path and checkpoint_every, a checkpoint is written after
        every checkpoint_every-th step."""
        steps = steps or self.cfg.steps
        t0 = time.perf_counter()
        for t in range(first_step, steps + 1):
            self.step(t)
            if checkpoint_path and checkpoint_every and t % checkpoint_every == 0:
                self.save(checkpoint_path, t)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if log_path:
            with open(log_path, "w") as f:
                for rec in self.log:
                    f.write(json.dumps(rec) + "\n")
        return wall


def offset_views_problem(n: int = 4096, size: int = 128, device="cuda"):
    """Differentiation/training workload: tiny-scene distributions with n
    Gaussians, four size x size views at the origin shifted by (+-0.25,
    +-0.25, 0), targets rendered from a hidden scene (seed 1) of the same size."""
    import synth
    scene = synth.tiny_scene(0, n)
    hidden = synth.tiny_scene(1, n)
    cams = synth.offset_cameras(size, size, float(size))
    st = synth.Settings()
    hg = B.GaussianTensors.from_scene(hidden, device)
    targets = []
    for c in cams:
        vb = PL.ViewBuffers.alloc(hidden.n, c, st, device=device)
        targets.append(PL.render(hg, vb).clone())
    return B.GaussianTensors.from_scene(scene, device), cams, targets, st


def run_training(steps: int = 2000, log_path: str | None = None, **cfg_kw) -> dict:
    g, cams, targets, st = offset_views_problem()
    tr = SteepGSTrainer(g, cams, targets, st, TrainConfig(steps=steps, **cfg_kw))
    wall = tr.run(steps, log_path)
    losses = [r["loss"] for r in tr.log if "loss" in r]
    splits = [r for r in tr.log if r.get("densify")]
    return {"steps": steps, "wall_s": wall, "ms_per_step": 1e3 * wall / steps, "loss_first": losses[0],
            "loss_last": losses[-1], "gaussians_first": g.n, "gaussians_last": tr.n, "densify_events": len(splits),
            "splits": [s["split"] for s in splits]}


if __name__ == "__main__":
    import sys
    out = run_training(int(sys.argv[1]) if len(sys.argv) > 1 else 2000,
                      sys.argv[2] if len(sys.argv) > 2 else None)
    print(json.dumps(out))
