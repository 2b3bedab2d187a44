"""Benchmark of the fused SteepGS fwd+bwd+splitting iteration on GB300.

Workload: scene-scale single view -- 1,000,000 Gaussians from the 64-cluster
mixture (SH degree 3), one 1237x822 view at distance 6, 16x16 tiles, L1 loss
to a uniform-random target, then the minimum-eigenpair split at
lambda_min < 0.  A step = one fused iteration: project, bin_sort, render_fwd,
l1_loss_grad, render_bwd_with_splitting, densify_split (all in libsteepgs).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Prints one JSON line (rank 0).  N>1 (torchrun) runs N independent replicas
("replicas only": the path has no exchange step on one view).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "fwd+bwd+splitting ms/iter @1M Gaussians; render frames/s + p50/p99 ms"
N_GAUSS = 1_000_000
WIDTH, HEIGHT = 1237, 822
SCENE_SEED, TARGET_SEED = 0, 1
EPS_SPLIT = 0.0
WORKLOAD = "scene-scale single view: 1M Gaussians (64-cluster mixture, SH3), 1237x822, 16x16 tiles"

# FP32 operations per pixel-Gaussian pair, counted from render.cu (FMA = 2).
OPS_FWD_COMPOSITED = 28      # offset, quadratic form, exp, alpha, T update, 3 colour FMAs
OPS_BWD_COMPOSITED = 68      # + T division, dL/dalpha, colour behind, 9 gradient and 4 split terms
OPS_PROJ_BWD = 420           # projection adjoint + S lift per visible Gaussian (counted)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock

# DRAM traffic of one render_bwd_with_splitting call on this workload (its three
# launches: zero_reached_rows_kernel, render_bwd_walk_kernel<16,16,0> and
# project_bwd_kernel<3,0,0,0>), dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture, valid only for the sources it was taken from (first 16 hex
# digits of the SHA-256 of render.cu, project.cu and api.cu, concatenated).
RENDER_BWD_TRAFFIC = {"bytes": (4_009_472 + 149_760) + (121_743_104 + 7_667_712) + (173_870_080 + 205_750_016),
                      "sources_sha256": "0b68179a1da1023d",
                      "profile": "profiles/render_bwd_scene_1M_1237x822.md"}
TRAFFIC_SOURCES = ("render.cu", "project.cu", "api.cu")


def _sources_sha():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2505_05587_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _render_bwd_traffic():
    try:
        sha = _sources_sha()
    except OSError:
        return None
    return RENDER_BWD_TRAFFIC["bytes"] if sha == RENDER_BWD_TRAFFIC["sources_sha256"] else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the GPU works."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 20):
        self.index, self.period = index, period_ms
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", f"-lms={self.period}"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        busy = [s for s in sm if mx is None or s > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# Algorithmic bytes of one fused iteration at SH degree 3 (236 B of parameters
# per Gaussian): every array the method needs, read or written once.  Atomics,
# extra sort passes and re-reads are implementation cost and are not counted.
# Rows: (stage, bytes per Gaussian, per instance, per pixel, per tile).
ALGORITHMIC_BYTES = (
    ("project: parameters read (236), projected state written (48)", 284, 0, 0, 0),
    ("instance offsets: tile counts read, offsets written", 8, 0, 0, 0),
    ("keys: (tile, depth) key and id written", 0, 12, 0, 0),
    ("sort: one read and one write of each key-id pair", 0, 24, 0, 0),
    ("tile ranges: keys read, [start, end) per tile written", 0, 8, 0, 8),
    ("forward: instance record read (40); colour, T, last contributor written (20)", 0, 40, 20, 0),
    ("L1 loss: colour and target read, dL/dC written", 0, 0, 36, 0),
    ("backward: instance record read; dL/dC, T, last contributor read; 2-D gradients (36) and "
     "splitting moments (16) written", 52, 40, 20, 0),
    ("projection adjoint and lift: parameters, projected state, 2-D sums read (336); gradients (236) "
     "and the splitting matrix (24) written", 596, 0, 0, 0),
)


def algorithmic_bytes(n, m, p, t):
    """Bytes each array of the iteration is read or written once (SH degree 3):
    940 n + 124 m + 76 p + 8 t for n Gaussians, m instances, p pixels, t tiles."""
    per = [sum(row[k] for row in ALGORITHMIC_BYTES) for k in (1, 2, 3, 4)]
    return per[0] * n + per[1] * m + per[2] * p + per[3] * t


def max_over_ranks(values, world, device):
    """Per-rank timings -> the maximum over all ranks (every rank gets it).
    The replicas' step time is the slowest replica's."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(ms_step_max, world):
    """Whole-job figure for the ms/iter metric: N replicas each finish one
    iteration per slowest-replica step time, so the job completes an iteration
    every ms_step_max / N milliseconds."""
    return ms_step_max / max(world, 1)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2505_05587_gb300 import binding as B
    from paper_2505_05587_gb300 import pipeline as PL

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.lib()

    scene = synth.cluster_scene(SCENE_SEED, N_GAUSS, 3)
    cam = synth.scene_camera(WIDTH, HEIGHT)
    st = synth.Settings()
    target_np = synth.target_image(TARGET_SEED, HEIGHT, WIDTH)
    g = B.GaussianTensors.from_scene(scene, dev)
    target = torch.as_tensor(target_np).to(dev)
    vb = PL.ViewBuffers.alloc(g.n, cam, st, capacity=4 * g.n, device=dev, walk=not args.no_walk)
    db = PL.DensifyBuffers.alloc(g, dim_theta=args.dim_theta)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # warm-up (the first call also sizes the instance buffers)
    PL.fused_iteration(g, [vb], [target], db, eps_split=EPS_SPLIT, stream=stream, check_capacity=True,
                       lambda_dssim=args.lambda_dssim)
    for _ in range(max(args.warmup - 1, 0)):
        PL.fused_iteration(g, [vb], [target], db, eps_split=EPS_SPLIT, stream=stream, check_capacity=False,
                           lambda_dssim=args.lambda_dssim)
    torch.cuda.synchronize(dev)
    M = B.check_count(int(vb.bins.count.item()))
    n_out = int(db.n_out.item())

    if args.lambda_dssim is None:                      # the L1 loss fused into the forward kernel
        fwd_names = ["render_fwd_l1"]
        fwd_calls = [lambda s: B.render_fwd_l1(vb.proj, vb.bins, cam, st, target, 1, vb.image, vb.final_T,
                                               vb.n_contrib, vb.dL, db.loss, s)]
    else:
        fwd_names = ["render_fwd", "ssim_l1_loss_grad"]
        fwd_calls = [lambda s: B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib, s),
                     lambda s: vb.loss_grad(target, 1, db.loss, args.lambda_dssim, s)]
    names = ["clear_loss", "project", "bin_sort", *fwd_names, "render_bwd_with_splitting", "densify_split"]
    NC = len(names)
    calls = [
        lambda s: db.zero_(grads=False, S=False, stream=s),   # the loss (a memset); the backward writes grads and S
        lambda s: B.project(g, cam, st, vb.proj, s),
        lambda s: B.bin_sort(vb.proj, g.n, cam, st, vb.bins, vb.sort_ws, s),
        *fwd_calls,
        lambda s: B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, vb.dL,
                                              db.grads, db.S, db.bwd_ws, s, accumulate=False, S_po=db.S_po,
                                              S_ls=db.S_ls, reset_S=True),
        lambda s: B.densify_split(g, db.S, 1.0, EPS_SPLIT, 1.0, None, 0.0, db.out, db.capacity, db.n_out,
                                  db.parent, db.lam, db.v, db.split_ws, s, S_po=db.S_po, S_ls=db.S_ls),
    ]

    # the fused iteration captured as one CUDA graph (the timed step), and each
    # call captured as its own graph (the per-call breakdown); library launches
    # are counted while capturing, since replays bypass the host-side counter
    step_graph = PL.FusedIterationGraph(g, [vb], [target], db, eps_split=EPS_SPLIT,
                                        lambda_dssim=args.lambda_dssim)
    l1 = B.kernel_launches()
    cap = torch.cuda.Stream(dev)
    call_graphs = []
    for c in calls:
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=cap):
            c(cap)
        call_graphs.append(cg)
    l2 = B.kernel_launches()
    launches_per_step = l2 - l1             # the per-call captures hold one iteration's launches
    torch.cuda.synchronize(dev)

    K = args.steps
    ev_step = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(NC + 1)] for _ in range(K)]
    sampler = ClockSampler(local)
    with sampler:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()                     # L2 flush between iterations, outside the events
            ev_step[k][0].record(stream)
            step_graph.replay()
            ev_step[k][1].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - wall0
        if world > 1:
            dist.barrier()
        # per-call breakdown: the same calls, one graph each, events between them
        for k in range(K):
            flush.zero_()
            evs[k][0].record(stream)
            for i, cg in enumerate(call_graphs):
                cg.replay()
                evs[k][i + 1].record(stream)
        torch.cuda.synchronize(dev)
        # the same iteration issued call by call from the host (no graph)
        eager_ms = []
        for k in range(max(K // 2, 3)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for c in calls:
                c(stream)
            e1.record(stream)
            e1.synchronize()
            eager_ms.append(e0.elapsed_time(e1))

        # end-to-end through the public API: pinned host inputs in, the graph
        # replayed, loss and count out
        host = [t.detach().cpu().pin_memory() for t in g.tensors()]
        host_tgt = target.detach().cpu().pin_memory()
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        nout_host = torch.empty(1, dtype=torch.int32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host) + host_tgt.numel() * 4
        serial_ms = []                        # copy, iterate, read back: one iteration at a time
        for k in range(max(K // 2, 3)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for dst, src in zip(g.tensors(), host):
                dst.copy_(src, non_blocking=True)
            target.copy_(host_tgt, non_blocking=True)
            step_graph.replay()
            loss_host.copy_(db.loss, non_blocking=True)
            nout_host.copy_(db.n_out, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            serial_ms.append(e0.elapsed_time(e1))
        # streamed: iteration k + 1's inputs are copied while iteration k runs
        pre = PL.PrefetchedIterations(g, [vb], [target], db, eps_split=EPS_SPLIT, lambda_dssim=args.lambda_dssim)
        pre.run(host, [host_tgt], 2, stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pre.copy_stream.wait_stream(stream)
        pre.run(host, [host_tgt], K, stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms = [e0.elapsed_time(e1) / K]
    clocks = sampler.summary()

    per_call = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(NC)] for k in range(K)])
    step_ms = np.array([ev_step[k][0].elapsed_time(ev_step[k][1]) for k in range(K)])
    ms_iter = float(step_ms.mean())
    e2e = float(np.mean(e2e_ms))
    ms_iter, e2e = max_over_ranks([ms_iter, e2e], world, dev)

    # work units of the dominant launch (outside the timed region)
    counts = torch.empty(HEIGHT, WIDTH, 2, dtype=torch.int32, device=dev)
    B.render_stats(vb.proj, vb.bins, cam, st, counts, stream)
    torch.cuda.synchronize(dev)
    c = counts.to(torch.int64)
    ev_fwd, comp = int(c[..., 0].sum()), int(c[..., 1].sum())
    ev_bwd = int(vb.n_contrib.to(torch.int64).sum())
    n_vis = int((vb.proj.tiles_touched > 0).sum())
    call_ms = per_call.mean(0)
    dom = int(np.argmax(call_ms))
    # algorithmic work = composited pairs (the pairs the method needs); pairs an
    # implementation evaluates and then skips are its own overhead
    flops_bwd = comp * OPS_BWD_COMPOSITED + n_vis * OPS_PROJ_BWD
    flops_fwd = comp * OPS_FWD_COMPOSITED
    hbm_peak, peak_kind = _peaks()
    T = B.num_tiles(cam, st)
    P = WIDTH * HEIGHT
    alg_bytes = algorithmic_bytes(N_GAUSS, M, P, T)
    if names[dom] in ("render_fwd", "render_fwd_l1"):
        achieved = flops_fwd / (call_ms[dom] * 1e-3) / 1e12
    else:
        dom = names.index("render_bwd_with_splitting")
        achieved = flops_bwd / (call_ms[dom] * 1e-3) / 1e12
    # attainable FP32 rate on this GPU: FMA probe (outside the timed region)
    probe_blocks, probe_iters = 152 * 8, 20000
    probe_out = torch.empty(probe_blocks * 256, device=dev)
    B.fma_probe(probe_out, probe_blocks, 2000, stream)
    fma_ms = []
    for _ in range(3):
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        B.fma_probe(probe_out, probe_blocks, probe_iters, stream)
        p1.record(stream)
        p1.synchronize()
        fma_ms.append(p0.elapsed_time(p1))
    fma_tflops = probe_blocks * 256 * probe_iters * 16 / (min(fma_ms) * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": names[dom], "achieved": round(achieved, 3),
                "peak": round(FP32_PEAK_TFLOPS, 2), "unit": "TFLOP/s",
                "frac": round(achieved / FP32_PEAK_TFLOPS, 4),
                "traffic": args.traffic if args.traffic is not None else (
                    _render_bwd_traffic() if names[dom] == "render_bwd_with_splitting" else None),
                "traffic_unit": "DRAM bytes per render_bwd_with_splitting call (ncu: its three launches)",
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "peak_check": {"fma_probe_tflops": round(fma_tflops, 2),
                               "what": "sgs_fma_probe: 1216 blocks x 256 threads x 8 independent FMA chains"},
                "work": {"pairs_evaluated_fwd": ev_fwd, "pairs_evaluated_bwd": ev_bwd,
                         "pairs_composited": comp, "visible_gaussians": n_vis}}
    hbm = {"bytes_per_iter": alg_bytes, "achieved": round(alg_bytes / (ms_iter * 1e-3) / 1e9, 1),
           "peak": hbm_peak, "unit": "GB/s", "frac": round(alg_bytes / (ms_iter * 1e-3) / 1e9 / hbm_peak, 4),
           "peak_kind": peak_kind}

    result = {
        "metric": METRIC, "value": round(job_value(ms_iter, world), 4), "unit": "ms/iter", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_iter, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT,
                   "sh_degree": 3, "tile": "16x16", "instances_M": M, "n_out": n_out,
                   "dim_theta": args.dim_theta,
                   "loss": "L1" if args.lambda_dssim is None else f"(1-{args.lambda_dssim:g}) L1 + "
                                                                 f"{args.lambda_dssim:g} (1-SSIM)",
                   "backward_walk": "culled list entries" if args.no_walk else "forward's walk lists",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "256 MiB buffer written between iterations, outside the timed events"},
        "timing": "each step = one replay of the fused iteration captured as a CUDA graph; per_call_ms from "
                  "the calls captured one graph each, events between them",
        "per_call_ms": {nm: round(float(v), 4) for nm, v in zip(names, call_ms)},
        "eager_ms_per_step": round(float(np.mean(eager_ms)), 4),
        "wall_ms_per_step": round(wall * 1e3 / K, 4),
        "roofline": roofline, "hbm_roofline": hbm,
        "e2e": {"value": round(job_value(e2e, world), 4), "unit": "ms/iter", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": 8,
                "how": f"{K} iterations through pipeline.PrefetchedIterations: every iteration's parameters and "
                       "target copied from pinned host memory (iteration k + 1's copy overlapping iteration k), "
                       "its loss and split count read back; inputs larger than L2",
                "serial_ms_per_step": round(float(np.mean(serial_ms)), 4)},
        "gpu_launches": int(launches_per_step * K),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_serving:
        result["serving"] = bench_serving(local, args.serve_requests)
    if rank == 0 and world == 1 and not args.no_batched:
        result["batched"] = bench_batched(local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline_full()
        if not (args.no_serving and args.no_batched):
            result["cpu_baseline"]["workloads"] = oracle_workloads()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# The metric's second half (render serving) and the batched densification
# step, each with its own clock record
# ---------------------------------------------------------------------------
def bench_serving(local: int, n_requests: int) -> dict:
    """Render serving: Poisson arrivals at 200 req/s over the 6 resident scenes
    (100k-3M Gaussians, SH3) at 640x480 / 1237x822 / 1920x1080; continuous
    batching against one request per launch, in real time (the configured
    load) and saturated (every request released at once)."""
    import torch

    from paper_2505_05587_gb300 import serve as SV
    st = synth.Settings()
    scenes = SV.resident_scenes()
    jobs = SV.serving_requests(3, n_requests, 200.0, len(scenes))
    warm = SV.serving_requests(99, 200, 200.0, len(scenes))
    server = SV.RenderServer(scenes, st)
    server.run(warm, realtime=False)                # warm-up: buffers, instance estimates
    SV.serve_one_per_launch(scenes, st, warm, realtime=False)
    torch.cuda.synchronize()
    out = {"workload": f"render serving: {n_requests} requests (Poisson 200 req/s, seed 3), 6 resident scenes "
                       "(100k, 300k, 1M, 1M, 2M, 3M Gaussians, SH3), 640x480 / 1237x822 / 1920x1080, 16x16 tiles",
           "latency": "arrival to completion on the host clock; p50/p99 over the requests"}
    sat = jobs[:max(n_requests // 2, 1)]
    for name, fn in (("continuous_batching_realtime", lambda: server.run(jobs, realtime=True)),
                     ("one_per_launch_realtime", lambda: SV.serve_one_per_launch(scenes, st, jobs, realtime=True)),
                     ("continuous_batching_saturated", lambda: server.run(sat, realtime=False)),
                     ("one_per_launch_saturated", lambda: SV.serve_one_per_launch(scenes, st, sat,
                                                                                   realtime=False))):
        server.stats.clear()
        sampler = ClockSampler(local)
        with sampler:
            r = fn()
        r["clocks"] = sampler.summary()
        out[name] = r
    out["saturated_speedup"] = round(out["continuous_batching_saturated"]["frames_per_s"] /
                                     out["one_per_launch_saturated"]["frames_per_s"], 3)
    del server, scenes
    torch.cuda.empty_cache()
    return out


def bench_batched(local: int, steps: int = 20, warmup: int = 3) -> dict:
    """Batched densification step: 3M Gaussians, 8 ring views of uneven
    resolution, one persistent pass per step replayed as a CUDA graph, against
    the same step one view per launch sequence.  Tile 16x16 and staging batch
    256, the autotuner's choice on this workload (python -m
    paper_2505_05587_gb300.batched runs the tuner)."""
    import torch

    from paper_2505_05587_gb300 import batched as BT
    from paper_2505_05587_gb300 import binding as B
    scene = synth.cluster_scene(0, 3_000_000, 3)
    cams = synth.ring_cameras(6.0)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    del scene
    tgs = [torch.as_tensor(synth.target_image(10 + k, c.height, c.width)).cuda() for k, c in enumerate(cams)]
    step = BT.BatchedDensifyStep(g, cams, BT.concat_images(tgs), st, batch=256)
    step.capture()
    sampler = ClockSampler(local)
    with sampler:
        ms_graph = BT.time_fn(step.replay, reps=steps, warmup=warmup)
    clk_b = sampler.summary()
    M, n_out = int(step.count.item()), int(step.db.n_out.item())
    del step
    torch.cuda.empty_cache()
    plain = BT.PlainDensifyStep(g, cams, tgs, st)
    sampler = ClockSampler(local)
    with sampler:
        ms_plain = BT.time_fn(plain.run, reps=steps, warmup=warmup)
    clk_p = sampler.summary()
    del plain, g
    torch.cuda.empty_cache()
    return {"workload": "batched densification step: 3M Gaussians (cluster mixture, SH3), 8 ring views 1957x1091, "
                        "1600x1060, 1237x822, 980x545 x2, 800x600 x3 (7,356,101 pixels), 16x16 tiles, batch 256",
            "instances_M": M, "n_out": n_out, "unit": "ms/step", "steps": steps, "warmup": warmup,
            "batched_graph_ms": round(ms_graph, 4), "one_view_per_launch_ms": round(ms_plain, 4),
            "speedup": round(ms_plain / ms_graph, 3), "clocks": {"batched": clk_b, "one_view_per_launch": clk_p}}


# ---------------------------------------------------------------------------
# CPU oracle timings
# ---------------------------------------------------------------------------
def _oracle_iteration(scene, cam, st, target, rows=None, all_cores=False):
    """One oracle fused iteration (the splitting matrix over the position, as
    the GPU arm computes); rows = (y0, h) restricts the pixel work to those
    rows of the same view (projection, binning, eigen-solve and split still
    cover the whole scene); all_cores: rows dealt to every host thread."""
    import oracle
    r = oracle.render(scene, cam, st, rows=rows, all_cores=all_cores)
    tgt = target if rows is None else target[rows[0]:rows[0] + rows[1]]
    _, g = oracle.l1_loss_grad(r["image"], tgt)
    acc = oracle.backward(scene, cam, st, g, rows=rows, all_cores=all_cores, blocks=False)
    lam, v = oracle.eig3_min(acc["S"])
    oracle.split(scene, lam, v, EPS_SPLIT, 1.0)


def cpu_baseline_full():
    """The float64 oracle on one full iteration of the same workload, on all
    host cores (OpenMP over rows) and on one thread."""
    import oracle
    scene = synth.cluster_scene(SCENE_SEED, N_GAUSS, 3)
    cam = synth.scene_camera(WIDTH, HEIGHT)
    tgt = synth.target_image(TARGET_SEED, HEIGHT, WIDTH)
    t0 = time.perf_counter()
    _oracle_iteration(scene, cam, synth.Settings(), tgt, all_cores=True)
    dt_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    _oracle_iteration(scene, cam, synth.Settings(), tgt)
    dt_one = time.perf_counter() - t0
    return {"value": round(dt_all * 1e3, 1), "unit": "ms/iter", "cores": oracle.threads(), "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": "one full fused iteration of the same workload (float64 C oracle, rows dealt to all host "
                      "threads; projection and binning serial)",
            "single_thread": {"value": round(dt_one * 1e3, 1), "unit": "ms/iter", "cores": 1,
                              "sample": "the same full iteration on one thread"}}


def oracle_workloads(n_requests: int = 20) -> dict:
    """The float64 oracle, on all host threads, on the two other workloads:
    the batched densification step (3M Gaussians, the 8 ring views rendered,
    L1 over the views, the backward with the splitting matrices summed over
    them, the eigenpairs and the split) once, and `n_requests` requests of
    the serving stream (seed 3: scene, pose and resolution drawn as the GPU
    run draws them) rendered one by one.  Timings only (nothing is compared):
    the CPU baselines beside the GPU figures."""
    import oracle
    st = synth.Settings()
    scene = synth.cluster_scene(0, 3_000_000, 3)
    cams = synth.ring_cameras(6.0)
    tgs = [synth.target_image(10 + k, c.height, c.width) for k, c in enumerate(cams)]
    t0 = time.perf_counter()
    acc = None
    for cam, tgt in zip(cams, tgs):
        r = oracle.render(scene, cam, st, all_cores=True)
        _, g = oracle.l1_loss_grad(r["image"], tgt, n_views=len(cams))
        acc = oracle.backward(scene, cam, st, g, acc=acc, all_cores=True, blocks=False)
    lam, v = oracle.eig3_min(acc["S"])
    oracle.split(scene, lam, v, EPS_SPLIT, 1.0)
    t_batched = time.perf_counter() - t0
    del scene, acc
    sizes = (100_000, 300_000, 1_000_000, 1_000_000, 2_000_000, 3_000_000)
    reqs = synth.request_stream(3, n_requests, 200.0, len(sizes))
    used = sorted({r.scene for r in reqs})
    scenes = {k: synth.cluster_scene(10 + k, sizes[k], 3) for k in used}
    per = []
    for r in reqs:
        t0 = time.perf_counter()
        oracle.render(scenes[r.scene], r.camera, st, all_cores=True)
        per.append(time.perf_counter() - t0)
    return {"kind": "oracle", "cores": oracle.threads(), "nproc": os.cpu_count(),
            "batched_step": {"value": round(t_batched, 2), "unit": "s/step",
                             "sample": "the whole step once: 3M Gaussians, 8 ring views (1957x1091, 1600x1060, "
                                       "1237x822, 980x545 x2, 800x600 x3), render, L1, backward with splitting "
                                       "matrices, eigenpairs, split (projection and binning serial)"},
            "serving": {"value": round(1e3 * float(np.mean(per)), 1), "unit": "ms/frame",
                        "requests": n_requests, "min_ms": round(1e3 * min(per), 1),
                        "max_ms": round(1e3 * max(per), 1),
                        "sample": f"the first {n_requests} requests of the serving stream (seed 3), each "
                                  "rendered alone (forward only)"}}


def run_reference(args):
    """Oracle arm, on all host cores.  When the whole run of full iterations
    fits about three minutes (the first full iteration tells), every step is
    one full fused iteration of the oracle, timed as it runs.  Otherwise each
    step runs the oracle's fused iteration on the full scene for a horizontal
    strip of rows, and the per-iteration time of a step is extrapolated along
    the line t(rows) = c + b rows through a one-row strip's time and the
    step's own, beside the measured full iteration."""
    import oracle
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scene = synth.cluster_scene(SCENE_SEED, N_GAUSS, 3)
    cam = synth.scene_camera(WIDTH, HEIGHT)
    st = synth.Settings()
    tgt = synth.target_image(TARGET_SEED, HEIGHT, WIDTH)
    t0 = time.perf_counter()
    _oracle_iteration(scene, cam, st, tgt, all_cores=True)         # also the first warm-up step
    full = time.perf_counter() - t0
    steps = args.steps + args.warmup
    if full * (steps - 1) <= 180.0:
        meas = []
        for k in range(1, steps):
            t0 = time.perf_counter()
            _oracle_iteration(scene, cam, st, tgt, all_cores=True)
            if k >= args.warmup:
                meas.append(time.perf_counter() - t0)
        v = float(np.mean(meas)) * 1e3
        sample = (f"per step: one full fused iteration of the workload (float64 C oracle, rows dealt to all host "
                  f"threads; projection and binning serial), {args.steps} measured after {args.warmup} warm-up")
        a = None
    else:
        t0 = time.perf_counter()
        _oracle_iteration(scene, cam, st, tgt, rows=(400, 1), all_cores=True)
        a = time.perf_counter() - t0
        budget = 120.0
        b_row = max(full - a, 1e-3) / HEIGHT
        rows = int((budget / steps - a) / b_row) // 16 * 16
        rows = max(16, min(HEIGHT // 16 * 16, rows))
        est = []
        for k in range(steps):
            y0 = (k * rows) % (HEIGHT - rows + 1) // 16 * 16
            t0 = time.perf_counter()
            _oracle_iteration(scene, cam, st, tgt, rows=(y0, rows), all_cores=True)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                est.append(a + (dt - a) * (HEIGHT - 1) / max(rows - 1, 1))
        v = float(np.mean(est)) * 1e3
        sample = (f"per step: full scene, rows of the view ({rows} per step, rotating), all host threads; "
                  f"t(rows) = c + b rows through a one-row strip ({a:.2f} s) and the step, extrapolated to {HEIGHT} rows")
    out = {"metric": METRIC, "value": round(v, 1), "unit": "ms/iter", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": WIDTH, "height": HEIGHT,
                      "sh_degree": 3, "tile": "16x16"},
           "cpu_baseline": {"value": round(v, 1), "unit": "ms/iter", "cores": oracle.threads(), "kind": "oracle",
                            "nproc": os.cpu_count(), "sample": sample, "measured": a is None,
                            "full_iteration_measured_ms": round(full * 1e3, 1)},
           "e2e": {"value": round(v, 1), "unit": "ms/iter", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the render-serving measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched densification step")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests in the real-time serving stream (the saturated run takes half of them)")
    ap.add_argument("--dim-theta", type=int, default=3, choices=[3, 4, 7],
                    help="splitting matrices over the position (3, the paper's experiments), (position, opacity) "
                         "(4) or (position, log-scales, opacity) (7)")
    ap.add_argument("--lambda-dssim", type=float, default=None,
                    help="add the SSIM term to the loss: (1 - l) L1 + l (1 - SSIM) (default: L1 only)")
    ap.add_argument("--no-walk", action="store_true",
                    help="no walk lists: the backward culls every list entry itself instead of following the "
                         "forward's per-warp lists of composited entries")
    ap.add_argument("--oracle-workloads", action="store_true",
                    help="time the float64 oracle (all host threads) on the batched step and on 20 serving requests, "
                         "print one JSON line and exit (no GPU work)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.oracle_workloads:
        print(json.dumps({"oracle_workloads": oracle_workloads()}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
