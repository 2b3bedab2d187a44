"""Differentiation pattern: the autograd Function's backward (the hand-written
adjoint) against float64 central differences and the oracle gradient on the
training workload (4,096 Gaussians, 128x128, 4 views), and the SteepGS
training loop (Algorithm 1) end to end."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402
from paper_2505_05587_gb300 import train as TR  # noqa: E402

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _autograd_grads(scene, cams, st, gs):
    """Gradient of sum_v <g_v, C_v> through RasterizeWithSplitting."""
    g = B.GaussianTensors.from_scene(scene)
    params = [t.clone().requires_grad_(True) for t in g.tensors()]
    S = torch.zeros(scene.n, 6, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    for cam, gv in zip(cams, gs):
        rc = TR.RenderContext(PL.ViewBuffers.alloc(scene.n, cam, st), S, ws, scene.sh_degree)
        img = TR.render(params, rc)
        img.backward(torch.as_tensor(gv.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return {f: p.grad.cpu().numpy().astype(np.float64) for f, p in zip(FIELDS, params)}, S.cpu().numpy()


def test_autograd_matches_oracle_gradient_offset_views():
    scene = synth.tiny_scene(0, 4096)
    cams = synth.offset_cameras(128, 128, 128.0)
    st = synth.Settings()
    rng = np.random.default_rng(5)
    gs = [rng.normal(size=(128, 128, 3)).astype(np.float32) / (128 * 128) for _ in cams]
    got, S = _autograd_grads(scene, cams, st, gs)
    acc = None
    for cam, gv in zip(cams, gs):
        acc = oracle.backward(scene, cam, st, gv.astype(np.float64), acc)
    for f in FIELDS:
        rel = np.linalg.norm(got[f] - acc[f]) / np.linalg.norm(acc[f])
        assert rel < 1e-4, (f, rel)
    So = acc["S"]
    up = np.stack([So[:, 0, 0], So[:, 0, 1], So[:, 0, 2], So[:, 1, 1], So[:, 1, 2], So[:, 2, 2]], 1)
    assert np.linalg.norm(S - up) / np.linalg.norm(up) < 1e-4


def test_autograd_central_differences_offset_views():
    """h = 1e-4 central differences of the float64 oracle render (smooth mode)
    against the float32 autograd gradient, on every parameter of a sample of
    Gaussians."""
    scene = synth.tiny_scene(0, 4096)
    cams = synth.offset_cameras(128, 128, 128.0)
    st = synth.Settings().smooth()
    rng = np.random.default_rng(6)
    gs = [rng.normal(size=(128, 128, 3)) / (128 * 128) for _ in cams]
    got, _ = _autograd_grads(scene, cams, st, gs)
    vis = np.nonzero(oracle.integer_stage(scene, cams[0], st)["tiles"])[0]
    sample = np.random.default_rng(7).choice(vis, 3, replace=False)
    h = 1e-4
    base_order = [oracle.bin_sort(scene, c, st)[1] for c in cams]

    def loss(sc):
        return sum(float(np.sum(oracle.render(sc, c, st)["image"] * gv)) for c, gv in zip(cams, gs))

    def same_order(sc):
        # the render is discontinuous where a step swaps two depths: skip those
        return all(np.array_equal(oracle.bin_sort(sc, c, st)[1], o) for c, o in zip(cams, base_order))

    fd, an = [], []
    for i in sample:
        for f in FIELDS:
            flat = getattr(scene, f).reshape(scene.n, -1)
            for k in range(flat.shape[1]):
                vals = []
                for sgn in (1, -1):
                    sc = scene.copy()
                    a = getattr(sc, f).reshape(scene.n, -1)
                    a[i, k] = np.float32(flat[i, k] + sgn * h)
                    if not same_order(sc):
                        break
                    vals.append((loss(sc), float(a[i, k])))
                if len(vals) < 2:
                    continue
                (lp, xp), (lm, xm) = vals
                fd.append((lp - lm) / (xp - xm))
                an.append(got[f].reshape(scene.n, -1)[i, k])
    fd, an = np.array(fd), np.array(an)
    assert fd.size >= 30
    rel = np.linalg.norm(fd - an) / np.linalg.norm(fd)
    assert rel < 1e-4, rel


def test_training_loop_densifies_and_reduces_loss():
    g, cams, targets, st = TR.offset_views_problem(n=1024, size=64)
    cfg = TR.TrainConfig(steps=400, start=200, T_split=100, log_every=20)
    tr = TR.SteepGSTrainer(g, cams, targets, st, cfg)
    tr.run()
    losses = [r["loss"] for r in tr.log if "loss" in r]
    events = [r for r in tr.log if r.get("densify")]
    assert len(events) == 3
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.95 * losses[0]
    assert tr.n == 1024 + sum(e["split"] for e in events) and tr.n > 1024
    for p in tr.params:
        assert bool(torch.isfinite(p).all())


@pytest.mark.parametrize("dim_theta,lam", [(4, None), (3, 0.2), (4, 0.2), (7, None)])
def test_training_loop_variants_theta4_and_ssim(dim_theta, lam):
    """Variants inside Algorithm 1: splitting over (position,
    opacity) or (position, log-scales, opacity) and the SSIM term in the
    loss."""
    g, cams, targets, st = TR.offset_views_problem(n=1024, size=64)
    cfg = TR.TrainConfig(steps=300, start=100, T_split=100, log_every=20, dim_theta=dim_theta, lambda_dssim=lam)
    tr = TR.SteepGSTrainer(g, cams, targets, st, cfg)
    tr.run()
    losses = [r["loss"] for r in tr.log if "loss" in r]
    events = [r for r in tr.log if r.get("densify")]
    assert len(events) == 3 and all(np.isfinite(losses))
    assert losses[-1] < 0.95 * losses[0]
    assert tr.n == 1024 + sum(e["split"] for e in events) and tr.n > 1024
    for p in tr.params:
        assert bool(torch.isfinite(p).all())
    o = torch.sigmoid(tr.params[3])
    assert bool(((o > 0) & (o < 1)).all())


def test_graphed_steps_follow_the_autograd_steps():
    """The trainer's captured-graph step and its autograd step take the same
    Adam trajectory (bias corrections and loss sums may round differently)."""
    runs = []
    for graphs in (False, True):
        g, cams, targets, st = TR.offset_views_problem(n=1024, size=64)
        cfg = TR.TrainConfig(steps=40, start=1000, T_split=100, log_every=10, graphs=graphs)
        tr = TR.SteepGSTrainer(g, cams, targets, st, cfg)
        tr.run()
        runs.append(tr)
    a, b = runs
    for pa, pb in zip(a.params, b.params):
        d = (pa.detach() - pb.detach()).double().norm() / pa.detach().double().norm()
        assert float(d) < 1e-4
    la = [r["loss"] for r in a.log if "loss" in r]
    lb = [r["loss"] for r in b.log if "loss" in r]
    assert len(la) == len(lb) and all(abs(x - y) <= 1e-4 * abs(x) for x, y in zip(la, lb))


def test_checkpoint_resume_continues_the_uninterrupted_run(tmp_path):
    """The training workload (4,096 Gaussians, four 128x128 views, SteepGS
    densification every 100 steps from step 500), checkpointed after step
    1050, halfway through an accumulation period: restored into a fresh
    trainer, every tensor of the state comes back bit for bit, and the resumed
    steps 1051..1400 continue the uninterrupted run.  Runs are not bit-exact
    repeats of one another (the backward's float atomics add in a
    run-dependent order, and training amplifies last-bit differences: two
    uninterrupted runs already differ by ~0.2% in Gaussian count at the first
    densification), so the count at the first densification after the resume
    is compared at 0.5%; restores that lose the splitting-matrix accumulator
    or the Adam moments miss it by 8% and 3%."""
    path = str(tmp_path / "ck.pt")
    g, cams, targets, st = TR.offset_views_problem()
    cfg = TR.TrainConfig(steps=1400, log_every=50)
    full = TR.SteepGSTrainer(g, cams, targets, st, cfg)
    full.run(checkpoint_path=path, checkpoint_every=1050)
    saved = torch.load(path, weights_only=False)
    assert saved["step"] == 1050 and saved["state"]["n_accum"] == 50

    res = TR.SteepGSTrainer(g, cams, targets, st, cfg)
    k = res.restore(path)
    assert k == 1050
    sd = res.state_dict()
    for key in ("params", "m", "v"):
        for a, b in zip(sd[key], saved["state"][key]):
            assert torch.equal(a.cpu(), b.cpu()), key
    for key in ("S", "G"):
        assert torch.equal(sd[key].cpu(), saved["state"][key].cpu()), key
    assert float(sd["S"].abs().sum()) > 0
    assert sd["adam_t"] == 1050 and sd["n_accum"] == 50 and sd["log"] == saved["state"]["log"]
    res.run(first_step=k + 1)

    ev_f = {r["step"]: r["gaussians"] for r in full.log if r.get("densify")}
    ev_r = {r["step"]: r["gaussians"] for r in res.log if r.get("densify")}
    assert sorted(ev_f) == sorted(ev_r) == list(range(500, 1401, 100))
    assert all(ev_f[s] == ev_r[s] for s in ev_f if s <= 1000)          # the restored history
    assert abs(ev_r[1100] - ev_f[1100]) <= 0.005 * ev_f[1100]
    for s in (1200, 1300, 1400):
        assert abs(ev_r[s] - ev_f[s]) <= 0.015 * ev_f[s]
    lf = [r["loss"] for r in full.log if "loss" in r]
    lr = [r["loss"] for r in res.log if "loss" in r]
    assert len(lf) == len(lr) and abs(lf[-1] - lr[-1]) <= 0.05 * lf[-1]
