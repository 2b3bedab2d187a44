"""The fused iteration captured as a CUDA graph: a replay gives what the
eager calls give (images bit for bit, accumulators to float32 atomics
reordering), reads the parameter buffers' current values, and every library
call it holds was capture-safe."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm().clamp_min(1e-30))


def _setup(dim_theta=3):
    scene = synth.cluster_scene(3, 3000, 3)
    res = [(150, 101), (96, 64)]
    cams = synth.ring_cameras(6.0, res)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    views = [PL.ViewBuffers.alloc(g.n, c, st) for c in cams]
    tg = [torch.as_tensor(synth.target_image(10 + k, h, w)).cuda() for k, (w, h) in enumerate(res)]
    db = PL.DensifyBuffers.alloc(g, dim_theta=dim_theta)
    return g, views, tg, db


def _snapshot(views, db):
    torch.cuda.synchronize()
    return dict(images=[vb.image.clone() for vb in views], S=db.S.clone(), loss=db.loss.clone(),
                grads=[t.clone() for t in db.grads.tensors()], n_out=int(db.n_out.item()),
                S_po=None if db.S_po is None else db.S_po.clone())


@pytest.mark.parametrize("dim_theta", [3, 4])
def test_graph_replay_equals_eager(dim_theta):
    g, views, tg, db = _setup(dim_theta)
    PL.fused_iteration(g, views, tg, db, eps_split=-1e-7)
    ref = _snapshot(views, db)
    graph = PL.FusedIterationGraph(g, views, tg, db, eps_split=-1e-7)
    for vb in views:                                  # the replay must rewrite every output
        vb.image.fill_(-1.0)
    db.S.fill_(123.0)
    db.loss.fill_(-5.0)
    for t in db.grads.tensors():
        t.fill_(7.0)
    graph.replay(check=True)
    got = _snapshot(views, db)
    for a, b in zip(got["images"], ref["images"]):
        assert torch.equal(a, b)
    assert _rel(got["S"], ref["S"]) < 1e-5
    assert _rel(got["loss"], ref["loss"]) < 1e-6
    for a, b in zip(got["grads"], ref["grads"]):
        assert _rel(a, b) < 1e-5
    if dim_theta == 4:
        assert _rel(got["S_po"], ref["S_po"]) < 1e-5
    assert abs(got["n_out"] - ref["n_out"]) <= 2     # flags at lambda ~ eps may flip under atomics noise


def test_graph_reads_current_parameter_values():
    g, views, tg, db = _setup()
    graph = PL.FusedIterationGraph(g, views, tg, db, eps_split=-1e-7)
    with torch.no_grad():
        g.means.add_(0.01)                            # move the scene in place
        g.opacity_logit.mul_(0.9)
    graph.replay(check=True)
    got = _snapshot(views, db)
    PL.fused_iteration(g, views, tg, db, eps_split=-1e-7)
    ref = _snapshot(views, db)
    for a, b in zip(got["images"], ref["images"]):
        assert torch.equal(a, b)
    assert _rel(got["S"], ref["S"]) < 1e-5


def test_zero_on_a_side_stream_orders_with_the_calls():
    g, views, tg, db = _setup()
    s = torch.cuda.Stream()
    db.S.fill_(1.0)
    with torch.cuda.stream(torch.cuda.current_stream()):
        PL.fused_iteration(g, views, tg, db, eps_split=-1e-7, stream=s)
    s.synchronize()
    ref = db.S.clone()
    db.S.fill_(1.0)
    PL.fused_iteration(g, views, tg, db, eps_split=-1e-7)
    torch.cuda.synchronize()
    assert _rel(ref, db.S) < 1e-5


def test_prefetched_iterations_match_eager_ones():
    """Streamed iterations (inputs of k + 1 copied during k) give each
    iteration's loss and split count as the eager calls on the same inputs."""
    g, views, tg, db = _setup()
    host_sets, host_tgts, ref = [], [], []
    for k in range(4):                                # four different parameter sets
        gk = B.GaussianTensors(*[t.clone() for t in g.tensors()], g.sh_degree)
        with torch.no_grad():
            gk.means.add_(0.003 * k)
            gk.opacity_logit.mul_(1.0 - 0.05 * k)
        PL.fused_iteration(gk, views, tg, db, eps_split=-1e-7)
        torch.cuda.synchronize()
        ref.append((float(db.loss.item()), int(db.n_out.item())))
        host_sets.append([t.cpu().pin_memory() for t in gk.tensors()])
        host_tgts.append([t.cpu().pin_memory() for t in tg])
    pre = PL.PrefetchedIterations(g, views, tg, db, eps_split=-1e-7)
    loss, nout = pre.run(host_sets, host_tgts, 4)
    torch.cuda.synchronize()
    for k in range(4):
        assert abs(float(loss[k]) - ref[k][0]) <= 1e-5 * abs(ref[k][0])
        assert abs(int(nout[k]) - ref[k][1]) <= 2
