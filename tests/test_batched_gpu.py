"""Batched pattern: several views of uneven resolution in one pass
(sgs_render_views_with_splitting), captured in a CUDA graph, against the CPU
oracle and against the one-view-per-launch form."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import batched as BT  # noqa: E402
from paper_2505_05587_gb300 import binding as B  # noqa: E402

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")
RES = [(150, 101), (96, 64), (77, 59)]


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def _problem(n=3000, res=RES, seed=3):
    scene = synth.cluster_scene(seed, n, 3)
    cams = synth.ring_cameras(6.0, res)
    tg = [synth.target_image(10 + k, h, w) for k, (w, h) in enumerate(res)]
    return scene, cams, tg


@pytest.mark.parametrize("tile,batch", [((16, 16), 256), ((8, 8), 64), ((32, 8), 128), ((16, 8), 256)])
def test_batched_views_match_oracle(tile, batch):
    scene, cams, tg = _problem()
    st = dataclasses.replace(synth.Settings(), tile_w=tile[0], tile_h=tile[1])
    g = B.GaussianTensors.from_scene(scene)
    targets = BT.concat_images([torch.as_tensor(t).cuda() for t in tg])
    step = BT.BatchedDensifyStep(g, cams, targets, st, batch=batch)
    step.fit_capacity()
    torch.cuda.synchronize()
    refs = [oracle.render(scene, c, st) for c in cams]
    img = step.images.cpu().numpy().astype(np.float64)
    off = 0
    acc = None
    loss = 0.0
    for c, r, t in zip(cams, refs, tg):
        P = c.width * c.height
        ok = ~r["band"].reshape(-1)
        assert np.abs(img[off:off + P] - r["image"].reshape(-1, 3))[ok].max() < 1e-5
        L, dL = oracle.l1_loss_grad(r["image"], t, len(cams))
        loss += L
        acc = oracle.backward(scene, c, st, dL, acc)
        off += P
    assert abs(step.loss.item() - loss) < 1e-5 * loss
    for f, t in zip(FIELDS, step.grads.tensors()):
        assert _rel(t.cpu().numpy(), acc[f]) < 1e-4, f
    assert _rel(step.S.cpu().numpy(), _upper6(acc["S"])) < 1e-4


def test_batched_equals_one_view_per_launch_and_graph_replay():
    scene, cams, tg = _problem(20000, [(320, 200), (200, 150), (160, 160), (96, 64)], seed=4)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    tgs = [torch.as_tensor(t).cuda() for t in tg]
    plain = BT.PlainDensifyStep(g, cams, tgs, st)
    plain.run()
    step = BT.BatchedDensifyStep(g, cams, BT.concat_images(tgs), st, batch=256)
    step.capture()
    step.images.zero_()
    step.replay()
    torch.cuda.synchronize()
    pimg = BT.concat_images([vb.image for vb in plain.views])
    assert torch.equal(step.images, pimg)
    for a, b in zip(step.grads.tensors(), plain.db.grads.tensors()):
        assert _rel(a.cpu().numpy(), b.cpu().numpy().astype(np.float64)) < 1e-5
    assert _rel(step.S.cpu().numpy(), plain.db.S.cpu().numpy().astype(np.float64)) < 1e-5
    assert abs(step.loss.item() - plain.db.loss.item()) < 1e-5 * plain.db.loss.item()
    # eigenvalues agree; decisions agree wherever lambda_min is clearly nonzero
    lam_b, lam_p = step.db.lam.cpu().numpy(), plain.db.lam.cpu().numpy()
    nrm = np.linalg.norm(plain.db.S.cpu().numpy(), axis=1)
    assert np.all(np.abs(lam_b - lam_p) <= 1e-4 * np.maximum(nrm, 1e-30))
    # graph replay equals an eager run (up to the order of the float atomics)
    grads_graph = [t.clone() for t in step.grads.tensors()]
    step.run_eager()
    torch.cuda.synchronize()
    for a, b in zip(grads_graph, step.grads.tensors()):
        assert _rel(a.cpu().numpy(), b.cpu().numpy().astype(np.float64)) < 1e-5


def test_autotuner_picks_a_valid_configuration():
    scene, cams, tg = _problem(5000, [(160, 120), (96, 64)], seed=5)
    g = B.GaussianTensors.from_scene(scene)
    targets = BT.concat_images([torch.as_tensor(t).cuda() for t in tg])
    st, batch, table = BT.autotune(g, cams, targets, synth.Settings(), reps=1, shapes=[(16, 16), (8, 8)],
                                   batches=[64, 256])
    assert len(table) == 4 and batch in (64, 256) and (st.tile_w, st.tile_h) in ((16, 16), (8, 8))
    assert all(r["ms"] > 0 for r in table)
