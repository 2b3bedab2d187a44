"""The forward pass's walk lists and the backward pass that follows them.

For every warp of every tile the forward records the positions of the
tile's list entries that it composited in at least one of its 8x4 pixels.
Checked here: the forward's outputs do not change when it records; each list
holds exactly as many entries as the measurement walk (sgs_render_stats, a
walk over every list entry without culling) finds composited in some pixel
of the warp's block, in front-to-back order with each entry once; the
backward pass over the lists equals the backward pass that culls every list
entry itself, and both equal the oracle.
Also at the full benchmark size (1M Gaussians, 1237x822)."""
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

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")

CASES = [
    ("tiny", lambda: synth.tiny_scene(0), lambda: synth.camera_identity(64, 64, 64.0), synth.Settings()),
    ("ragged_70x45", lambda: synth.tiny_scene(7, 300), lambda: synth.camera_identity(70, 45, 60.0),
     synth.Settings()),
    ("cluster_sh3", lambda: synth.cluster_scene(3, 3000, 3),
     lambda: synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0), synth.Settings()),
    ("tile16x8", lambda: synth.tiny_scene(1), lambda: synth.camera_identity(64, 48, 64.0),
     synth.Settings(tile_w=16, tile_h=8)),
    ("tile32x8_bg", lambda: synth.cluster_scene(6, 1500, 2),
     lambda: synth.camera_lookat((2.0, 0.0, -5.5), (0, 0, 0), 96, 64, 96.0),
     synth.Settings(tile_w=32, tile_h=8, bg=(0.1, 0.2, 0.3))),
]


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def _views(scene, cam, st, capacity=None):
    g = B.GaussianTensors.from_scene(scene)
    out = []
    for walk in (True, False):
        vb = PL.ViewBuffers.alloc(scene.n, cam, st, capacity=capacity, walk=walk)
        PL.project_and_sort(g, vb)
        B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
        out.append(vb)
    torch.cuda.synchronize()
    return g, out


def _check_lists(vb, cam, st):
    """Every warp's list: as many entries as the measurement walk finds
    composited in some pixel of the warp's block (exactly), positions inside
    the tile's list, strictly increasing (front to back, each entry once);
    returns the number of recorded (warp, entry) pairs."""
    TW, TH = st.tile_w, st.tile_h
    NW = TW * TH // 32
    gx = (cam.width + TW - 1) // TW
    gy = (cam.height + TH - 1) // TH
    ranges = vb.bins.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    counts = vb.bins.walk_count.cpu().numpy().view(np.uint32)[:gx * gy * NW].astype(np.int64)
    walk = vb.bins.walk.cpu().numpy().view(np.uint32).astype(np.int64)
    # the measurement walk's per-block count of entries composited in some pixel
    stats = torch.empty(cam.height, cam.width, 2, dtype=torch.int32, device="cuda")
    uni = torch.empty(gx * gy * NW, dtype=torch.int32, device="cuda")
    B.render_stats(vb.proj, vb.bins, cam, st, stats, warp_union=uni)
    torch.cuda.synchronize()
    assert np.array_equal(counts, uni.cpu().numpy().astype(np.int64))
    total = 0
    for t in range(gx * gy):
        L = ranges[t, 1] - ranges[t, 0]
        c = counts[t * NW:(t + 1) * NW]
        assert np.all((c >= 0) & (c <= L))
        for w in range(NW):
            if c[w] == 0:
                continue
            base = NW * ranges[t, 0] + w * L
            pos = walk[base:base + c[w]]
            assert np.all(np.diff(pos) > 0) and pos[0] >= 0 and pos[-1] < L
        total += int(c.sum())
    return total


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_walk_lists_and_backward_over_them(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    g, (vw, vc) = _views(scene, cam, st)
    # the forward's outputs do not depend on recording the lists
    assert torch.equal(vw.image, vc.image) and torch.equal(vw.final_T, vc.final_T)
    assert torch.equal(vw.n_contrib, vc.n_contrib)
    assert _check_lists(vw, cam, st) > 0
    ref = oracle.render(scene, cam, st)
    _, dL_ref = oracle.l1_loss_grad(ref["image"], synth.target_image(2, cam.height, cam.width))
    dL = torch.as_tensor(dL_ref.astype(np.float32)).cuda().contiguous()
    acc = oracle.backward(scene, cam, st, dL_ref.astype(np.float32).astype(np.float64))
    res = []
    for vb in (vw, vc):
        grads = g.zeros_like()
        S = torch.zeros(scene.n, 6, device="cuda")
        S_po = torch.zeros(scene.n, 3, device="cuda")
        S_ls = torch.zeros(scene.n, 18, device="cuda")      # the higher-moment variant of both passes
        ws = B.workspace(B.render_bwd_workspace_size(scene.n))
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                    accumulate=False, S_po=S_po, S_ls=S_ls)
        torch.cuda.synchronize()
        res.append((grads, S, S_po, S_ls))
    for (grads, S, S_po, S_ls) in res:
        for f, t in zip(FIELDS, grads.tensors()):
            assert _rel(t.cpu().numpy(), acc[f]) < 1e-4, f
        assert _rel(S.cpu().numpy(), _upper6(acc["S"])) < 1e-4
        assert _rel(S_po.cpu().numpy(), acc["S_po"]) < 1e-4
        assert _rel(S_ls.cpu().numpy(), acc["S_ls"]) < 1e-4
    (ga, Sa, Pa, La), (gb, Sb, Pb, Lb) = res
    for a, b in ((Sa, Sb), (Pa, Pb), (La, Lb)):
        assert _rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
    for a, b in zip(ga.tensors(), gb.tensors()):       # the gradients' bar: atomics add in another order
        assert _rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-4


def test_walk_lists_full_size():
    """The benchmark view: every warp list against the measurement walk, and
    the two backward passes against each other (the oracle comparison at this
    size is in the full-size parity file)."""
    N, W, H = 1_000_000, 1237, 822
    scene = synth.cluster_scene(0, N, 3)
    cam = synth.scene_camera(W, H)
    st = synth.Settings()
    g, (vw, vc) = _views(scene, cam, st, capacity=4 * N)
    assert torch.equal(vw.image, vc.image) and torch.equal(vw.n_contrib, vc.n_contrib)
    total = _check_lists(vw, cam, st)
    assert 1_000_000 < total < int(vw.bins.count.item()) * 8
    dL = torch.as_tensor(synth.target_image(1, H, W)).cuda().sub_(vw.image).sign_().mul_(1.0 / (3 * H * W))
    out = []
    for vb in (vw, vc):
        grads = g.zeros_like()
        S = torch.zeros(N, 6, device="cuda")
        ws = B.workspace(B.render_bwd_workspace_size(N))
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                    accumulate=False)
        torch.cuda.synchronize()
        out.append((grads, S))
    assert _rel(out[0][1].cpu().numpy(), out[1][1].cpu().numpy()) < 1e-5
    for nm, a, b in zip(FIELDS, out[0][0].tensors(), out[1][0].tensors()):
        assert _rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-4, nm
