"""Splitting matrices over theta = (p, o) on the GPU (the position-opacity
block from the backward, the 4x4 minimum eigenpair and the split with
displaced half opacities) against the float64 oracle."""
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
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402

import split_parity as SP  # noqa: E402

CASES = [
    ("tiny", lambda: synth.tiny_scene(0), lambda: synth.camera_identity(64, 64, 64.0), synth.Settings()),
    ("cluster_sh3_lookat", lambda: synth.cluster_scene(3, 3000, 3),
     lambda: synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0), synth.Settings()),
    ("tile8x8_sh1", lambda: synth.cluster_scene(5, 800, 1),
     lambda: synth.camera_lookat((0.0, -1.0, -6.0), (0, 0, 0), 77, 59, 77.0), synth.Settings(tile_w=8, tile_h=8)),
]


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def _backward4(scene, cam, st):
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st)
    PL.project_and_sort(g, vb)
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    ref = oracle.render(scene, cam, st)
    _, dL_ref = oracle.l1_loss_grad(ref["image"], synth.target_image(2, cam.height, cam.width))
    dL = torch.as_tensor(dL_ref.astype(np.float32)).cuda().contiguous()
    grads = g.zeros_like()
    S = torch.zeros(scene.n, 6, device="cuda")
    S_po = torch.zeros(scene.n, 3, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                accumulate=False, S_po=S_po)
    torch.cuda.synchronize()
    acc = oracle.backward(scene, cam, st, dL_ref.astype(np.float32).astype(np.float64))
    return g, S, S_po, acc


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_position_opacity_block_parity(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    _, S, S_po, acc = _backward4(scene, cam, st)
    assert _rel(S_po.cpu().numpy(), acc["S_po"]) < 1e-4
    assert _rel(S.cpu().numpy(), _upper6(acc["S"])) < 1e-4


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_densify_theta4_parity(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    g, _, _, acc = _backward4(scene, cam, st)
    # the split reads the oracle's matrices as float32, so it is checked on its own
    S32 = acc["S"].astype(np.float32).astype(np.float64)
    Spo32 = acc["S_po"].astype(np.float32).astype(np.float64)
    S_gpu = torch.as_tensor(_upper6(S32).astype(np.float32)).cuda().contiguous()
    Spo_gpu = torch.as_tensor(Spo32.astype(np.float32)).cuda().contiguous()
    db = PL.DensifyBuffers.alloc(g, dim_theta=4)
    inv_T, step = 0.5, 0.3
    B.densify_split(g, S_gpu, inv_T, -1e-7, step, None, 0.0, db.out, db.capacity, db.n_out, db.parent, db.lam,
                    db.v, db.split_ws, S_po=Spo_gpu)
    torch.cuda.synchronize()
    S4 = oracle.S4_matrix(S32, Spo32)
    lam_o, v_o = oracle.eig_min_sym(S4, inv_T)
    lam_g, v_g = db.lam.cpu().numpy(), db.v.cpu().numpy()
    nrm = np.linalg.norm(S4.reshape(len(S4), -1), axis=1) * inv_T
    assert np.all(np.abs(lam_g - lam_o) <= 1e-4 * np.maximum(nrm, 1e-30))
    ev = np.linalg.eigvalsh(S4 * inv_T)
    gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
    assert gap.sum() > 10
    cosang = np.abs(np.sum(v_g * v_o, 1))
    assert np.all(1 - cosang[gap] <= 1e-4)
    decided = np.abs(lam_o + 1e-7) > 1e-6 * np.maximum(nrm, 1e-30)
    n = scene.n
    n_out = int(db.n_out.item())
    sp = oracle.split_po(scene, lam_o, v_o, -1e-7, step)
    out = SP.gpu_out(db, n_out)
    Sx = oracle.S4_matrix(acc["S"], acc["S_po"])                 # the oracle's own float64 matrices
    lam_x, _ = oracle.eig_min_sym(Sx, inv_T)
    structural = SP.structural_zeros(lam_x, np.linalg.norm(Sx.reshape(n, -1), axis=1) * inv_T, -1e-7)
    flags_g = SP.check_split(scene, out, db.parent.cpu().numpy(), n_out, lam_o, v_o, sp["flags"], decided, gap,
                             -1e-7, step, dim=4, v_gpu=v_g, structural=structural)
    assert flags_g.sum() > 0


def test_theta4_multi_view_sums_views():
    scene = synth.cluster_scene(3, 3000, 3)
    res = [(150, 101), (96, 64)]
    cams = synth.ring_cameras(6.0, res)
    st = synth.Settings()
    tg = [synth.target_image(10 + k, h, w) for k, (w, h) in enumerate(res)]
    g = B.GaussianTensors.from_scene(scene)
    step = BT.BatchedDensifyStep(g, cams, BT.concat_images([torch.as_tensor(t).cuda() for t in tg]), st,
                                 batch=128)
    step.fit_capacity()
    S_po = torch.zeros(scene.n, 3, device="cuda")
    step.S.zero_()
    step.loss.zero_()
    B.render_views_with_splitting(g, cams, st, 128, step.targets, step.images, step.loss, step.grads, False, step.S,
                                  step.count, step.capacity, step.ws, S_po=S_po)
    torch.cuda.synchronize()
    acc = None
    for c, t in zip(cams, tg):
        r = oracle.render(scene, c, st)
        _, dL = oracle.l1_loss_grad(r["image"], t, len(cams))
        acc = oracle.backward(scene, c, st, dL, acc)
    assert _rel(S_po.cpu().numpy(), acc["S_po"]) < 1e-4


def test_theta4_noalloc_equals_workspace_path():
    scene = synth.tiny_scene(0)
    g, S, S_po, _ = _backward4(scene, synth.camera_identity(64, 64, 64.0), synth.Settings())
    a = PL.DensifyBuffers.alloc(g, dim_theta=4)
    b = PL.DensifyBuffers.alloc(g, dim_theta=4)
    B.densify_split(g, S, 1.0, 0.0, 1.0, None, 0.0, a.out, a.capacity, a.n_out, a.parent, a.lam, a.v, a.split_ws,
                    S_po=S_po)
    B.densify_split_noalloc(g, S, 1.0, 0.0, 1.0, None, 0.0, b.out, b.capacity, b.n_out, b.parent, b.lam, b.v,
                            S_po=S_po)
    torch.cuda.synchronize()
    assert int(a.n_out.item()) == int(b.n_out.item())
    n2 = int(a.n_out.item())
    assert torch.equal(a.lam, b.lam) and torch.equal(a.v, b.v)
    for x, y in zip(a.out.tensors(), b.out.tensors()):
        assert torch.equal(x[:n2], y[:n2])
