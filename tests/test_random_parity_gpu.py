"""Seeded random configurations, GPU path against the oracle through the C ABI.

Each seed draws a scene (the tiny uniform recipe or the cluster mixture, 40
to 4,000 Gaussians, SH degree 0-3), a camera (identity at the origin or a
look-at from 4-8 units), an image size from 9x7 up to 211x157 pixels (ragged
against every tile shape), one of the four tile shapes, the background and
the splitting threshold, then checks every stage of the path at the bars of
the other parity tests: binning bit for bit (keys, sorted ids, ranges), the
forward outside the threshold band, the backward's gradients and splitting
matrices (relative Frobenius 1e-4), and the split of the GPU's own matrices
(eigenvalues, and the compaction and offspring from the GPU's decisions).
"""
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

import split_parity as SP  # noqa: E402

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")
TILES = [(16, 16), (16, 8), (8, 8), (32, 8)]
SEEDS = list(range(12))


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    W = int(rng.integers(9, 212))
    H = int(rng.integers(7, 158))
    tw, th = TILES[int(rng.integers(0, len(TILES)))]
    bg = tuple(float(x) for x in rng.uniform(0.0, 1.0, 3)) if rng.uniform() < 0.5 else (0.0, 0.0, 0.0)
    st = synth.Settings(tile_w=tw, tile_h=th, bg=bg)
    deg = int(rng.integers(0, 4))
    if rng.uniform() < 0.4:
        scene = synth.tiny_scene(seed, int(rng.integers(40, 600)))
        cam = synth.camera_identity(W, H, float(W) * float(rng.uniform(0.7, 1.3)))
    else:
        scene = synth.cluster_scene(seed, int(rng.integers(200, 4000)), deg)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        centre = tuple(float(x) for x in d * rng.uniform(4.0, 8.0))
        cam = synth.camera_lookat(centre, (0.0, 0.0, 0.0), W, H, float(W))
    eps_split = 0.0 if rng.uniform() < 0.5 else -1e-6
    return scene, cam, st, eps_split


@pytest.mark.parametrize("seed", SEEDS)
def test_random_configuration_parity(seed):
    scene, cam, st, eps_split = _config(seed)
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st, with_keys=True)
    M = PL.project_and_sort(g, vb)
    torch.cuda.synchronize()
    # binning and depth order, bit for bit
    keys, gids, ranges = oracle.bin_sort(scene, cam, st)
    assert M == len(keys)
    assert np.array_equal(vb.bins.gids[:M].cpu().numpy().view(np.uint32), gids)
    assert np.array_equal(vb.bins.keys[:M].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(vb.bins.ranges.cpu().numpy().view(np.uint32), ranges)
    # forward, outside the band of threshold decisions
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    torch.cuda.synchronize()
    ref = oracle.render(scene, cam, st)
    ok = ~ref["band"]
    assert ok.mean() > 0.995
    img = vb.image.cpu().numpy().astype(np.float64)
    assert np.abs(img - ref["image"])[ok].max() < 1e-5
    assert np.array_equal(vb.n_contrib.cpu().numpy()[ok], ref["n_contrib"][ok])
    # backward with the splitting matrices, on the oracle's dL/dC as float32
    tgt = synth.target_image(seed + 50, cam.height, cam.width)
    _, dL_ref = oracle.l1_loss_grad(ref["image"], tgt)
    dL32 = dL_ref.astype(np.float32)
    grads = g.zeros_like()
    S = torch.zeros(scene.n, 6, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib,
                                torch.as_tensor(dL32).cuda().contiguous(), grads, S, ws)
    torch.cuda.synchronize()
    acc = oracle.backward(scene, cam, st, dL32.astype(np.float64))
    if ref["band"].mean() < 1e-3:        # a pixel in the band flips a whole pair's terms
        for f, t in zip(FIELDS, grads.tensors()):
            assert _rel(t.cpu().numpy(), acc[f]) < 1e-4, f
        assert _rel(S.cpu().numpy(), _upper6(acc["S"])) < 1e-4
    # eigenpairs and the split of the GPU's own matrices
    db = PL.DensifyBuffers.alloc(g)
    B.densify_split(g, S, 1.0, eps_split, 0.5, None, 0.0, db.out, db.capacity, db.n_out, db.parent, db.lam, db.v,
                    db.split_ws)
    torch.cuda.synchronize()
    S_in = S.cpu().numpy().astype(np.float64)
    n = scene.n
    S_full = np.zeros((n, 3, 3))
    for k, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        S_full[:, a, b] = S_in[:, k]
        S_full[:, b, a] = S_in[:, k]
    lam_o, v_o = oracle.eig3_min(S_full)
    nrm = np.linalg.norm(S_full.reshape(n, 9), axis=1)
    lam_g = db.lam.cpu().numpy()
    assert np.all(np.abs(lam_g - lam_o) <= 1e-4 * np.maximum(nrm, 1e-30))
    ev = np.linalg.eigvalsh(S_full)
    gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
    v_g = db.v.cpu().numpy()
    assert np.all(1 - np.abs(np.sum(v_g * v_o, 1))[gap] <= 1e-4)
    decided = np.abs(lam_o - eps_split) > 1e-6 * np.maximum(nrm, 1e-30)
    lam_x, _ = oracle.eig3_min(acc["S"])
    structural = SP.structural_zeros(lam_x, np.linalg.norm(acc["S"].reshape(n, 9), axis=1), eps_split)
    n_out = int(db.n_out.item())
    SP.check_split(scene, SP.gpu_out(db, n_out), db.parent.cpu().numpy(), n_out, lam_o, v_o, lam_o < eps_split,
                   decided, gap, eps_split, 0.5, v_gpu=v_g, structural=structural)
