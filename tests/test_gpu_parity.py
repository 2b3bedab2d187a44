"""GPU path vs CPU oracle, element by element, through the C ABI.

Bars: bit-exact integer work (tile rects, keys, sort order, ranges, split
indices); colour within 1e-5 absolute; gradients and splitting matrices
within 1e-4 relative (Frobenius); eigenvalues within 1e-4 |S_bar|_F with
identical split decisions wherever |lambda_min| > 1e-6.  Pixels whose
compositing decisions lie within a relative 1e-5 of a threshold (the oracle's
band mask) are excluded from colour comparisons.
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


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def _gpu_view(scene, cam, st, capacity=None, with_keys=True):
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st, capacity=capacity, with_keys=with_keys)
    M = PL.project_and_sort(g, vb)
    torch.cuda.synchronize()
    return g, vb, M


CASES = [
    ("tiny", lambda: synth.tiny_scene(0), lambda: synth.camera_identity(64, 64, 64.0), synth.Settings()),
    ("tiny_seed7_ragged", lambda: synth.tiny_scene(7, 300), lambda: synth.camera_identity(70, 45, 60.0),
     synth.Settings()),
    ("cluster_sh3_lookat", lambda: synth.cluster_scene(3, 3000, 3),
     lambda: synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0), synth.Settings()),
    ("tile16x8", lambda: synth.tiny_scene(1), lambda: synth.camera_identity(64, 48, 64.0),
     synth.Settings(tile_w=16, tile_h=8)),
    ("tile8x8_sh1", lambda: synth.cluster_scene(5, 800, 1),
     lambda: synth.camera_lookat((0.0, -1.0, -6.0), (0, 0, 0), 77, 59, 77.0), synth.Settings(tile_w=8, tile_h=8)),
    ("tile32x8_sh2_bg", lambda: synth.cluster_scene(6, 1500, 2),
     lambda: synth.camera_lookat((2.0, 0.0, -5.5), (0, 0, 0), 96, 64, 96.0),
     synth.Settings(tile_w=32, tile_h=8, bg=(0.1, 0.2, 0.3))),
]


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_integer_stage_and_sort_bit_exact(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    g, vb, M = _gpu_view(scene, cam, st)
    isg = oracle.integer_stage(scene, cam, st)
    keys, gids, ranges = oracle.bin_sort(scene, cam, st)
    assert M == len(keys)
    tiles = vb.proj.tiles_touched.cpu().numpy()
    assert np.array_equal(tiles, isg["tiles"])
    rect = vb.proj.rect.cpu().numpy().astype(np.int32)
    vis = isg["tiles"] > 0
    assert np.array_equal(rect[vis][:, [0, 2, 1, 3]], isg["rect"][vis])
    depth = vb.proj.depth.cpu().numpy()
    assert np.array_equal(depth[vis].view(np.uint32), isg["depth"][vis].view(np.uint32))
    assert np.array_equal(vb.bins.gids[:M].cpu().numpy().view(np.uint32), gids)
    assert np.array_equal(vb.bins.keys[:M].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(vb.bins.ranges.cpu().numpy().view(np.uint32), ranges)


def _render_gpu(scene, cam, st):
    g, vb, M = _gpu_view(scene, cam, st)
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    torch.cuda.synchronize()
    return g, vb


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_render_fwd_parity(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    g, vb = _render_gpu(scene, cam, st)
    ref = oracle.render(scene, cam, st)
    ok = ~ref["band"]
    assert ok.mean() > 0.999
    img = vb.image.cpu().numpy().astype(np.float64)
    assert np.abs(img - ref["image"])[ok].max() < 1e-5
    assert np.array_equal(vb.n_contrib.cpu().numpy()[ok], ref["n_contrib"][ok])
    assert np.abs(vb.final_T.cpu().numpy() - ref["final_T"])[ok].max() < 1e-5


def test_single_opaque_gaussian_exact_colour():
    c0 = 0.5 / np.sqrt(np.pi)
    sc = synth.Scene(np.array([[0, 0, 3.0]], np.float32), np.full((1, 3), -3.0, np.float32),
                     np.array([[1, 0, 0, 0]], np.float32), np.array([np.log(0.999 / 0.001)], np.float32),
                     (np.array([[[0.6, -0.4, 0.0]]]) / c0).astype(np.float32), 0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings(bg=(0.2, 0.3, 0.4))
    g, vb = _render_gpu(sc, cam, st)
    ref = oracle.render(sc, cam, st)
    assert np.abs(vb.image.cpu().numpy()[32, 32] - ref["image"][32, 32]).max() < 1e-6


def _backward_both(scene, cam, st, target_seed=2):
    g, vb = _render_gpu(scene, cam, st)
    ref = oracle.render(scene, cam, st)
    tgt = synth.target_image(target_seed, cam.height, cam.width)
    L_ref, dL_ref = oracle.l1_loss_grad(ref["image"], tgt)
    # the backward is compared on the same dL/dC (the oracle's, as float32)
    dL = torch.as_tensor(dL_ref.astype(np.float32)).cuda().contiguous()
    grads = g.zeros_like()
    S = torch.zeros(scene.n, 6, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws)
    torch.cuda.synchronize()
    acc = oracle.backward(scene, cam, st, dL_ref.astype(np.float32).astype(np.float64))
    return grads, S, acc, ref, tgt


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_backward_with_splitting_parity(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    grads, S, acc, ref, _ = _backward_both(scene, cam, st)
    assert ref["band"].mean() < 1e-3
    for f, t in zip(FIELDS, grads.tensors()):
        r = _rel(t.cpu().numpy(), acc[f])
        assert r < 1e-4, (f, r)
    Sg = S.cpu().numpy()
    So = _upper6(acc["S"])
    assert _rel(Sg, So) < 1e-4


def test_backward_overwrite_and_accumulate_modes():
    """accumulate_grads = 0 overwrites every row (stale contents do not leak);
    = 1 adds; S always adds."""
    scene = synth.cluster_scene(3, 3000, 3)
    cam = synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0)
    st = synth.Settings()
    grads_ref, S_ref, acc, _, _ = _backward_both(scene, cam, st)
    g, vb = _render_gpu(scene, cam, st)
    ref = oracle.render(scene, cam, st)
    _, dL_ref = oracle.l1_loss_grad(ref["image"], synth.target_image(2, cam.height, cam.width))
    dL = torch.as_tensor(dL_ref.astype(np.float32)).cuda().contiguous()
    grads = g.zeros_like()
    for t in grads.tensors():
        t.fill_(1234.5)                      # stale contents must be overwritten
    S = torch.zeros(scene.n, 6, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                accumulate=False)
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                accumulate=True)
    torch.cuda.synchronize()
    for f, t in zip(FIELDS, grads.tensors()):
        assert _rel(t.cpu().numpy(), 2.0 * acc[f]) < 1e-4, f
    assert _rel(S.cpu().numpy(), 2.0 * _upper6(acc["S"])) < 1e-4


def test_backward_reset_of_splitting_matrices():
    """reset_S: the call writes S (every row, zeros where nothing composited)
    instead of adding, whatever S held before; with gradients accumulated or
    overwritten; a following call without it adds.  Single view at dim
    Theta 3 and 4, and the multi-view pass."""
    scene = synth.cluster_scene(3, 3000, 3)
    cam = synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0)
    st = synth.Settings()
    grads_ref, S_ref, acc, _, _ = _backward_both(scene, cam, st)
    g, vb = _render_gpu(scene, cam, st)
    ref = oracle.render(scene, cam, st)
    _, dL_ref = oracle.l1_loss_grad(ref["image"], synth.target_image(2, cam.height, cam.width))
    dL = torch.as_tensor(dL_ref.astype(np.float32)).cuda().contiguous()
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    for accumulate in (False, True):
        grads = g.zeros_like()
        S = torch.full((scene.n, 6), 7.25, device="cuda")          # stale contents everywhere
        S_po = torch.full((scene.n, 3), -3.5, device="cuda")
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                    accumulate=accumulate, S_po=S_po, reset_S=True)
        torch.cuda.synchronize()
        assert _rel(S.cpu().numpy(), _upper6(acc["S"])) < 1e-4
        assert _rel(S_po.cpu().numpy(), acc["S_po"]) < 1e-4
        unreached = vb.proj.tiles_touched.cpu().numpy() == 0
        assert unreached.sum() > 0 and np.all(S.cpu().numpy()[unreached] == 0.0)
        assert np.all(S_po.cpu().numpy()[unreached] == 0.0)
        for f, t in zip(FIELDS, grads.tensors()):
            assert _rel(t.cpu().numpy(), acc[f]) < 1e-4, f
        B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                    accumulate=True, S_po=S_po)
        torch.cuda.synchronize()
        assert _rel(S.cpu().numpy(), 2.0 * _upper6(acc["S"])) < 1e-4
        assert _rel(S_po.cpu().numpy(), 2.0 * acc["S_po"]) < 1e-4


def test_multi_view_reset_of_splitting_matrices():
    from paper_2505_05587_gb300 import batched as BT
    scene = synth.cluster_scene(3, 3000, 3)
    res = [(150, 101), (96, 64)]
    cams = synth.ring_cameras(6.0, res)
    st = synth.Settings()
    tg = [torch.as_tensor(synth.target_image(10 + k, h, w)).cuda() for k, (w, h) in enumerate(res)]
    g = B.GaussianTensors.from_scene(scene)
    step = BT.BatchedDensifyStep(g, cams, BT.concat_images(tg), st, batch=128)
    step.fit_capacity()
    S_add = torch.zeros(scene.n, 6, device="cuda")
    S_set = torch.full((scene.n, 6), 11.0, device="cuda")
    for S, reset in ((S_add, False), (S_set, True)):
        step.loss.zero_()
        B.render_views_with_splitting(g, cams, st, 128, step.targets, step.images, step.loss, step.grads, False, S,
                                      step.count, step.capacity, step.ws, reset_S=reset)
    torch.cuda.synchronize()
    unreached = (S_add == 0).all(dim=1)
    assert bool(unreached.any()) and bool((S_set[unreached] == 0).all())
    assert _rel(S_set.cpu().numpy(), S_add.cpu().numpy()) < 1e-5     # atomics may add in another order


def test_l1_loss_grad_parity():
    rng = np.random.default_rng(0)
    img = rng.uniform(size=(37, 53, 3)).astype(np.float32)
    tgt = synth.target_image(1, 37, 53)
    L_ref, g_ref = oracle.l1_loss_grad(img.astype(np.float64), tgt, n_views=3)
    ti, tt = torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda()
    dL = torch.empty_like(ti)
    loss = torch.zeros(1, device="cuda")
    B.l1_loss_grad(ti, tt, 3, dL, loss)
    torch.cuda.synchronize()
    assert np.array_equal(np.sign(dL.cpu().numpy()), np.sign(g_ref))
    assert np.abs(dL.cpu().numpy() - g_ref).max() < 1e-6 * np.abs(g_ref).max()
    assert abs(loss.item() - L_ref) < 1e-5 * L_ref


def _densify_both(scene, S_or, S_gpu, eps_split, step_scale=1.0, inv_T=1.0, grad_norm=None, eps_grad=0.0,
                  budget=0):
    g = B.GaussianTensors.from_scene(scene)
    db = PL.DensifyBuffers.alloc(g)
    gn = None if grad_norm is None else torch.as_tensor(grad_norm.astype(np.float32)).cuda()
    B.densify_split(g, S_gpu, inv_T, eps_split, step_scale, gn, eps_grad, db.out, db.capacity, db.n_out, db.parent,
                    db.lam, db.v, db.split_ws, max_splits=budget)
    torch.cuda.synchronize()
    lam_o, v_o = oracle.eig3_min(S_or, inv_T)
    sp = oracle.split(scene, lam_o, v_o, eps_split, step_scale, grad_norm, eps_grad, budget=budget)
    return db, lam_o, v_o, sp


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_densify_split_parity(name, mk_scene, mk_cam, st):
    scene, cam = mk_scene(), mk_cam()
    grads, S, acc, ref, _ = _backward_both(scene, cam, st)
    # the densify step reads the oracle's S (as float32), so its checks are independent of the backward's
    S_or = acc["S"].astype(np.float32).astype(np.float64)
    S_gpu = torch.as_tensor(_upper6(acc["S"]).astype(np.float32)).cuda().contiguous()
    for eps_split in (0.0, -1e-6):
        db, lam_o, v_o, sp = _densify_both(scene, S_or, S_gpu, eps_split, step_scale=0.5, inv_T=0.5)
        lam_g = db.lam.cpu().numpy()
        v_g = db.v.cpu().numpy()
        nrm = np.linalg.norm(S_or.reshape(-1, 9), axis=1) * 0.5
        assert np.all(np.abs(lam_g - lam_o) <= 1e-4 * np.maximum(nrm, 1e-30))
        ev = np.linalg.eigvalsh(S_or * 0.5)
        gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
        cosang = np.abs(np.sum(v_g * v_o, 1))
        assert np.all(1 - cosang[gap] <= 1e-4)
        decided = np.abs(lam_o - eps_split) > max(1e-6, 0.0)
        n_out = int(db.n_out.item())
        lam_x, _ = oracle.eig3_min(acc["S"], 0.5)
        structural = SP.structural_zeros(lam_x, nrm, eps_split)
        SP.check_split(scene, SP.gpu_out(db, n_out), db.parent.cpu().numpy(), n_out, lam_o, v_o, sp["flags"],
                       decided, gap, eps_split, 0.5, v_gpu=v_g, structural=structural)


def test_densify_gradient_gate_parity():
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    _, _, acc, _, _ = _backward_both(scene, cam, synth.Settings())
    S_or = acc["S"].astype(np.float32).astype(np.float64)
    S_gpu = torch.as_tensor(_upper6(acc["S"]).astype(np.float32)).cuda().contiguous()
    gn = np.random.default_rng(3).uniform(size=scene.n).astype(np.float32).astype(np.float64)
    db, lam_o, v_o, sp = _densify_both(scene, S_or, S_gpu, -1e-6, grad_norm=gn, eps_grad=0.4)
    n_out = int(db.n_out.item())
    decided = np.abs(lam_o + 1e-6) > 1e-6
    nrm = np.linalg.norm(S_or.reshape(-1, 9), axis=1)
    ev = np.linalg.eigvalsh(S_or)
    gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
    lam_x, _ = oracle.eig3_min(acc["S"])
    flags_g = SP.check_split(scene, SP.gpu_out(db, n_out), db.parent.cpu().numpy(), n_out, lam_o, v_o,
                             sp["flags"], decided, gap, -1e-6, 1.0, v_gpu=db.v.cpu().numpy(),
                             structural=SP.structural_zeros(lam_x, nrm, -1e-6))
    assert flags_g.sum() < (lam_o < -1e-6).sum()        # the gate removed some splits


def _budget_scene(n=50_000, seed=7):
    """A scene with a random symmetric S per Gaussian (about half of them
    with lambda_min < 0) and a block of exactly repeated rows, so that the
    budget threshold falls inside a group of equal lambda_min."""
    scene = synth.cluster_scene(seed, n, 3)
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, 3, 3))
    S = (A + A.transpose(0, 2, 1)) * 0.5 + 0.3 * np.eye(3)
    S[1000:1400] = S[999]                     # 401 Gaussians with the same S
    S = S.astype(np.float32).astype(np.float64)
    S_gpu = torch.as_tensor(_upper6(S).astype(np.float32)).cuda().contiguous()
    return scene, S, S_gpu


@pytest.mark.parametrize("budget", [1, 37, 1200, 10**9])
def test_densify_budget_parity(budget):
    scene, S_or, S_gpu = _budget_scene()
    db, lam_o, v_o, sp = _densify_both(scene, S_or, S_gpu, 0.0, budget=budget)
    n = scene.n
    n_out = int(db.n_out.item())
    flags_g = np.zeros(n, bool)
    flags_g[db.parent.cpu().numpy()[n:n_out]] = True
    lam_g = db.lam.cpu().numpy()
    cand_g = lam_g < 0.0
    # selection on the kernel's own lambda: exactly the K least, ties by index
    K = min(budget, int(cand_g.sum()))
    order = np.lexsort((np.arange(n), lam_g.astype(np.float64)))
    want = np.zeros(n, bool)
    want[[i for i in order if cand_g[i]][:K]] = True
    assert np.array_equal(flags_g, want)
    # against the oracle: same set wherever lambda is not within rounding of the threshold
    nrm = np.linalg.norm(S_or.reshape(-1, 9), axis=1)
    kept = lam_o[sp["flags"]]
    thr = kept.max() if kept.size else -np.inf
    near0 = np.abs(lam_o) <= 1e-4 * nrm
    near = (np.abs(lam_o - thr) <= 1e-4 * nrm) | near0
    assert abs(n_out - sp["n_out"]) <= int(near0.sum())
    if budget < (lam_o < 0).sum() - near0.sum():
        assert n_out - n == budget == sp["n_out"] - n
    assert np.array_equal(flags_g[~near], sp["flags"][~near])
    # compaction indices and offspring from the GPU's own selection, always
    ev = np.linalg.eigvalsh(S_or)
    gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
    SP.check_split(scene, SP.gpu_out(db, n_out), db.parent.cpu().numpy(), n_out, lam_o, v_o, flags_g,
                   np.ones(n, bool), gap, 0.0, 1.0, v_gpu=db.v.cpu().numpy())


def test_densify_budget_cuts_a_tie_group():
    scene, S_or, S_gpu = _budget_scene()
    db, _, _, _ = _densify_both(scene, S_or, S_gpu, 0.0, budget=0)
    lam = db.lam.cpu().numpy()
    tie = lam[999]
    assert np.all(lam[1000:1400] == tie) and tie < 0
    below = int(((lam < tie)).sum())
    budget = below + 150                      # the cut falls inside the 401 equal values
    db, _, _, _ = _densify_both(scene, S_or, S_gpu, 0.0, budget=budget)
    n = scene.n
    par = db.parent.cpu().numpy()[n:int(db.n_out.item())]
    chosen = set(par.tolist())
    assert len(chosen) == budget
    assert chosen.issuperset(set(range(999, 1149))) and not chosen & set(range(1149, 1400))


def test_fused_iteration_end_to_end():
    """The whole pipeline (both views summed) against the oracle iteration."""
    scene = synth.tiny_scene(0)
    cams = [synth.camera_identity(64, 64, 64.0), synth.camera_identity(64, 64, 64.0, centre=(0.2, -0.1, 0.0))]
    st = synth.Settings()
    tg = [synth.target_image(2, 64, 64), synth.target_image(3, 64, 64)]
    g = B.GaussianTensors.from_scene(scene)
    views = [PL.ViewBuffers.alloc(scene.n, c, st) for c in cams]
    db = PL.DensifyBuffers.alloc(g)
    targets = [torch.as_tensor(t).cuda() for t in tg]
    PL.fused_iteration(g, views, targets, db, eps_split=-1e-6)
    torch.cuda.synchronize()
    ref = oracle.densify_iteration(scene, cams, st, tg, eps_split=-1e-6)
    assert abs(db.loss.item() - ref["loss"]) < 1e-5 * ref["loss"]
    assert _rel(db.S.cpu().numpy(), _upper6(ref["grads"]["S"])) < 1e-4
    for f, t in zip(FIELDS, db.grads.tensors()):
        assert _rel(t.cpu().numpy(), ref["grads"][f]) < 1e-4, f


def test_empty_and_fully_culled_scenes():
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    empty = synth.subset(synth.tiny_scene(0), slice(0, 0))
    g, vb = _render_gpu(empty, cam, st)
    assert int(vb.bins.count.item()) == 0
    assert np.all(vb.image.cpu().numpy() == 0.0) and np.all(vb.final_T.cpu().numpy() == 1.0)
    behind = synth.tiny_scene(1)
    behind.means[:, 2] = -behind.means[:, 2]
    g, vb = _render_gpu(behind, cam, st)
    assert int(vb.bins.count.item()) == 0
    assert np.all(vb.proj.tiles_touched.cpu().numpy() == 0)
    grads = g.zeros_like()
    S = torch.zeros(behind.n, 6, device="cuda")
    dL = torch.ones(64, 64, 3, device="cuda")
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S,
                                B.workspace(B.render_bwd_workspace_size(behind.n)), accumulate=False)
    torch.cuda.synchronize()
    assert float(S.abs().max()) == 0.0 and float(grads.means.abs().max()) == 0.0


def test_capacity_overflow_reported_and_regrown():
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st, capacity=16, with_keys=True)
    B.project(g, cam, st, vb.proj)
    B.bin_sort(vb.proj, scene.n, cam, st, vb.bins, vb.sort_ws)
    torch.cuda.synchronize()
    M = int(vb.bins.count.item())
    keys, gids, ranges = oracle.bin_sort(scene, cam, st)
    assert M == len(keys) > 16
    M2 = PL.project_and_sort(g, vb)
    torch.cuda.synchronize()
    assert M2 == M and vb.bins.capacity >= M
    assert np.array_equal(vb.bins.gids[:M].cpu().numpy().view(np.uint32), gids)


def test_invalid_arguments_rejected_on_host():
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, synth.Settings())
    with pytest.raises(B.SteepGSError) as e:
        B.project(g, cam, synth.Settings(tile_w=12, tile_h=12), vb.proj)
    assert e.value.status == 1
    with pytest.raises(B.SteepGSError) as e:
        B.bin_sort(vb.proj, scene.n, cam, synth.Settings(), vb.bins, B.workspace(16))
    assert e.value.status == 2


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES, ids=[c[0] for c in CASES])
def test_tile_order_is_the_longest_first_permutation(name, mk_scene, mk_cam, st):
    """bins.order: every tile once, list lengths in quarter octaves (the leading
    three bits) descending, empty tiles last, ties by tile id (bit-exact
    against a host sort)."""
    scene, cam = mk_scene(), mk_cam()
    _, vb, _ = _gpu_view(scene, cam, st)
    ranges = vb.bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    length = ranges[:, 1] - ranges[:, 0]
    cls = np.full(len(length), 128, np.int64)
    for t, n in enumerate(length):
        if n > 0:
            k = int(n).bit_length() - 1                   # floor(log2 n)
            next2 = (int(n) >> (k - 2)) & 3 if k >= 2 else ((int(n) & 1) << 1 if k == 1 else 0)
            cls[t] = 4 * (31 - k) + 3 - next2
    expect = np.lexsort((np.arange(len(length)), cls))
    assert np.array_equal(vb.bins.order.cpu().numpy().view(np.uint32), expect.astype(np.uint32))


def test_results_do_not_depend_on_the_tile_order():
    scene = synth.cluster_scene(3, 3000, 3)
    cam = synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0)
    st = synth.Settings()
    g, vb, _ = _gpu_view(scene, cam, st)
    tgt = torch.as_tensor(synth.target_image(2, cam.height, cam.width)).cuda()
    out = {}
    for use_order in (True, False):
        bins = vb.bins if use_order else B.BinBuffers(vb.bins.gids, vb.bins.keys, vb.bins.ranges, vb.bins.count,
                                                      vb.bins.capacity, None)
        B.render_fwd(vb.proj, bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
        dL = torch.empty_like(vb.image)
        loss = torch.zeros(1, device="cuda")
        B.l1_loss_grad(vb.image, tgt, 1, dL, loss)
        grads = g.zeros_like()
        S = torch.zeros(g.n, 6, device="cuda")
        ws = B.workspace(B.render_bwd_workspace_size(g.n))
        B.render_bwd_with_splitting(g, vb.proj, bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                    accumulate=False)
        torch.cuda.synchronize()
        out[use_order] = (vb.image.clone(), vb.n_contrib.clone(), S.cpu().numpy(),
                          [t.cpu().numpy() for t in grads.tensors()])
    a, b = out[True], out[False]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert _rel(a[2], b[2]) < 1e-5
    for x, y in zip(a[3], b[3]):
        assert _rel(x, y) < 1e-5


@pytest.mark.parametrize("name,mk_scene,mk_cam,st", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_forward_with_fused_l1_equals_forward_then_l1(name, mk_scene, mk_cam, st):
    """render_fwd_l1: image, final_T, n_contrib and dL bit for bit as
    render_fwd followed by l1_loss_grad; the loss to float summation order."""
    scene, cam = mk_scene(), mk_cam()
    _, vb, _ = _gpu_view(scene, cam, st)
    tgt = torch.as_tensor(synth.target_image(4, cam.height, cam.width)).cuda()
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    dL1 = torch.empty_like(vb.image)
    loss1 = torch.zeros(1, device="cuda")
    B.l1_loss_grad(vb.image, tgt, 2, dL1, loss1)
    ref = (vb.image.clone(), vb.final_T.clone(), vb.n_contrib.clone())
    dL2 = torch.full_like(vb.image, 7.0)
    loss2 = torch.full((1,), 0.25, device="cuda")
    img = torch.full_like(vb.image, -1.0)
    B.render_fwd_l1(vb.proj, vb.bins, cam, st, tgt, 2, img, vb.final_T, vb.n_contrib, dL2, loss2)
    torch.cuda.synchronize()
    assert torch.equal(img, ref[0]) and torch.equal(vb.final_T, ref[1]) and torch.equal(vb.n_contrib, ref[2])
    assert torch.equal(dL2, dL1)
    assert abs(float(loss2.item()) - 0.25 - float(loss1.item())) <= 1e-6 * float(loss1.item()) + 1e-9


def test_schedule_entries_out_of_range_are_skipped():
    """The render kernels bound every schedule entry by the tile count: a
    schedule holding out-of-range ids renders nothing for them (no access
    outside the buffers) and leaves the valid tiles exact."""
    scene, cam, st = CASES[0][1](), CASES[0][2](), CASES[0][3]
    g, vb, _ = _gpu_view(scene, cam, st)
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    ref = vb.image.clone()
    T = B.num_tiles(cam, st)
    bad = vb.bins.order.clone()
    bad[: T // 2] = T + 7                            # first half of the schedule out of range
    bins = B.BinBuffers(vb.bins.gids, vb.bins.keys, vb.bins.ranges, vb.bins.count, vb.bins.capacity, bad)
    img = torch.full_like(vb.image, -1.0)
    B.render_fwd(vb.proj, bins, cam, st, img, vb.final_T, vb.n_contrib)
    torch.cuda.synchronize()
    kept = vb.bins.order[T // 2:].cpu().numpy()
    gx = (cam.width + st.tile_w - 1) // st.tile_w
    for t in kept[:8]:
        ty, tx = divmod(int(t), gx)
        ys, xs = slice(ty * st.tile_h, (ty + 1) * st.tile_h), slice(tx * st.tile_w, (tx + 1) * st.tile_w)
        assert torch.equal(img[ys, xs], ref[ys, xs])
    assert bool((img == -1.0).any())                  # the skipped tiles stay unwritten
