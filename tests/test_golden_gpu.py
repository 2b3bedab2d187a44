"""The CUDA path against the stored golden fixture of the tiny scene
(tests/golden/tiny_64x64_seed0.json, written by the oracle), through the C
ABI, with no oracle call at run time.

Bars as in the live parity tests: integer work bit-exact (tile counts, the
sorted keys, gids and tile ranges by SHA-256); colour and transmittance within
1e-5 outside the threshold band; loss within 1e-5 relative; gradients and
splitting matrices of the sampled Gaussians within 1e-4 relative (Frobenius);
eigenvalues within 1e-4 relative and identical split decisions wherever
|lambda_min| > 1e-6."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "golden", "tiny_64x64_seed0.json")) as f:
        return json.load(f)


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _bits(hexstr, count):
    return np.unpackbits(np.frombuffer(bytes.fromhex(hexstr), np.uint8))[:count].astype(bool)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


@pytest.fixture(scope="module")
def run(gold):
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    target = torch.as_tensor(synth.target_image(2, cam.height, cam.width)).cuda()
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st, with_keys=True)
    M = PL.project_and_sort(g, vb)
    B.render_fwd(vb.proj, vb.bins, cam, st, vb.image, vb.final_T, vb.n_contrib)
    dL_own = torch.empty_like(vb.image)
    loss = torch.zeros(1, device="cuda")
    B.l1_loss_grad(vb.image, target, 1, dL_own, loss)
    # the backward takes the fixture's dL/dC: sign bits times the L1 normalisation, in float32
    pos = _bits(gold["dL_positive_bits"], cam.height * cam.width * 3).reshape(cam.height, cam.width, 3)
    dL = np.where(pos, 1.0, -1.0) * gold["dL_magnitude"]
    dL = torch.as_tensor(dL.astype(np.float32)).cuda().contiguous()
    grads = g.zeros_like()
    S = torch.zeros(scene.n, 6, device="cuda")
    S_po = torch.zeros(scene.n, 3, device="cuda")
    ws = B.workspace(B.render_bwd_workspace_size(scene.n))
    B.render_bwd_with_splitting(g, vb.proj, vb.bins, cam, st, vb.final_T, vb.n_contrib, dL, grads, S, ws,
                                accumulate=False, S_po=S_po)
    db = PL.DensifyBuffers.alloc(g)
    w = gold["workload"]
    B.densify_split(g, S, 1.0 / w["T_split"], w["eps_split"], w["step_scale"], None, 0.0, db.out, db.capacity,
                    db.n_out, db.parent, db.lam, db.v, db.split_ws)
    torch.cuda.synchronize()
    return dict(scene=scene, cam=cam, M=M, vb=vb, dL_own=dL_own.cpu().numpy(), loss=float(loss.item()),
                grads={f: t.cpu().numpy() for f, t in zip(("means", "log_scales", "quats", "opacity_logit", "sh"),
                                                          grads.tensors())},
                S=S.cpu().numpy(), S_po=S_po.cpu().numpy(), lam=db.lam.cpu().numpy(), v=db.v.cpu().numpy(),
                n_out=int(db.n_out.item()), parent=db.parent.cpu().numpy())


def test_integer_stage_bit_exact(gold, run):
    vb = run["vb"]
    M = run["M"]
    assert M == gold["integer"]["instances"]
    assert vb.proj.tiles_touched.cpu().numpy().tolist() == gold["integer"]["tiles_touched"]
    assert _sha(vb.bins.keys[:M].cpu().numpy().view(np.uint64)) == gold["integer"]["keys_sha256"]
    assert _sha(vb.bins.gids[:M].cpu().numpy().view(np.uint32)) == gold["integer"]["gids_sha256"]
    assert _sha(vb.bins.ranges.cpu().numpy().view(np.uint32)) == gold["integer"]["ranges_sha256"]


def test_sampled_pixels_and_loss(gold, run):
    vb = run["vb"]
    img, T, nc = vb.image.cpu().numpy(), vb.final_T.cpu().numpy(), vb.n_contrib.cpu().numpy()
    checked = 0
    for y, x, r, g_, b, t, n, band in gold["pixels"]:
        if band:
            continue
        assert np.abs(img[y, x] - np.array([r, g_, b])).max() < 1e-5, (y, x)
        assert abs(T[y, x] - t) < 1e-5, (y, x)
        assert nc[y, x] == n, (y, x)
        checked += 1
    assert checked >= 0.99 * len(gold["pixels"])
    assert abs(run["loss"] - gold["loss"]) <= 1e-5 * gold["loss"]
    # the L1 gradient's own sign pattern: a flip needs |C - C_hat| below the colour error
    pos = _bits(gold["dL_positive_bits"], img.size).reshape(img.shape)
    assert int(np.sum((run["dL_own"] > 0) != pos)) <= 3
    assert np.abs(np.abs(run["dL_own"]) - gold["dL_magnitude"]).max() <= 1e-6 * gold["dL_magnitude"]


def test_sampled_gradients_and_splitting_matrices(gold, run):
    idx = [r["i"] for r in gold["rows"]]
    for key, got in (("S", run["S"]), ("S_po", run["S_po"]), ("grad_means", run["grads"]["means"]),
                     ("grad_log_scales", run["grads"]["log_scales"]), ("grad_quats", run["grads"]["quats"]),
                     ("grad_opacity_logit", run["grads"]["opacity_logit"]),
                     ("grad_sh", run["grads"]["sh"].reshape(run["scene"].n, -1))):
        want = np.array([r[key] for r in gold["rows"]], np.float64)
        assert _rel(got[idx], want) < 1e-4, key


def test_eigenpairs_and_split(gold, run):
    lam_o = np.array(gold["lambda_min"])
    n = lam_o.size
    assert _rel(run["lam"], lam_o) < 1e-4
    for r in gold["rows"]:
        a, b, c, d, e, f = r["S"]
        ev = np.linalg.eigvalsh(np.array([[a, b, c], [b, d, e], [c, e, f]]))
        nrm = float(np.sqrt(np.sum(ev ** 2)))
        assert abs(run["lam"][r["i"]] - r["lambda_min"]) <= 1e-4 * max(nrm, 1e-30)
        if ev[1] - ev[0] > 1e-3 * nrm:
            assert 1.0 - abs(float(np.dot(run["v"][r["i"]], r["v_min"]))) <= 1e-4
    flags_o = _bits(gold["split"]["flags_bits"], n)
    flags_g = np.zeros(n, bool)
    flags_g[run["parent"][n:run["n_out"]]] = True
    decided = np.abs(lam_o - gold["workload"]["eps_split"]) > 1e-6
    assert decided.sum() > 0.8 * n
    assert np.array_equal(flags_g[decided], flags_o[decided])
    # decisions at exactly the threshold in exact arithmetic (a rank-2 single-view S with lambda_min = 0)
    # are the sign of rounding on both sides and are not counted
    structural = np.abs(lam_o - gold["workload"]["eps_split"]) <= 1e-12 * np.abs(lam_o).max()
    assert int(np.sum((flags_g != flags_o) & ~structural)) <= int(np.ceil(1e-4 * n))
    # the compaction is the exclusive scan of the GPU's own flags: the first n
    # rows in place, the split Gaussians appended once each in index order
    par = np.asarray(run["parent"][:run["n_out"]])
    assert run["n_out"] == n + int(flags_g.sum())
    assert np.array_equal(par[:n], np.arange(n))
    assert par[n:].tolist() == np.flatnonzero(flags_g).tolist()
    # the stored split's appended rows, restricted to decisions both sides share
    both = flags_g & flags_o
    assert [i for i in par[n:].tolist() if both[i]] == [i for i in gold["split"]["parent"] if both[i]]
