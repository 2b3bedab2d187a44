"""SSIM term of the loss on the GPU (sgs_ssim_l1_loss_grad) against the
float64 oracle, alone and feeding the backward with splitting matrices."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ssim as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import pipeline as PL  # noqa: E402

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def _gpu(img, tgt, n_views, lam):
    ti, tt = torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda()
    dL = torch.full_like(ti, float("nan"))
    loss = torch.zeros(1, device="cuda")
    ws = B.workspace(B.ssim_l1_workspace_size(img.shape[0], img.shape[1]))
    B.ssim_l1_loss_grad(ti, tt, n_views, lam, dL, loss, ws)
    torch.cuda.synchronize()
    return float(loss.item()), dL.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 64), (37, 53), (150, 101), (9, 5), (1, 1), (822, 1237)])
@pytest.mark.parametrize("lam", [0.2, 1.0, 0.0])
def test_ssim_l1_matches_oracle(shape, lam):
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    img = rng.uniform(size=(H, W, 3)).astype(np.float32)
    tgt = synth.target_image(7, H, W)
    L, g = _gpu(img, tgt, 3, lam)
    L_ref, g_ref = OS.ssim_l1_loss_grad(img.astype(np.float64), tgt.astype(np.float64), 3, lam)
    assert abs(L - L_ref) <= 1e-5 * abs(L_ref) + 1e-7
    assert np.all(np.isfinite(g))
    assert _rel(g, g_ref) < 1e-4
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max() + 1e-12


def test_ssim_identical_images_and_smooth_regions():
    # SSIM = 1 and only the L1 sign term remains (zero where x = y)
    H, W = 48, 70
    y = np.linspace(0, 1, H * W * 3, dtype=np.float32).reshape(H, W, 3)
    L, g = _gpu(y.copy(), y, 1, 0.2)
    assert abs(L) < 1e-6 and np.abs(g).max() < 1e-3 / (3 * H * W)
    # a smooth rendered-like image against a flat target (small local variances)
    x = (0.5 + 0.01 * np.sin(np.arange(H)[:, None, None] / 7.0) * np.ones((1, W, 3))).astype(np.float32)
    t = np.full((H, W, 3), 0.5, np.float32)
    L, g = _gpu(x, t, 1, 0.2)
    L_ref, g_ref = OS.ssim_l1_loss_grad(x.astype(np.float64), t.astype(np.float64), 1, 0.2)
    # float32 bound: each filtered second moment carries ~11 eps E[x^2] of
    # rounding per pass (two 11-tap passes), and the variance sum enters S
    # through B2 >= C2, so |dS| <~ 2 * 11 eps (E[x^2] + E[y^2]) / C2 per pixel.
    eps = 2.0 ** -24
    dS = 2 * 11 * eps * (np.mean(x.astype(np.float64) ** 2) + np.mean(t.astype(np.float64) ** 2)) / OS.C2
    assert abs(L - L_ref) <= 1e-5 * abs(L_ref) + 0.2 * dS
    assert _rel(g, g_ref) < 1e-4 + dS


def test_ssim_loss_feeds_the_splitting_matrices():
    """The SSIM gradient changes dL/dalpha and hence S: the fused iteration with
    the SSIM term against the oracle backward driven by the oracle's SSIM
    gradient of the oracle's image."""
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    tg = synth.target_image(2, 64, 64)
    g = B.GaussianTensors.from_scene(scene)
    vb = PL.ViewBuffers.alloc(scene.n, cam, st)
    db = PL.DensifyBuffers.alloc(g)
    PL.fused_iteration(g, [vb], [torch.as_tensor(tg).cuda()], db, eps_split=-1e-6, lambda_dssim=0.2)
    torch.cuda.synchronize()
    ref = oracle.render(scene, cam, st)
    L_ref, dL_ref = OS.ssim_l1_loss_grad(ref["image"], tg.astype(np.float64), 1, 0.2)
    acc = oracle.backward(scene, cam, st, dL_ref)
    assert abs(db.loss.item() - L_ref) < 1e-5 * L_ref
    S = acc["S"]
    up = np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)
    assert _rel(db.S.cpu().numpy(), up) < 1e-4
    for f, t in zip(FIELDS, db.grads.tensors()):
        assert _rel(t.cpu().numpy(), acc[f]) < 1e-4, f
    # the SSIM term changes S relative to L1 alone
    _, dL_l1 = oracle.l1_loss_grad(ref["image"], tg)
    S_l1 = oracle.backward(scene, cam, st, dL_l1)["S"]
    assert _rel(S_l1.reshape(-1, 9), S.reshape(-1, 9)) > 1e-2


def test_ssim_invalid_arguments():
    x = torch.zeros(8, 8, 3, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = B.workspace(B.ssim_l1_workspace_size(8, 8))
    with pytest.raises(Exception):
        B.ssim_l1_loss_grad(x, x, 1, 1.5, x.clone(), loss, ws)
    with pytest.raises(Exception):
        B.ssim_l1_loss_grad(x, x, 1, 0.2, x.clone(), loss, B.workspace(16))
