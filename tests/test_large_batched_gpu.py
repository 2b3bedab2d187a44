"""Parity of the batched forms at the sizes they are measured at.

Batched densification step (3M Gaussians from the 64-cluster mixture, SH3,
the 8 ring views 1957x1091 ... 800x600, about 48.6M instances), one
render_views_with_splitting pass:
  * the binning it leaves in its workspace, bit for bit against the oracle's
    stable sort, for two views (global tile ids and projection rows mapped
    back to each view);
  * every view's image bit for bit against the single-view path (whose
    binning and colours are compared with the oracle at full size elsewhere);
  * colours, parameter gradients and splitting matrices on row strips of two
    views against the oracle: the targets equal the rendered image outside
    the strips (so dL/dC = sign(0) = 0 there) and differ from it by at least
    0.01 inside them (so both sides take the same L1 signs).
Serving batch: three requests whose scenes add up to 8M projection rows (the
sort path without dependent launches), each image bit for bit against its
single-view render.
"""
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

N = 3_000_000
FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")
STRIPS = {0: (541, 16), 5: (296, 9)}          # view -> (first row, rows)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def _upper6(S):
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


@pytest.fixture(scope="module")
def ring():
    scene = synth.cluster_scene(0, N, 3)
    cams = synth.ring_cameras(6.0)
    st = synth.Settings()
    g = B.GaussianTensors.from_scene(scene)
    tgs = [torch.as_tensor(synth.target_image(10 + k, c.height, c.width)).cuda() for k, c in enumerate(cams)]
    step = BT.BatchedDensifyStep(g, cams, BT.concat_images(tgs), st, batch=128)
    M = step.fit_capacity()
    torch.cuda.synchronize()
    return scene, cams, st, g, step, M


def _pix_off(cams):
    return np.cumsum([0] + [c.width * c.height for c in cams])


def test_batched_binning_bit_exact_on_two_views(ring):
    scene, cams, st, g, step, M = ring
    assert M > 40_000_000
    bins = B.render_views_bins(N, cams, st, step.capacity, step.ws, step.count)
    ranges = bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    tile_off = np.cumsum([0] + [B.num_tiles(c, st) for c in cams])
    for v in (2, 7):
        keys, gids, rg = oracle.bin_sort(scene, cams[v], st)
        T = tile_off[v + 1] - tile_off[v]
        r = ranges[tile_off[v]:tile_off[v + 1]]
        s, e = int(r[0, 0]), int(r[-1, 1])
        assert e - s == len(gids)
        got = bins.gids[s:e].cpu().numpy().view(np.uint32).astype(np.int64) - v * N
        assert np.array_equal(got, gids.astype(np.int64))
        assert np.array_equal(r - s, rg.astype(np.int64).reshape(T, 2))


def test_batched_images_equal_single_view_renders(ring):
    scene, cams, st, g, step, M = ring
    off = _pix_off(cams)
    img = step.images.clone()
    for v, cam in enumerate(cams):
        vb = PL.ViewBuffers.alloc(N, cam, st, walk=False)
        PL.render(g, vb)
        torch.cuda.synchronize()
        assert torch.equal(img[off[v]:off[v + 1]].reshape(cam.height, cam.width, 3), vb.image), v
        del vb


def test_batched_colours_and_backward_on_strips_of_two_views(ring):
    scene, cams, st, g, step, M = ring
    off = _pix_off(cams)
    images = step.images.clone()
    targets = images.clone()
    rng = np.random.default_rng(4)
    for v, (y0, h) in STRIPS.items():
        W = cams[v].width
        a, b = off[v] + y0 * W, off[v] + (y0 + h) * W
        d = rng.uniform(0.01, 0.3, size=(b - a, 3)) * rng.choice([-1.0, 1.0], size=(b - a, 3))
        targets[a:b] += torch.as_tensor(d.astype(np.float32)).cuda()
    grads = g.zeros_like()
    S = torch.zeros(N, 6, device="cuda")
    loss = torch.zeros(1, device="cuda")
    B.render_views_with_splitting(g, cams, st, 128, targets, step.images, loss, grads, False, S, step.count,
                                  step.capacity, step.ws, reset_S=True)
    torch.cuda.synchronize()
    assert torch.equal(step.images, images)                # the forward pass is deterministic
    acc = None
    tg = targets.cpu().numpy().astype(np.float64)
    for v, (y0, h) in STRIPS.items():
        cam = cams[v]
        r = oracle.render(scene, cam, st, rows=(y0, h), all_cores=True)
        gpu = images[off[v] + y0 * cam.width:off[v] + (y0 + h) * cam.width].cpu().numpy().reshape(h, cam.width, 3)
        ok = ~r["band"]
        assert ok.mean() > 0.999
        assert np.abs(gpu.astype(np.float64) - r["image"])[ok].max() < 1e-5
        t = tg[off[v] + y0 * cam.width:off[v] + (y0 + h) * cam.width].reshape(h, cam.width, 3)
        _, dL = oracle.l1_loss_grad(r["image"], t.astype(np.float32), len(cams))
        dL *= h / cam.height                  # the L1 mean runs over the whole view, not the strip
        acc = oracle.backward(scene, cam, st, dL, acc, rows=(y0, h), all_cores=True, blocks=False)
    for f, tgrad in zip(FIELDS, grads.tensors()):
        assert _rel(tgrad.cpu().numpy(), acc[f]) < 1e-4, f
    assert _rel(S.cpu().numpy(), _upper6(acc["S"])) < 1e-4


def test_serving_batch_above_four_million_rows():
    st = synth.Settings()
    scenes = [B.GaussianTensors.from_scene(synth.cluster_scene(30 + k, n, 3)) for k, n in
              enumerate((3_000_000, 2_000_000))]
    rng = np.random.default_rng(8)
    cams = [synth.sphere_camera(rng, w, h) for (w, h) in ((1920, 1080), (640, 480), (1237, 822))]
    which = [0, 1, 0]                                       # 8M projection rows
    sc = [scenes[k] for k in which]
    cap = 4 * sum(s.n for s in sc)
    ws = B.workspace(B.render_batch_workspace_size(sc, cams, st, cap))
    P = sum(c.width * c.height for c in cams)
    images = torch.empty(P, 3, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.render_batch_fwd(sc, cams, st, 0, images, count, cap, ws)
    torch.cuda.synchronize()
    assert 0 < int(count.item()) <= cap
    off = _pix_off(cams)
    for v, (g, cam) in enumerate(zip(sc, cams)):
        vb = PL.ViewBuffers.alloc(g.n, cam, st, walk=False)
        PL.render(g, vb)
        torch.cuda.synchronize()
        assert torch.equal(images[off[v]:off[v + 1]].reshape(cam.height, cam.width, 3), vb.image), v
