"""The seeded input generators against the recipe they state (sizes, ranges,
moments of the distributions, camera placement, request stream)."""
import math

import numpy as np

import synth


def test_tiny_scene_recipe():
    sc = synth.tiny_scene(0, 20_000)
    assert sc.n == 20_000 and sc.sh_degree == 0 and sc.sh.shape == (20_000, 1, 3)
    for a in (sc.means, sc.log_scales, sc.quats, sc.opacity_logit, sc.sh):
        assert a.dtype == np.float32
    assert np.all(np.abs(sc.means[:, :2]) <= 1.0) and np.all((sc.means[:, 2] >= 2.0) & (sc.means[:, 2] <= 4.0))
    assert abs(sc.log_scales.mean() + 3.0) < 0.02 and abs(sc.log_scales.std() - 0.5) < 0.02
    assert np.allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-6)
    assert abs(sc.opacity_logit.mean()) < 0.03 and abs(sc.opacity_logit.std() - 1.0) < 0.03
    rgb = sc.sh[:, 0, :] * (0.5 / math.sqrt(math.pi)) + 0.5            # degree-0 colour map
    assert rgb.min() >= 0.0 and rgb.max() <= 1.0 and abs(rgb.mean() - 0.5) < 0.01
    assert synth.tiny_scene(0).n == 256
    assert np.array_equal(synth.tiny_scene(3).means, synth.tiny_scene(3).means)     # seeded


def test_cluster_scene_recipe():
    sc = synth.cluster_scene(0, 50_000, 3)
    assert sc.sh.shape == (50_000, 16, 3)
    assert np.all(np.abs(sc.means) <= 5.0)                               # 10-unit box
    assert abs(sc.log_scales.mean() + 4.5) < 0.02 and abs(sc.log_scales.std() - 0.7) < 0.02
    assert abs(sc.opacity_logit.mean() + 1.0) < 0.03 and abs(sc.opacity_logit.std() - 1.5) < 0.03
    dc, rest = sc.sh[:, 0, :], sc.sh[:, 1:, :]
    assert abs(dc.mean() - 0.5) < 0.01 and abs(dc.std() - 0.2) < 0.01
    assert abs(rest.mean()) < 0.01 and abs(rest.std() - 0.2) < 0.01
    # a mixture of 64 clusters, not a uniform fill: cell counts vary far more
    # than the Poisson spread (sqrt of the mean) a uniform draw would give
    hist, _ = np.histogramdd(sc.means, bins=(5, 5, 5), range=[(-5, 5)] * 3)
    assert hist.std() > 5 * math.sqrt(hist.mean())


def test_cameras_look_at_the_origin():
    cams = synth.ring_cameras(6.0)
    assert [(c.width, c.height) for c in cams] == synth.RING_RESOLUTIONS
    assert sum(c.width * c.height for c in cams) == 7_356_101
    for k, c in enumerate(cams):
        R = c.R.astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        centre = -R.T @ c.t.astype(np.float64)
        phi = 2 * math.pi * k / 8
        assert np.allclose(centre, [6 * math.sin(phi), 0.0, -6 * math.cos(phi)], atol=1e-5)
        o_cam = R @ np.zeros(3) + c.t                                   # the origin lies on the optical axis
        assert abs(o_cam[0]) < 1e-5 and abs(o_cam[1]) < 1e-5 and abs(o_cam[2] - 6.0) < 1e-5
        assert c.fx == c.fy == c.width and c.cx == c.width / 2 and c.cy == c.height / 2
    offs = synth.offset_cameras(128, 128, 128.0, 0.25)
    centres = sorted(tuple(np.round(-c.t, 6)) for c in offs)
    assert centres == sorted((sx * 0.25, sy * 0.25, 0.0) for sx in (-1, 1) for sy in (-1, 1))


def test_request_stream_recipe():
    reqs = synth.request_stream(3, 4000, 200.0, 6)
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(t)
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0      # Poisson at 200/s
    scenes = np.bincount([r.scene for r in reqs], minlength=6)
    assert scenes.min() > 0.8 * 4000 / 6
    res = {(r.camera.width, r.camera.height) for r in reqs}
    assert res == set(synth.SERVE_RESOLUTIONS)
    for r in reqs[:50]:
        centre = -r.camera.R.astype(np.float64).T @ r.camera.t.astype(np.float64)
        assert abs(np.linalg.norm(centre) - 6.0) < 1e-4


def test_target_image():
    t = synth.target_image(2, 64, 48)
    assert t.shape == (64, 48, 3) and t.dtype == np.float32
    assert t.min() >= 0.0 and t.max() <= 1.0 and abs(t.mean() - 0.5) < 0.02
