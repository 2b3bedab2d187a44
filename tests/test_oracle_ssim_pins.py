"""Pins of the SSIM oracle (oracle/ssim.py) to facts outside its own code:
the explicit 2-D window, a brute-force non-separable SSIM, the constant-image
closed form, the maximum at x = y, symmetry, and central differences."""
import numpy as np
import pytest

from oracle import ssim as OS


def _window2d():
    r = np.arange(11) - 5
    g = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2 * 1.5 ** 2))   # the 2-D Gaussian written out
    return g / g.sum()


def test_filter_of_a_delta_is_the_2d_window():
    img = np.zeros((21, 23))
    img[10, 11] = 1.0
    out = OS.gaussian_filter(img)
    np.testing.assert_allclose(out[5:16, 6:17], _window2d(), rtol=0, atol=1e-15)
    assert abs(out.sum() - 1.0) < 1e-14


def _ssim_brute(x, y):
    """Direct per-pixel 11x11 window sums with zero padding (no separability)."""
    H, W = x.shape
    w = _window2d()
    S = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        k = w[di + 5, dj + 5]
                        a, b = x[ii, jj], y[ii, jj]
                        mx += k * a
                        my += k * b
                        exx += k * a * a
                        eyy += k * b * b
                        exy += k * a * b
            sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            S[i, j] = ((2 * mx * my + 0.01 ** 2) * (2 * sxy + 0.03 ** 2)) / (
                (mx * mx + my * my + 0.01 ** 2) * (sxx + syy + 0.03 ** 2))
    return S


def test_ssim_map_matches_brute_force_window_sums():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(size=(9, 14)), rng.uniform(size=(9, 14))
    S, _ = OS.ssim_map(x, y)
    np.testing.assert_allclose(S, _ssim_brute(x, y), rtol=1e-12, atol=1e-13)


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x, y = np.full((23, 25), a), np.full((23, 25), b)
    S, _ = OS.ssim_map(x, y)
    want = (2 * a * b + 0.01 ** 2) / (a * a + b * b + 0.01 ** 2)     # variances and covariance vanish
    np.testing.assert_allclose(S[5:-5, 5:-5], want, rtol=1e-12)


def test_identical_images_maximum_and_symmetry():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(12, 13, 3))
    y = rng.uniform(size=(12, 13, 3))
    assert abs(OS.ssim(x, x) - 1.0) < 1e-12
    assert np.abs(OS.ssim_grad(x, x)).max() < 1e-12
    assert abs(OS.ssim(x, y) - OS.ssim(y, x)) < 1e-14
    assert OS.ssim(x, y) < 1.0


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_loss_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(8, 11, 3))
    y = rng.uniform(size=(8, 11, 3))
    _, g = OS.ssim_l1_loss_grad(x, y, n_views=2, lam=lam)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 5, 1), (7, 10, 2), (4, 0, 1), (2, 7, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (OS.ssim_l1_loss_grad(xp, y, 2, lam)[0] - OS.ssim_l1_loss_grad(xm, y, 2, lam)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7 * max(1.0, abs(g[idx])) + 1e-9, (idx, fd, g[idx])
