"""SSIM term of the photometric loss -- TEST INFRASTRUCTURE ONLY (see the
package docstring for who may import it).

Section 3 (Eq. loss and its footnote) sets the per-pixel error to L1 and sets
the SSIM term of 3D Gaussian Splatting aside for the analysis; the training
objective of 3D Gaussian Splatting keeps it, and so does this module.  The
paper names SSIM (Wang et al., 2004) as a metric
but fixes none of its constants, so this module takes the published
definition: per channel,

    SSIM(x, y) = ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2))

with mu, s the local means, variances and covariance under an 11x11 Gaussian
window of standard deviation 1.5 (zero padding at the image border), C1 =
0.01^2, C2 = 0.03^2 (dynamic range 1), averaged over pixels and channels, and
the combined loss of Gaussian-splatting training

    loss = (1 - lambda) * L1 + lambda * (1 - SSIM),   lambda = 0.2 by default,

averaged over views like the L1 loss.  Plain float64 numpy: the filter is the
separable window applied as two explicit 11-tap sums; the gradient is the
chain rule through the three filtered moment maps written out term by term.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WINDOW = 11
SIGMA = 1.5


def window_taps(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """Normalised 1-D Gaussian taps; the 2-D window is their outer product."""
    r = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    return g / g.sum()


def gaussian_filter(img: np.ndarray, taps: np.ndarray | None = None) -> np.ndarray:
    """Zero-padded 'same' filtering of a 2-D array by the separable window."""
    w = window_taps() if taps is None else taps
    h = len(w) // 2
    H, W = img.shape
    pad = np.zeros((H + 2 * h, W + 2 * h))
    pad[h:h + H, h:h + W] = img
    rows = np.zeros((H + 2 * h, W))
    for k in range(len(w)):                       # horizontal taps
        rows += w[k] * pad[:, k:k + W]
    out = np.zeros((H, W))
    for k in range(len(w)):                       # vertical taps
        out += w[k] * rows[k:k + H, :]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray):
    """Per-pixel SSIM of one channel and the moments it was built from."""
    F = gaussian_filter
    mx, my = F(x), F(y)
    sxx = F(x * x) - mx * mx
    syy = F(y * y) - my * my
    sxy = F(x * y) - mx * my
    A1, A2 = 2.0 * mx * my + C1, 2.0 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    S = (A1 * A2) / (B1 * B2)
    return S, dict(mx=mx, my=my, A1=A1, A2=A2, B1=B1, B2=B2)


def ssim(image: np.ndarray, target: np.ndarray) -> float:
    """Mean SSIM over pixels and channels of [H, W, 3] images."""
    image = np.asarray(image, np.float64)
    target = np.asarray(target, np.float64)
    return float(np.mean([ssim_map(image[..., c], target[..., c])[0] for c in range(image.shape[2])]))


def ssim_grad(image: np.ndarray, target: np.ndarray) -> np.ndarray:
    """d(mean SSIM)/d(image) for [H, W, 3] images.

    With m = F(x), e = F(x^2), c = F(x y) (F the filter) the map depends on x
    through (m, e, c): s_xx = e - m^2, s_xy = c - m mu_y.  Per pixel q
      dS/dm = S (2 mu_y / A1 - 2 mu_x / B1) + (dS/ds_xx)(-2 mu_x) + (dS/ds_xy)(-mu_y)
      dS/de = dS/ds_xx = -S / B2
      dS/dc = dS/ds_xy = 2 S / A2
    and, F being symmetric with zero padding (its own adjoint),
      d mean(S) / d x(p) = [F(dS/dm) + 2 x F(dS/de) + y F(dS/dc)](p) / (H W C).
    """
    image = np.asarray(image, np.float64)
    target = np.asarray(target, np.float64)
    H, W, Cn = image.shape
    g = np.zeros_like(image)
    for ch in range(Cn):
        x, y = image[..., ch], target[..., ch]
        S, m = ssim_map(x, y)
        dS_dsxx = -S / m["B2"]
        dS_dsxy = 2.0 * S / m["A2"]
        dS_dmx = S * (2.0 * m["my"] / m["A1"] - 2.0 * m["mx"] / m["B1"])
        a = dS_dmx + dS_dsxx * (-2.0 * m["mx"]) + dS_dsxy * (-m["my"])
        g[..., ch] = (gaussian_filter(a) + 2.0 * x * gaussian_filter(dS_dsxx) + y * gaussian_filter(dS_dsxy))
    return g / (H * W * Cn)


def ssim_l1_loss_grad(image, target, n_views: int = 1, lam: float = 0.2):
    """Combined loss of one view, divided by the number of views, and dL/dC:
    ((1 - lam) L1 + lam (1 - SSIM)) / n_views."""
    image = np.asarray(image, np.float64)
    target = np.asarray(target, np.float64)
    H, W, Cn = image.shape
    P = H * W * Cn
    d = image - target
    l1 = np.abs(d).sum() / P
    s = ssim(image, target)
    loss = ((1.0 - lam) * l1 + lam * (1.0 - s)) / n_views
    grad = ((1.0 - lam) * np.sign(d) / P - lam * ssim_grad(image, target)) / n_views
    return loss, grad
