"""Image loss of the fine-tuning stage and its gradient (oracle, test infrastructure only).

Sec. 4.4 computes the image-space loss "as in" 3D Gaussian Splatting:
L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2.  SSIM follows Wang et
al. (2004) with an 11x11 Gaussian window (sigma 1.5, normalised to sum 1),
C1 = 0.01^2, C2 = 0.03^2, computed per channel with zero padding ("same"
size) and averaged over all pixels, channels and views.  L1 is the mean
absolute difference over the same elements.  Readings: sign(0) = 0 for the
L1 subgradient; images are planar (V, 3, H, W).

The windowed sums are written as the direct 2D sum over the 121 window
offsets, without separation into row and column passes.
"""

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WIN = 11
SIGMA = 1.5


def gaussian_window():
    """Normalised 11x11 window w[a, b] = g[a] g[b], g[i] ~ exp(-(i-5)^2 / (2 1.5^2))."""
    i = np.arange(WIN, dtype=np.float64) - WIN // 2
    g = np.exp(-(i * i) / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def window_sum(img, w):
    """out[y, x] = sum_{a,b} w[a, b] img[y + a - 5, x + b - 5], zero outside (last two axes)."""
    r = WIN // 2
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W + 2 * r), dtype=np.float64)
    pad[..., r:r + H, r:r + W] = img
    out = np.zeros(img.shape, dtype=np.float64)
    for a in range(WIN):
        for b in range(WIN):
            out += w[a, b] * pad[..., a:a + H, b:b + W]
    return out


def ssim_terms(x, y):
    """Per-pixel SSIM map and the pieces its gradient needs."""
    w = gaussian_window()
    mx, my = window_sum(x, w), window_sum(y, w)
    exx, eyy, exy = window_sum(x * x, w), window_sum(y * y, w), window_sum(x * y, w)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    return dict(w=w, mx=mx, my=my, A1=A1, A2=A2, B1=B1, B2=B2, ssim=A1 * A2 / (B1 * B2))


def loss(img, target, lam=0.2):
    """Scalar L for planar images of shape (..., H, W)."""
    x = np.asarray(img, dtype=np.float64)
    y = np.asarray(target, dtype=np.float64)
    l1 = np.abs(x - y).mean()
    s = ssim_terms(x, y)["ssim"].mean()
    return (1.0 - lam) * l1 + lam * (1.0 - s)


def loss_and_grad(img, target, lam=0.2):
    """(L, dL/dimg).

    With m1 = w*x, m2 = w*(x^2), m3 = w*(x y) the SSIM map depends on x only
    through these windowed moments, so
      d sum(ssim) / dx[p] = sum_q w(q - p) [ds/dm1(q) + 2 x[p] ds/dm2(q) + y[p] ds/dm3(q)]
    with ds/dm1 = 2 my (A2 - A1) / (B1 B2) - 2 mx ssim (1/B1 - 1/B2),
    ds/dm2 = -ssim / B2 and ds/dm3 = 2 A1 / (B1 B2).
    """
    x = np.asarray(img, dtype=np.float64)
    y = np.asarray(target, dtype=np.float64)
    n = x.size
    s = ssim_terms(x, y)
    ssim = s["ssim"]
    L = (1.0 - lam) * np.abs(x - y).mean() + lam * (1.0 - ssim.mean())
    B1B2 = s["B1"] * s["B2"]
    g1 = 2 * s["my"] * (s["A2"] - s["A1"]) / B1B2 - 2 * s["mx"] * ssim * (1 / s["B1"] - 1 / s["B2"])
    g2 = -ssim / s["B2"]
    g3 = 2 * s["A1"] / B1B2
    w = s["w"]  # symmetric, so the adjoint window sum is the same sum
    dssim = window_sum(g1, w) + 2 * x * window_sum(g2, w) + y * window_sum(g3, w)
    grad = (1.0 - lam) * np.sign(x - y) / n - lam * dssim / n
    return L, grad
