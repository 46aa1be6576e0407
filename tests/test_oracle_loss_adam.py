"""Pins for the oracle's image loss (Sec. 4.4, 3DGS L1 + D-SSIM) and Adam (Sec. 5.2)."""

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import adam as oadam
from oracle import loss as oloss


def test_window_sum_matches_library_correlation():
    img = np.random.default_rng(0).standard_normal((13, 17))
    w = oloss.gaussian_window()
    ref = correlate2d(img, w, mode="same", boundary="fill", fillvalue=0.0)
    assert np.allclose(oloss.window_sum(img, w), ref, atol=1e-14)
    assert abs(w.sum() - 1.0) < 1e-15 and np.allclose(w, w.T)


def test_ssim_map_matches_per_pixel_definition():
    """Per pixel: weighted means, variances and covariance over the zero-padded window."""
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (9, 12)), rng.uniform(0, 1, (9, 12))
    w = oloss.gaussian_window()
    s = oloss.ssim_terms(x, y)["ssim"]
    H, W = x.shape
    for (r, c) in [(0, 0), (4, 6), (8, 11), (2, 9)]:
        mx = my = exx = eyy = exy = 0.0
        for a in range(11):
            for b in range(11):
                rr, cc = r + a - 5, c + b - 5
                if 0 <= rr < H and 0 <= cc < W:
                    wt = w[a, b]
                    mx += wt * x[rr, cc]; my += wt * y[rr, cc]
                    exx += wt * x[rr, cc] ** 2; eyy += wt * y[rr, cc] ** 2; exy += wt * x[rr, cc] * y[rr, cc]
        vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
        ref = ((2 * mx * my + oloss.C1) * (2 * cxy + oloss.C2)
               / ((mx * mx + my * my + oloss.C1) * (vx + vy + oloss.C2)))
        assert s[r, c] == pytest.approx(ref, rel=1e-12)


def test_identical_images():
    x = np.random.default_rng(2).uniform(0, 1, (2, 3, 10, 14))
    assert oloss.loss(x, x) == pytest.approx(0.0, abs=1e-15)
    assert np.allclose(oloss.ssim_terms(x, x)["ssim"], 1.0, atol=1e-14)


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (2, 3, 7, 9))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    L, g = oloss.loss_and_grad(x, y)
    assert L == pytest.approx(oloss.loss(x, y), rel=1e-14)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 6, 8), (0, 1, 3, 4), (1, 0, 5, 1), (0, 2, 0, 8)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oloss.loss(xp, y) - oloss.loss(xm, y)) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adam_matches_torch_optimizer():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    n = 7
    P = rng.standard_normal((14, n))
    lrs = oadam.default_lrs(32.0)
    m, v = np.zeros_like(P), np.zeros_like(P)
    tp = torch.tensor(P.copy(), dtype=torch.float64, requires_grad=True)
    groups = [dict(params=[]) for _ in oadam.ROW_GROUPS]
    leaves = [torch.tensor(P[lo:hi].copy(), dtype=torch.float64, requires_grad=True)
              for lo, hi in oadam.ROW_GROUPS]
    opt = torch.optim.Adam([dict(params=[leaf], lr=lr) for leaf, lr in zip(leaves, lrs)],
                           betas=(0.9, 0.999), eps=1e-15)
    Pn = P.copy()
    for step in range(1, 6):
        grad = rng.standard_normal((14, n))
        oadam.adam_step(Pn, grad, m, v, step, lrs)
        for leaf, (lo, hi) in zip(leaves, oadam.ROW_GROUPS):
            leaf.grad = torch.tensor(grad[lo:hi])
        opt.step()
    ref = np.concatenate([leaf.detach().numpy() for leaf in leaves])
    assert np.abs(Pn - ref).max() < 1e-12
    del tp, groups
