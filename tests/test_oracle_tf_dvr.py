"""Pins for the oracle's transfer function (Sec. 3) and DVR target renderer (Sec. 4.4)."""

import numpy as np
import pytest

from oracle.dvr import render_dvr, ray_setup
from oracle.tf import apply_tf, apply_tf_vectorised
from vbm_inputs import TF_KNOTS_RGBA, TF_KNOTS_X, blob_volume, orbit_cameras
from vbm_inputs.cameras import look_at


def test_tf_at_knots_and_midpoints():
    out = apply_tf(TF_KNOTS_X, TF_KNOTS_X, TF_KNOTS_RGBA)
    assert np.array_equal(out, TF_KNOTS_RGBA)
    mids = 0.5 * (TF_KNOTS_X[1:] + TF_KNOTS_X[:-1])
    assert np.allclose(apply_tf(mids, TF_KNOTS_X, TF_KNOTS_RGBA),
                       0.5 * (TF_KNOTS_RGBA[1:] + TF_KNOTS_RGBA[:-1]), atol=1e-15)


def test_tf_clamp_and_library_interp():
    f = np.random.default_rng(0).uniform(-0.5, 1.5, size=500)
    out = apply_tf(f, TF_KNOTS_X, TF_KNOTS_RGBA)
    for c in range(4):
        assert np.allclose(out[:, c], np.interp(np.clip(f, 0, 1), TF_KNOTS_X, TF_KNOTS_RGBA[:, c]),
                           atol=1e-15)
    assert np.allclose(apply_tf_vectorised(f, TF_KNOTS_X, TF_KNOTS_RGBA), out, atol=1e-15)


def _axis_camera(G, W=8, H=8):
    """Camera on the +x axis looking at the volume centre: central rays run along -x."""
    pos = np.array([3.0 * G, G / 2.0, G / 2.0])
    R, t = look_at(pos, np.array([G / 2.0, G / 2.0, G / 2.0]))
    return dict(R=R, t=t, fx=40.0, fy=40.0, cx=W / 2.0, cy=H / 2.0, znear=0.2, width=W, height=H)


@pytest.mark.parametrize("f0", [0.3, 0.8])
def test_constant_field_closed_form(f0):
    """Constant field: C = c (1 - (1 - a)^len), 1 - T = 1 - (1 - a)^len with len the chord."""
    G = 16
    F = np.full((G, G, G), f0)
    cam = _axis_camera(G, W=2, H=2)
    rgba = np.interp(f0, TF_KNOTS_X, TF_KNOTS_RGBA[:, 3])
    col = np.array([np.interp(f0, TF_KNOTS_X, TF_KNOTS_RGBA[:, c]) for c in range(3)])
    out = render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam, step=0.5)
    px = np.arange(2, dtype=np.float64)
    for j in range(2):
        o, d, t0, t1 = ray_setup(cam, px, np.full(2, float(j)), (G, G, G))
        for i in range(2):
            L = t1[i] - t0[i]
            T = (1.0 - rgba) ** L
            assert out[3, j, i] == pytest.approx(1.0 - T, abs=1e-12)
            assert np.allclose(out[:3, j, i], col * (1.0 - T), atol=1e-12)
    # the chord of a near-axial ray through the cube is close to the edge length
    o, d, t0, t1 = ray_setup(cam, np.array([1.0]), np.array([1.0]), (G, G, G))
    assert abs((t1[0] - t0[0]) - G) < 0.05 * G


def test_empty_volume_and_miss():
    G = 8
    F = np.zeros((G, G, G))
    cam = orbit_cameras((G, G, G), 1, 16, 16)[0]
    out = render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam)
    assert np.abs(out).max() == 0.0
    cam2 = dict(cam)
    cam2["cx"] = 1e4           # every ray misses the box
    F2 = np.ones((G, G, G))
    assert np.abs(render_dvr(F2, TF_KNOTS_X, TF_KNOTS_RGBA, cam2)).max() == 0.0


def test_transmittance_monotone_along_ray():
    """Zeroing part of the field can only raise T: the TF opacity is non-decreasing in F and
    trilinear samples of the truncated field are never larger."""
    G = 16
    F = blob_volume(G, 3, seed=5).astype(np.float64)
    cam = orbit_cameras((G, G, G), 1, 24, 24)[0]
    full = render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam)
    Ft = F.copy()
    Ft[:, :, G // 2:] = 0.0
    part = render_dvr(Ft, TF_KNOTS_X, TF_KNOTS_RGBA, cam)
    assert np.all(part[3] <= full[3] + 1e-15)
    assert (part[3] < full[3] - 1e-6).any()
    assert np.all((full[3] >= 0) & (full[3] <= 1))


def test_step_convergence():
    """Midpoint rule: halving the step shrinks the change roughly fourfold."""
    G = 16
    F = blob_volume(G, 3, seed=6).astype(np.float64)
    cam = orbit_cameras((G, G, G), 1, 12, 12)[0]
    r = [render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam, step=s) for s in (0.5, 0.25, 0.125)]
    d1 = np.abs(r[0] - r[1]).max()
    d2 = np.abs(r[1] - r[2]).max()
    assert d2 < 0.5 * d1 and d2 < 5e-3


def test_pixel_subset_matches_full_image():
    G = 16
    F = blob_volume(G, 3, seed=7).astype(np.float64)
    cam = orbit_cameras((G, G, G), 2, 20, 16)[1]
    full = render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam)
    pix = [(0, 0), (19, 15), (7, 9)]
    sub = render_dvr(F, TF_KNOTS_X, TF_KNOTS_RGBA, cam, pixels=pix)
    for n, (i, j) in enumerate(pix):
        assert np.allclose(sub[:, n], full[:, j, i], atol=0)


def test_tf_modes_disjoint_and_union_is_their_sum():
    """The five TF modes (Sec. 4.4: each non-zero only over its own value interval)
    have disjoint supports, peak at their interval's midpoint with the tabulated
    colour, and the union TF equals their sum everywhere (checked through the
    oracle's TF on a dense grid, against numpy's own interpolation of each mode)."""
    from vbm_inputs import TF_MODE_EDGES, tf_mode, tf_modes_union
    x = np.linspace(0.0, 1.0, 4001)
    per_mode = []
    for h in range(5):
        kx, krgba = tf_mode(h)
        rgba = apply_tf_vectorised(x, kx, krgba)
        ref = np.stack([np.interp(x, kx, krgba[:, c]) for c in range(4)], axis=-1)
        assert np.allclose(rgba, ref, atol=1e-15)
        a, b = TF_MODE_EDGES[h], TF_MODE_EDGES[h + 1]
        outside = (x <= a) | (x >= b)
        assert np.all(rgba[outside] == 0.0) and np.all(rgba[~outside, 3] > 0.0)
        mid = apply_tf_vectorised(np.array([0.5 * (a + b)]), kx, krgba)[0]
        assert np.array_equal(mid, krgba[2])
        per_mode.append(rgba)
    support = np.stack([m[:, 3] > 0 for m in per_mode])
    assert support.sum(axis=0).max() == 1
    ux, urgba = tf_modes_union()
    assert len(ux) <= 16 and np.all(np.diff(ux) > 0)
    assert np.allclose(apply_tf_vectorised(x, ux, urgba), sum(per_mode), atol=1e-15)
