"""Pins for the oracle's EWA projection, binning, compositing and their derivative
(Sec. 4.4, computed "as in" 3D Gaussian Splatting)."""

import numpy as np
import pytest

from oracle import raster
from oracle.raster import PJ
from vbm_inputs import gaussians_in_view, orbit_cameras


def _simple_camera(W=64, H=48, f=50.0):
    return dict(R=np.eye(3), t=np.zeros(3), fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, znear=0.2,
                width=W, height=H)


def _one_gaussian(mean, sigma, logit=0.5, color=(0.2, 0.5, 0.9), quat=(1, 0, 0, 0)):
    P = np.zeros((14, 1))
    P[0:3, 0] = mean
    P[3:6, 0] = np.log(sigma)
    P[6:10, 0] = quat
    P[10, 0] = logit
    P[11:14, 0] = color
    return P


@pytest.mark.parametrize("sigma,z", [(0.5, 10.0), (2.0, 25.0), (1.3, 4.0)])
def test_on_axis_isotropic_projection(sigma, z):
    """Sigma' = (f^2 sigma^2 / z^2 + 0.3) I exactly; conic = its inverse; mean2D = (cx, cy);
    lambda_max = a + sqrt(0.1) for an isotropic 2D covariance."""
    cam = _simple_camera()
    f = cam["fx"]
    P = _one_gaussian((0.0, 0.0, z), sigma, quat=(0.3, -0.2, 0.7, 0.1))   # rotation irrelevant
    pj = raster.project(P, cam, [0], 16, 16)[0]
    a = f * f * sigma * sigma / (z * z) + 0.3
    assert pj[PJ["A"]] == pytest.approx(1 / a, rel=1e-12)
    assert pj[PJ["C"]] == pytest.approx(1 / a, rel=1e-12)
    assert abs(pj[PJ["B"]]) < 1e-14
    assert pj[PJ["U"]] == pytest.approx(cam["cx"], abs=1e-12)
    assert pj[PJ["V"]] == pytest.approx(cam["cy"], abs=1e-12)
    assert pj[PJ["RADIUS"]] == np.ceil(3 * np.sqrt(a + np.sqrt(0.1)))   # o = 0.62: k = 3
    assert pj[PJ["DEPTH"]] == pytest.approx(z)
    assert pj[PJ["OPAC"]] == pytest.approx(1 / (1 + np.exp(-0.5)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_every_visible_pixel_is_inside_the_tile_rectangle(seed):
    """The radius rule keeps every pixel where o e^power >= 1/255 inside the Gaussian's tile
    rectangle (checked by evaluating the splat at every pixel), and a Gaussian whose opacity
    is below 1/255 gets no tiles."""
    W, H = 96, 80
    cams = orbit_cameras((32, 32, 32), 1, W, H)
    P = gaussians_in_view(300, 32, seed=seed, opacity_logit_range=(-7.0, 3.0))
    pj = raster.project(P, cams[0], np.arange(300), 16, 16)
    jj, ii = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    n_visible = 0
    for g in range(300):
        r = pj[g]
        o = r[PJ["OPAC"]]
        if o < 1 / 255:
            assert r[PJ["TOUCHED"]] == 0
            continue
        if r[PJ["RADIUS"]] == 0:
            continue
        dx, dy = r[PJ["U"]] - ii, r[PJ["V"]] - jj
        power = -0.5 * (r[PJ["A"]] * dx * dx + r[PJ["C"]] * dy * dy) - r[PJ["B"]] * dx * dy
        vis = o * np.exp(power) >= 1 / 255
        n_visible += int(vis.any())
        tx, ty = (ii // 16).astype(int), (jj // 16).astype(int)
        inside = (tx >= r[PJ["X0"]]) & (tx < r[PJ["X1"]]) & (ty >= r[PJ["Y0"]]) & (ty < r[PJ["Y1"]])
        assert not (vis & ~inside).any(), g
    assert n_visible > 50


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_every_visible_pixel_is_in_a_listed_tile(seed):
    """The binning lists, of each rectangle, only the tiles passing the exact tile test;
    every pixel where o e^power >= 1/255 (evaluated at every pixel) lies in a listed tile,
    and elongated splats leave some tiles of their rectangle unlisted."""
    W, H = 96, 80
    cams = orbit_cameras((32, 32, 32), 1, W, H)
    P = gaussians_in_view(300, 32, seed=seed, scale_range=(0.3, 4.0), opacity_logit_range=(-5.0, 3.0))
    out = raster.splat_forward(P, cams, 16, 16)
    listed = set(zip(out["tiles"].tolist(), out["items"].tolist()))
    jj, ii = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    tile_of = (jj // 16).astype(int) * ((W + 15) // 16) + (ii // 16).astype(int)
    unlisted = 0
    for g in range(300):
        r = out["proj"][g]
        if r[PJ["RADIUS"]] == 0 or r[PJ["OPAC"]] < 1 / 255:
            continue
        dx, dy = r[PJ["U"]] - ii, r[PJ["V"]] - jj
        power = -0.5 * (r[PJ["A"]] * dx * dx + r[PJ["C"]] * dy * dy) - r[PJ["B"]] * dx * dy
        vis = r[PJ["OPAC"]] * np.exp(power) >= 1 / 255
        for t in np.unique(tile_of[vis]):
            assert (int(t), g) in listed, (g, t)
        area = (r[PJ["X1"]] - r[PJ["X0"]]) * (r[PJ["Y1"]] - r[PJ["Y0"]])
        assert r[PJ["TOUCHED"]] <= area
        unlisted += int(area - r[PJ["TOUCHED"]])
    assert unlisted > 0


def test_tile_min_q_is_the_minimum_over_the_rectangle():
    """tile_min_q against brute-force minimisation of the quadratic form on a dense grid of
    the rectangle (edges included), for random positive-definite conics and rectangles,
    with the splat centre inside, beside and diagonal to the rectangle."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        L = rng.normal(size=(2, 2)) * rng.uniform(0.05, 2.0)
        M = L @ L.T + np.eye(2) * rng.uniform(0.01, 0.5)
        A, B, C = M[0, 0], M[0, 1], M[1, 1]
        x0, y0 = rng.uniform(-10, 10, 2)
        x1, y1 = x0 + rng.uniform(0.5, 12), y0 + rng.uniform(0.5, 12)
        u, v = rng.uniform(-25, 25, 2)
        xs, ys = np.linspace(x0, x1, 801), np.linspace(y0, y1, 801)
        X, Y = np.meshgrid(xs, ys)
        dX, dY = X - u, Y - v
        brute = (A * dX * dX + 2 * B * dX * dY + C * dY * dY).min()
        got = raster.tile_min_q(u, v, A, B, C, x0, x1, y0, y1)
        assert got <= brute + 1e-9 * max(1.0, brute)
        # the grid spacing bounds how far the grid minimum can lie above the true one
        h = max(xs[1] - xs[0], ys[1] - ys[0])
        slope = 2 * (abs(A) + abs(B) + abs(C)) * (max(abs(x1 - u), abs(x0 - u)) + max(abs(y1 - v), abs(y0 - v)))
        assert brute - got <= slope * h + 1e-9


def _four_edge_f32(u, v, A, B, C, bc, ba, x0, x1, y0, y1):
    """All four edges in float32 (numpy scalars round every operation), the order of the
    binning test's four-edge form."""
    f = np.float32
    u, v, A, B, C, bc, ba, x0, x1, y0, y1 = (f(a) for a in (u, v, A, B, C, bc, ba, x0, x1, y0, y1))
    if x0 <= u <= x1 and y0 <= v <= y1:
        return 0.0
    best = np.inf
    for e in (0, 1):
        dx = (x1 if e else x0) - u
        dy = min(max(v - bc * dx, y0), y1) - v
        best = min(best, (A * dx) * dx + ((f(2) * B) * dx) * dy + (C * dy) * dy)
        ey = (y1 if e else y0) - v
        ex = min(max(u - ba * ey, x0), x1) - u
        best = min(best, (A * ex) * ex + ((f(2) * B) * ex) * ey + (C * ey) * ey)
    return float(best)


def test_tile_min_q_two_facing_edges_suffice():
    """The float32 tile test evaluates only the edges whose half-planes exclude the centre.
    The minimum of a convex quadratic over a box lies on such an edge, so its value equals
    the four-edge FP64 definition to float32 rounding and, where the kept edges hold the
    minimum, the float32 four-edge form bit for bit; cases put the centre inside, beside,
    diagonal to and on the lines through the rectangle's edges, with strongly tilted
    ellipses."""
    rng = np.random.default_rng(41)
    same = 0
    for it in range(3000):
        L = rng.normal(size=(2, 2)) * rng.uniform(0.05, 2.0)
        M = L @ L.T + np.eye(2) * rng.uniform(0.001, 0.5)
        A, B, C = (float(np.float32(a)) for a in (M[0, 0], M[0, 1], M[1, 1]))
        x0, y0 = (float(np.float32(a)) for a in rng.uniform(-10, 10, 2))
        x1, y1 = float(np.float32(x0 + rng.uniform(0.5, 12))), float(np.float32(y0 + rng.uniform(0.5, 12)))
        u, v = (float(np.float32(a)) for a in rng.uniform(-25, 25, 2))
        if it % 5 == 1:
            u = x0 if it % 2 else x1          # on a vertical edge's line
        if it % 7 == 2:
            v = y0 if it % 3 else y1          # on a horizontal edge's line
        bc, ba = float(np.float32(B) / np.float32(C)), float(np.float32(B) / np.float32(A))
        got = raster.tile_min_q_f32(u, v, A, B, C, bc, ba, x0, x1, y0, y1)
        ref64 = raster.tile_min_q(u, v, A, B, C, x0, x1, y0, y1)
        four = _four_edge_f32(u, v, A, B, C, bc, ba, x0, x1, y0, y1)
        scale = (abs(A) + abs(B) + abs(C)) * (abs(u) + abs(v) + abs(x0) + abs(x1) + abs(y0) + abs(y1) + 1) ** 2
        assert abs(got - ref64) <= 2e-6 * scale, (it, got, ref64)
        assert got >= four                  # dropping edges can only raise the float minimum
        assert got - four <= 2e-6 * scale    # and then only by rounding
        same += got == four
    assert same > 0.99 * 3000


def test_two_facing_edges_hold_the_minimum_fp64():
    """In exact arithmetic the two-edge rule is the definition: in FP64 the edges facing
    the centre give the four-edge minimum of the oracle to 1e-12 relative (both edges of a
    corner evaluate the same point)."""
    rng = np.random.default_rng(42)
    for it in range(3000):
        L = rng.normal(size=(2, 2)) * rng.uniform(0.05, 2.0)
        M = L @ L.T + np.eye(2) * rng.uniform(0.001, 0.5)
        A, B, C = M[0, 0], M[0, 1], M[1, 1]
        x0, y0 = rng.uniform(-10, 10, 2)
        x1, y1 = x0 + rng.uniform(0.5, 12), y0 + rng.uniform(0.5, 12)
        u, v = rng.uniform(-25, 25, 2)
        if x0 <= u <= x1 and y0 <= v <= y1:
            continue
        cand = []
        if u < x0 or u > x1:
            dx = (x0 if u < x0 else x1) - u
            dy = min(max(v - B / C * dx, y0), y1) - v
            cand.append(A * dx * dx + 2 * B * dx * dy + C * dy * dy)
        if v < y0 or v > y1:
            ey = (y0 if v < y0 else y1) - v
            ex = min(max(u - B / A * ey, x0), x1) - u
            cand.append(A * ex * ex + 2 * B * ex * ey + C * ey * ey)
        ref = raster.tile_min_q(u, v, A, B, C, x0, x1, y0, y1)
        assert abs(min(cand) - ref) <= 1e-12 * max(1.0, ref), (it, min(cand), ref)


def test_projection_covariance_is_symmetric_pd_and_culls():
    cams = orbit_cameras((32, 32, 32), 3, 80, 60)
    P = gaussians_in_view(200, 32, seed=3)
    for cam in cams:
        pj = raster.project(P, cam, np.arange(200), 16, 16)
        A, B, C = pj[:, PJ["A"]], pj[:, PJ["B"]], pj[:, PJ["C"]]
        vis = pj[:, PJ["TOUCHED"]] > 0
        assert vis.any()
        assert np.all(A[vis] > 0) and np.all(A[vis] * C[vis] - B[vis] ** 2 > 0)
    # behind the camera: culled
    Pb = _one_gaussian((0.0, 0.0, 0.1), 1.0)
    assert raster.project(Pb, _simple_camera(), [0], 16, 16)[0, PJ["TOUCHED"]] == 0


def test_single_gaussian_closed_form_image():
    cam = _simple_camera(W=48, H=40, f=30.0)
    sigma, z = 1.5, 12.0
    P = _one_gaussian((0.7, -0.4, z), sigma, logit=1.2, color=(0.3, 0.6, 0.9))
    out = raster.splat_forward(P, [cam], 16, 16, bg=(0.1, 0.0, 0.2))
    pj = out["proj"][0]
    u, v = pj[PJ["U"]], pj[PJ["V"]]
    A, B, C, o = pj[PJ["A"]], pj[PJ["B"]], pj[PJ["C"]], pj[PJ["OPAC"]]
    x0, y0, x1, y1 = (int(pj[PJ[k]]) for k in ("X0", "Y0", "X1", "Y1"))
    jj, ii = np.meshgrid(np.arange(40), np.arange(48), indexing="ij")
    dx, dy = u - (ii + 0.5), v - (jj + 0.5)
    alpha = np.minimum(0.99, o * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy))
    inrect = (ii // 16 >= x0) & (ii // 16 < x1) & (jj // 16 >= y0) & (jj // 16 < y1)
    alpha = np.where(inrect & (alpha >= 1 / 255), alpha, 0.0)
    for ch, (c, b) in enumerate(zip((0.3, 0.6, 0.9), (0.1, 0.0, 0.2))):
        assert np.allclose(out["img"][0, ch], c * alpha + (1 - alpha) * b, atol=1e-14)
    assert np.allclose(out["T_final"][0], 1 - alpha, atol=1e-14)


def _scene(seed, n=300, G=32, W=96, H=80, V=2):
    cams = orbit_cameras((G, G, G), V, W, H)
    P = gaussians_in_view(n, G, seed=seed)
    return P, cams


def test_tiled_equals_brute_force_and_weights_sum_to_one():
    P, cams = _scene(1)
    P[11:14] = 1.0       # unit colour: C = sum_k alpha_k T_k, so C + T_final = 1
    out = raster.splat_forward(P, cams, 16, 16)
    img, T = raster.render_brute(len(cams), out["W"], out["H"], 16, 16, out["view_of"], out["rect"],
                                 out["proj"][:, PJ["DEPTH"]], out["splat"], out["color"], out["bg"])
    assert np.array_equal(img, out["img"]) and np.array_equal(T, out["T_final"])
    for ch in range(3):
        assert np.allclose(out["img"][:, ch] + out["T_final"], 1.0, atol=1e-12)
    assert np.all(out["T_final"] >= 1e-4) and np.all(out["T_final"] <= 1.0)


def test_binning_is_complete_and_ordered():
    P, cams = _scene(2, V=3, W=70, H=50)
    out = raster.splat_forward(P, cams, 16, 16)
    tiles, items, ranges = out["tiles"], out["items"], out["ranges"]
    TX, TY = (70 + 15) // 16, (50 + 15) // 16
    # every (item, listed tile of its rectangle) pair appears exactly once
    expect = set()
    for it, (x0, y0, x1, y1) in enumerate(out["rect"]):
        u, v, A, B, C, o = out["splat"][it]
        tau = 2.0 * (np.log(255.0 * o) + 1e-3) if o > 0 else -1.0
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                r = (tx * 16 + 0.5, min(tx * 16 + 16, 70) - 0.5, ty * 16 + 0.5, min(ty * 16 + 16, 50) - 0.5)
                if raster.tile_min_q(u, v, A, B, C, *r) <= tau:
                    expect.add((out["view_of"][it] * TX * TY + ty * TX + tx, it))
    got = list(zip(tiles.tolist(), items.tolist()))
    assert len(got) == len(expect) and set(got) == expect
    depth = out["proj"][:, PJ["DEPTH"]]
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        seg = items[s:e]
        assert np.all(tiles[s:e] == t)
        key = list(zip(depth[seg], seg))
        assert key == sorted(key)


def _linear_loss_grad_check(P, cams, w, wa=None, bg=(0.0, 0.0, 0.0), h=1e-6):
    fwd = raster.splat_forward(P, cams, 16, 16, bg=bg)
    grad, _, _ = raster.splat_backward(fwd, P, cams, w, wa)

    def L(Pp):
        o = raster.splat_forward(Pp, cams, 16, 16, bg=bg)
        val = (o["img"] * w).sum()
        if wa is not None:
            val += ((1.0 - o["T_final"]) * wa).sum()
        return val
    fd = np.zeros_like(P)
    for r in range(14):
        for g in range(P.shape[1]):
            Pp, Pm = P.copy(), P.copy()
            step = h * max(1.0, abs(P[r, g]))
            Pp[r, g] += step
            Pm[r, g] -= step
            fd[r, g] = (L(Pp) - L(Pm)) / (2 * step)
    return grad, fd, fwd


def _far_from_cutoffs(fwd, tol=1e-3):
    pj = fwd["proj"]
    vis = pj[:, PJ["TOUCHED"]] > 0
    return (fwd["margin"].min() > tol and pj[vis, PJ["M_RADIUS"]].min() > tol
            and pj[vis, PJ["M_RECT"]].min() > tol and pj[vis, PJ["M_CLAMP"]].min() > tol)


@pytest.mark.parametrize("with_alpha", [False, True])
def test_backward_matches_central_differences(with_alpha):
    G, W, H = 16, 40, 32
    cams = orbit_cameras((G, G, G), 2, W, H)
    for seed in range(50):
        P = gaussians_in_view(4, G, seed=100 + seed, scale_range=(0.8, 2.0),
                              opacity_logit_range=(-1.5, 1.0))
        fwd = raster.splat_forward(P, cams, 16, 16)
        if _far_from_cutoffs(fwd):
            break
    else:
        pytest.fail("no scene far from the cut-offs")
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((2, 3, H, W))
    wa = rng.standard_normal((2, H, W)) if with_alpha else None
    grad, fd, _ = _linear_loss_grad_check(P, cams, w, wa, bg=(0.2, 0.1, 0.3))
    scale = np.abs(fd).max()
    assert np.abs(grad - fd).max() < 1e-6 * scale
    assert np.abs(grad).max() > 0


def test_projection_backward_matches_differences_with_clamp():
    """Per-item chain rule, including a Gaussian far outside the frustum (clamped Jacobian)."""
    cam = _simple_camera(W=64, H=48, f=40.0)
    rng = np.random.default_rng(11)
    P = np.zeros((14, 3))
    P[0:3, 0], P[0:3, 1], P[0:3, 2] = (0.5, -0.3, 6.0), (30.0, 2.0, 5.0), (-1.0, 20.0, 8.0)
    P[3:6] = np.log(rng.uniform(0.3, 1.5, size=(3, 3)))
    P[6:10] = rng.standard_normal((4, 3))
    P[10] = rng.uniform(-1, 1, size=3)
    g6 = rng.standard_normal((3, 6))
    out = raster.project_bwd(P, cam, np.arange(3), g6)
    pj = raster.project(P, cam, np.arange(3), 16, 16)
    assert pj[1, PJ["M_CLAMP"]] > 0.1 and pj[2, PJ["M_CLAMP"]] > 0.1   # both clamped, not at the kink
    cols = [PJ["U"], PJ["V"], PJ["A"], PJ["B"], PJ["C"], PJ["OPAC"]]
    for g in range(3):
        for r in range(14):
            h = 1e-6 * max(1.0, abs(P[r, g]))
            Pp, Pm = P.copy(), P.copy()
            Pp[r, g] += h
            Pm[r, g] -= h
            fp = raster.project(Pp, cam, [g], 16, 16)[0, cols]
            fm = raster.project(Pm, cam, [g], 16, 16)[0, cols]
            fd = ((fp - fm) / (2 * h) * g6[g]).sum()
            assert out[g, r] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(out[g]).max()), (g, r)


def test_full_loss_gradient_through_splatting():
    """Chain of the composite L1 + D-SSIM loss through the splatting backward (Sec. 4.4)."""
    from oracle.loss import loss, loss_and_grad
    G, W, H = 16, 40, 32
    cams = orbit_cameras((G, G, G), 1, W, H)
    for seed in range(50):
        P = gaussians_in_view(3, G, seed=300 + seed, scale_range=(0.8, 2.0),
                              opacity_logit_range=(-1.5, 1.0))
        fwd = raster.splat_forward(P, cams, 16, 16)
        if _far_from_cutoffs(fwd):
            break
    target = np.random.default_rng(5).uniform(0, 0.3, fwd["img"].shape)
    L0, dimg = loss_and_grad(fwd["img"], target)
    grad, _, _ = raster.splat_backward(fwd, P, cams, dimg)
    for r, g in [(0, 0), (2, 1), (4, 2), (7, 0), (10, 1), (12, 2)]:
        h = 1e-6 * max(1.0, abs(P[r, g]))
        Pp, Pm = P.copy(), P.copy()
        Pp[r, g] += h
        Pm[r, g] -= h
        fd = (loss(raster.splat_forward(Pp, cams)["img"], target)
              - loss(raster.splat_forward(Pm, cams)["img"], target)) / (2 * h)
        assert grad[r, g] == pytest.approx(fd, rel=1e-5, abs=1e-9), (r, g)
