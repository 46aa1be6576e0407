"""Off-axis pins for the oracle's EWA projection (Sec. 4.4, projected "as in" 3D
Gaussian Splatting: Sigma' = J W Sigma W^T J^T + 0.3 I with J the Jacobian of the
perspective map at the Gaussian's camera-space mean).

None of these checks restates the oracle's own J / T = J W construction:
  * the Jacobian of the world -> pixel map is taken by central differences of
    the pinhole map itself, so a sign or index slip in the analytic J, or a
    transposed world -> camera rotation, changes Sigma';
  * a Monte-Carlo sample of 3D points of a small Gaussian, each projected
    exactly, has a sample covariance equal to Sigma' - 0.3 I up to the
    linearisation and sampling error;
  * the projected mean lies on the ray the DVR oracle casts through that image
    point (an independent construction of the same camera: origin -R^T t,
    direction R^T d);
  * past the image extended by 15% per side, the Jacobian is evaluated at the
    point moved to that limit (pixel coordinate -0.15 W or 1.15 W, and the same
    for H), at the same depth.
"""

import numpy as np
import pytest

from oracle import dvr, raster
from oracle.raster import PJ
from vbm_inputs import orbit_cameras


def _gaussian(mean, log_scale, quat, logit=1.0):
    P = np.zeros((14, 1))
    P[0:3, 0] = mean
    P[3:6, 0] = log_scale
    P[6:10, 0] = quat
    P[10, 0] = logit
    P[11:14, 0] = (0.3, 0.6, 0.9)
    return P


def _pixel_of(cam, p):
    """World point -> continuous image coordinates through the pinhole camera
    (camera frame x right, y down, z forward; p_c = R p + t)."""
    R = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    pc = R @ np.asarray(p, dtype=np.float64) + np.asarray(cam["t"], dtype=np.float64)
    return np.array([cam["fx"] * pc[0] / pc[2] + cam["cx"], cam["fy"] * pc[1] / pc[2] + cam["cy"]])


def _fd_jacobian(cam, p, h=1e-4):
    """2x3 Jacobian d(pixel)/d(world point) by central differences (O(h^2) error)."""
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pixel_of(cam, p + e) - _pixel_of(cam, p - e)) / (2 * h)
    return J


def _sigma3d(log_scale, quat):
    """Sigma = R diag(s^2) R^T from the rotation scipy builds for the unit quaternion."""
    from scipy.spatial.transform import Rotation
    w, x, y, z = np.asarray(quat, dtype=np.float64) / np.linalg.norm(quat)
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()          # scipy's (x, y, z, w) order
    return Rq @ np.diag(np.exp(2 * np.asarray(log_scale, dtype=np.float64))) @ Rq.T


def _cov2d(pj):
    """The oracle's 2D covariance: the inverse of its conic [[A, B], [B, C]]."""
    return np.linalg.inv(np.array([[pj[PJ["A"]], pj[PJ["B"]]], [pj[PJ["B"]], pj[PJ["C"]]]]))


def _cams():
    # orbit cameras: general rotations (azimuth pi/7 + 2 pi v / 3, elevation +-20 deg)
    cams = orbit_cameras((64, 64, 64), 3, 160, 120)
    # and one with a principal point off the image centre and fx != fy
    c = dict(cams[1])
    c["fx"], c["fy"], c["cx"], c["cy"] = 131.0, 97.0, 71.3, 52.9
    return cams + [c]


def _off_axis_points(cam, n, seed):
    """World points that project inside the image well away from its centre."""
    rng = np.random.default_rng(seed)
    R = np.asarray(cam["R"]).reshape(3, 3)
    t = np.asarray(cam["t"])
    out = []
    while len(out) < n:
        u = rng.uniform(0.05, 0.95) * cam["width"]
        v = rng.uniform(0.05, 0.95) * cam["height"]
        if abs(u - cam["width"] / 2) < 0.2 * cam["width"] and abs(v - cam["height"] / 2) < 0.2 * cam["height"]:
            continue
        z = rng.uniform(60.0, 170.0)
        pc = np.array([(u - cam["cx"]) / cam["fx"] * z, (v - cam["cy"]) / cam["fy"] * z, z])
        out.append(R.T @ (pc - t))
    return out


@pytest.mark.parametrize("ci", range(4))
def test_isotropic_off_axis_matches_fd_jacobian(ci):
    """Isotropic Sigma = s^2 I: Sigma' = s^2 J J^T + 0.3 I with J the finite-difference
    Jacobian of the pinhole map (rotation-invariant 3D part, so this pins J alone)."""
    cam = _cams()[ci]
    for k, mu in enumerate(_off_axis_points(cam, 6, seed=ci)):
        s = 0.6 + 0.3 * k
        P = _gaussian(mu, [np.log(s)] * 3, (0.9, 0.1, -0.3, 0.2))
        pj = raster.project(P, cam, [0], 16, 16)[0]
        J = _fd_jacobian(cam, mu)
        want = s * s * J @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(_cov2d(pj), want, rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose([pj[PJ["U"]], pj[PJ["V"]]], _pixel_of(cam, mu), rtol=0, atol=1e-9)
        R = np.asarray(cam["R"]).reshape(3, 3)
        assert pj[PJ["DEPTH"]] == pytest.approx((R @ mu + np.asarray(cam["t"]))[2], rel=1e-13)


@pytest.mark.parametrize("ci", range(4))
def test_anisotropic_off_axis_matches_fd_jacobian(ci):
    """Rotated anisotropic Sigma: Sigma' = J Sigma J^T + 0.3 I, J by finite differences of
    the world -> pixel map (a transposed world -> camera rotation changes J)."""
    cam = _cams()[ci]
    rng = np.random.default_rng(10 + ci)
    for mu in _off_axis_points(cam, 8, seed=20 + ci):
        ls = rng.uniform(-0.7, 1.0, 3)
        q = rng.normal(size=4)
        P = _gaussian(mu, ls, q)
        pj = raster.project(P, cam, [0], 16, 16)[0]
        J = _fd_jacobian(cam, mu)
        want = J @ _sigma3d(ls, q) @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(_cov2d(pj), want, rtol=1e-7, atol=1e-9)


def test_monte_carlo_sample_covariance():
    """Points drawn from a small off-axis Gaussian and projected exactly have a sample
    covariance equal to Sigma' - 0.3 I (first-order EWA; sigma / z ~ 2e-3 keeps the
    linearisation error far below the sampling error of 2e5 samples)."""
    cam = _cams()[0]
    rng = np.random.default_rng(5)
    mu = _off_axis_points(cam, 1, seed=7)[0]
    ls = np.log([0.12, 0.35, 0.2])
    q = (0.4, -0.5, 0.6, 0.3)
    P = _gaussian(mu, ls, q)
    pj = raster.project(P, cam, [0], 16, 16)[0]
    want = _cov2d(pj) - 0.3 * np.eye(2)
    Sig = _sigma3d(ls, q)
    X = rng.multivariate_normal(mu, Sig, size=200000)
    R = np.asarray(cam["R"]).reshape(3, 3)
    pc = X @ R.T + np.asarray(cam["t"])
    uv = np.stack([cam["fx"] * pc[:, 0] / pc[:, 2] + cam["cx"], cam["fy"] * pc[:, 1] / pc[:, 2] + cam["cy"]], 1)
    got = np.cov(uv.T)
    scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    assert np.abs(got - want).max() < 0.02 * scale.max(), (got, want)
    assert np.abs(uv.mean(0) - [pj[PJ["U"]], pj[PJ["V"]]]).max() < 0.02 * np.sqrt(np.diag(want)).max()


@pytest.mark.parametrize("ci", range(4))
def test_projected_mean_lies_on_the_dvr_ray(ci):
    """The DVR oracle casts the ray of image point (x, y) as origin -R^T t, direction
    R^T ((x - cx)/fx, (y - cy)/fy, 1); the Gaussian's centre lies on the ray through
    its own projected mean."""
    cam = _cams()[ci]
    for mu in _off_axis_points(cam, 10, seed=30 + ci):
        P = _gaussian(mu, [0.0] * 3, (1, 0, 0, 0))
        pj = raster.project(P, cam, [0], 16, 16)[0]
        # ray_setup adds the pixel-centre half: pass the continuous point minus 1/2
        o, d, _, _ = dvr.ray_setup(cam, np.array([pj[PJ["U"]] - 0.5]), np.array([pj[PJ["V"]] - 0.5]),
                                   (64, 64, 64))
        w = mu - o
        along = w @ d[0]
        assert along > 0
        assert np.linalg.norm(w - along * d[0]) < 1e-9 * np.linalg.norm(w)


@pytest.mark.parametrize("side", ["left", "right", "top", "bottom"])
def test_frustum_clamp_moves_the_jacobian_to_the_guard_band(side):
    """A Gaussian beyond the image extended by 15% per side is projected with the
    Jacobian of the point at the same depth moved onto that limit: pixel coordinate
    -0.15 W / 1.15 W (x) or -0.15 H / 1.15 H (y); its mean is not moved."""
    cam = _cams()[3]                                  # off-centre principal point, fx != fy
    W, H = cam["width"], cam["height"]
    R = np.asarray(cam["R"]).reshape(3, 3)
    t = np.asarray(cam["t"])
    z = 90.0
    u, v = {"left": (-0.6 * W, 0.3 * H), "right": (1.7 * W, 0.6 * H),
            "top": (0.4 * W, -0.5 * H), "bottom": (0.7 * W, 1.9 * H)}[side]
    ul = min(max(u, -0.15 * W), 1.15 * W)
    vl = min(max(v, -0.15 * H), 1.15 * H)
    assert (ul, vl) != (u, v)

    def world(uu, vv):
        return R.T @ (np.array([(uu - cam["cx"]) / cam["fx"] * z, (vv - cam["cy"]) / cam["fy"] * z, z]) - t)
    mu = world(u, v)
    ls = np.log([1.5, 0.7, 2.2])
    q = (0.8, 0.2, -0.4, 0.1)
    P = _gaussian(mu, ls, q)
    pj = raster.project(P, cam, [0], 16, 16)[0]
    J = _fd_jacobian(cam, world(ul, vl))
    want = J @ _sigma3d(ls, q) @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(_cov2d(pj), want, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose([pj[PJ["U"]], pj[PJ["V"]]], [u, v], atol=1e-8)
    # inside the guard band nothing is clamped: the limit is exactly 15%
    for frac in (-0.149, 1.149):
        mu_in = world(frac * W, 0.5 * H)
        pj_in = raster.project(_gaussian(mu_in, ls, q), cam, [0], 16, 16)[0]
        J_in = _fd_jacobian(cam, mu_in)
        np.testing.assert_allclose(_cov2d(pj_in), J_in @ _sigma3d(ls, q) @ J_in.T + 0.3 * np.eye(2),
                                   rtol=1e-7, atol=1e-9)
