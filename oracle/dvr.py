"""Emission-absorption volume rendering of the supervision images (oracle).

Test infrastructure only.  Sec. 4.4 renders 64 images per TF "through
volumetric integration" as the fine-tuning targets; the paper's renderer
(ParaView + IndeX, Sec. 5.2) is a graphics application that is unavailable
here, so this is a CPU restatement of emission-absorption ray marching.
Readings (the paper gives no step size, interpolation, opacity correction or
background):
  * ray through the pixel centre (i + 1/2, j + 1/2): camera-space direction
    ((i + 1/2 - cx)/fx, (j + 1/2 - cy)/fy, 1), world direction R^T d
    normalised, origin -R^T t;
  * the volume occupies the box [0, nx] x [0, ny] x [0, nz]; the ray is
    clipped to it (slab test) and to t >= 0;
  * the clipped interval [t0, t1] is cut into segments of length step
    (world units = voxels), the last one possibly shorter; each segment is
    sampled once at its midpoint;
  * sampling: trilinear interpolation of the scalar field at grid coordinate
    p - 1/2 (voxel centres), coordinates clamped to [0, n-1] per axis;
  * the TF (piecewise-linear, oracle.tf) is applied to the interpolated value;
  * opacity correction for a segment of length l: a' = 1 - (1 - a)^l;
  * front to back: C += T a' c, T *= (1 - a'); no early termination; black
    background.  Output (C_r, C_g, C_b, 1 - T).
The last-segment rule makes the result continuous in the ray's exit point.
"""

import numpy as np

from .tf import apply_tf_vectorised


def _trilinear(F, q):
    """Trilinear sample of F[z, y, x] at grid coordinates q (n, 3) = (x, y, z)."""
    nz, ny, nx = F.shape
    dims = np.array([nx, ny, nz], dtype=np.float64)
    qc = np.clip(q, 0.0, dims - 1.0)
    i0 = np.minimum(np.floor(qc).astype(np.int64), np.maximum(dims.astype(np.int64) - 2, 0))
    f = qc - i0
    x0, y0, z0 = i0[:, 0], i0[:, 1], i0[:, 2]
    x1 = np.minimum(x0 + 1, nx - 1)
    y1 = np.minimum(y0 + 1, ny - 1)
    z1 = np.minimum(z0 + 1, nz - 1)
    fx, fy, fz = f[:, 0], f[:, 1], f[:, 2]
    c00 = F[z0, y0, x0] * (1 - fx) + F[z0, y0, x1] * fx
    c10 = F[z0, y1, x0] * (1 - fx) + F[z0, y1, x1] * fx
    c01 = F[z1, y0, x0] * (1 - fx) + F[z1, y0, x1] * fx
    c11 = F[z1, y1, x0] * (1 - fx) + F[z1, y1, x1] * fx
    c0 = c00 * (1 - fy) + c10 * fy
    c1 = c01 * (1 - fy) + c11 * fy
    return c0 * (1 - fz) + c1 * fz


def ray_setup(cam, px, py, dims):
    """Origins, unit directions and clipped [t0, t1] for pixel centres (px, py)."""
    R = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], dtype=np.float64)
    dc = np.stack([(px + 0.5 - cam["cx"]) / cam["fx"], (py + 0.5 - cam["cy"]) / cam["fy"],
                   np.ones_like(px, dtype=np.float64)], axis=1)
    d = dc @ R            # rows: R^T dc
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = -R.T @ t
    box = np.asarray(dims, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (0.0 - o[None, :]) * inv
        tb = (box[None, :] - o[None, :]) * inv
    tmin = np.where(np.isnan(ta), -np.inf, np.minimum(ta, tb))
    tmax = np.where(np.isnan(ta), np.inf, np.maximum(ta, tb))
    # A ray parallel to a slab lies inside it iff its origin does.
    par = d == 0.0
    inside = (o[None, :] >= 0.0) & (o[None, :] <= box[None, :])
    tmin = np.where(par, np.where(inside, -np.inf, np.inf), tmin)
    tmax = np.where(par, np.where(inside, np.inf, -np.inf), tmax)
    t0 = np.maximum(tmin.max(axis=1), 0.0)
    t1 = tmax.min(axis=1)
    return o, d, t0, t1


def render_dvr(F, knots_x, knots_rgba, cam, step=0.5, pixels=None):
    """RGBA (4, H, W) for one camera, or (4, n) for a list of pixels [(i, j), ...]."""
    F = np.asarray(F, dtype=np.float64)
    nz, ny, nx = F.shape
    W, H = cam["width"], cam["height"]
    if pixels is None:
        jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        px, py = ii.reshape(-1).astype(np.float64), jj.reshape(-1).astype(np.float64)
    else:
        pix = np.asarray(pixels, dtype=np.float64).reshape(-1, 2)
        px, py = pix[:, 0], pix[:, 1]
    o, d, t0, t1 = ray_setup(cam, px, py, (nx, ny, nz))
    n = px.size
    C = np.zeros((n, 3))
    T = np.ones(n)
    length = np.where(t1 > t0, t1 - t0, 0.0)
    n_seg = np.ceil(length / step).astype(np.int64)
    for m in range(int(n_seg.max()) if n > 0 else 0):
        act = m < n_seg
        if not act.any():
            break
        idx = np.nonzero(act)[0]
        a_start = t0[idx] + m * step
        seg = np.minimum(step, t1[idx] - a_start)
        tm = a_start + 0.5 * seg
        p = o[None, :] + tm[:, None] * d[idx]
        val = _trilinear(F, p - 0.5)
        rgba = apply_tf_vectorised(val, knots_x, knots_rgba)
        a_corr = 1.0 - (1.0 - rgba[:, 3]) ** seg
        C[idx] += (T[idx] * a_corr)[:, None] * rgba[:, :3]
        T[idx] *= (1.0 - a_corr)
    out = np.concatenate([C.T, (1.0 - T)[None, :]], axis=0)
    if pixels is None:
        return out.reshape(4, H, W)
    return out
