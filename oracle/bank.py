"""Wavelet-to-Gaussian transition bank (oracle, test infrastructure only).

Sec. 4.2.  For every kept subband (j, o):
  1. canonical kernel psi_hat_{j,o}: IDWT of a unit impulse in that subband
     (Eq. 9-10);
  2. normalised magnitude W = |psi| / sum |psi|, region of interest
     R = {x : W(x) > tau max W} (Eq. 13, strict inequality);
  3. W-weighted centroid u and covariance Sigma over R (Eq. 14), which define
     g_{j,o} (Eq. 15);
  4. energy weight w = argmin || |Y| - w G ||^2 + lambda w^2 over R, i.e.
     w = sum |Y| G / (sum G^2 + lambda) (Eq. 16-17), broadcast to RGBA.

Readings:
  * "Centring the impulse at k = 0" on a periodic grid wraps the kernel, so
    the impulse is placed at an interior index k_c and 2^j k_c is subtracted
    from the centroid; the translation theorem (Eq. 12, Supp. Sec. 2) makes
    this exact on the grid.
  * The grid has side 2^j S with S = 16 (bior4.4) so the kernel's support
    (< 7 2^j + 1 samples) never overlaps itself.  For grids above 64^3 the 3D
    IDWT of the impulse is evaluated as the outer product of 1D IDWT
    responses, which the separable transform makes identical (Supp. Sec. 2,
    Step 1; checked against the 3D IDWT on small levels by the tests).
  * tau and lambda are not given: tau = 0.1 and lambda = 1e-6 sum G^2.
  * Coordinates are grid indices; the paper's sub-voxel offset delta ~ (1/2,
    1/2, 1/2) (Eq. 12) is read as the voxel-centre convention (sample i sits
    at i + 1/2 in world units) and is added by the mapping, not stored here.
  * Splat parameters per entry: log_scale = log(sqrt(eig Sigma)) and the
    rotation of the eigenvectors as a quaternion (w, x, y, z); a diagonal
    Sigma keeps the axis order and the identity rotation.
"""

import numpy as np

from .dwt import idwt3d, impulse_response_1d, subband_slices, subbands
from .filters import filter_bank


def canonical_kernel(j, o, bank, S=16, max_3d=64):
    """(kernel array [z, y, x], k_c) for subband (j, o): the response of an impulse at k_c.

    Grids of side <= max_3d run the full 3D IDWT; larger ones the outer product.
    """
    L = (1 << j) * S
    kc = S // 2
    if L <= max_3d:
        levels = j
        pyr = np.zeros((L, L, L), dtype=np.float64)
        sl = subband_slices((L, L, L), j, o)
        pyr[sl[0].start + kc, sl[1].start + kc, sl[2].start + kc] = 1.0
        return idwt3d(pyr, levels, bank), kc
    rx = impulse_response_1d(L, j, o[0], kc, bank)
    ry = impulse_response_1d(L, j, o[1], kc, bank)
    rz = impulse_response_1d(L, j, o[2], kc, bank)
    return rz[:, None, None] * ry[None, :, None] * rx[None, None, :], kc


def dominant_lobe(psi, tau):
    """ROI mask, centroid u (x, y, z) and covariance (3x3) of Eq. 13-14."""
    mag = np.abs(psi)
    W = mag / mag.sum()
    roi = W > tau * W.max()
    z, y, x = np.nonzero(roi)
    wts = W[roi]
    pts = np.stack([x, y, z], axis=1).astype(np.float64)
    u = (wts[:, None] * pts).sum(axis=0) / wts.sum()
    d = pts - u
    cov = (wts[:, None, None] * d[:, :, None] * d[:, None, :]).sum(axis=0) / wts.sum()
    return roi, u, cov, pts


def ridge_weight(psi, roi, pts, u, cov, ridge_rel):
    """w = sum |Y| G / (sum G^2 + lambda) over the ROI (Eq. 17)."""
    Y = np.abs(psi[roi])
    d = pts - u
    prec = np.linalg.inv(cov)
    G = np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, prec, d))
    lam = ridge_rel * float((G * G).sum())
    return float((Y * G).sum() / ((G * G).sum() + lam))


def _quat_from_matrix(R):
    """Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's method)."""
    tr = np.trace(R)
    if tr > 0:
        s = np.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    return q / np.linalg.norm(q)


def splat_shape(cov):
    """(log_scale[3], quat[4]) with R diag(exp(2 log_scale)) R^T = cov."""
    off = max(abs(cov[0, 1]), abs(cov[0, 2]), abs(cov[1, 2]))
    scale = np.sqrt(np.max(np.diag(cov)))
    if off <= 1e-9 * scale * scale:
        return 0.5 * np.log(np.diag(cov)), np.array([1.0, 0.0, 0.0, 0.0])
    evals, evecs = np.linalg.eigh(cov)
    if np.linalg.det(evecs) < 0:
        evecs[:, 0] = -evecs[:, 0]
    return 0.5 * np.log(evals), _quat_from_matrix(evecs)


def build_bank(levels, wavelet="bior4.4", tau=0.1, ridge_rel=1e-6):
    """List of 7J+1 bank entries (dicts) in oracle.dwt.subbands order (Eq. 18)."""
    bank = filter_bank(wavelet)
    S = 16 if bank["name"] == "bior4.4" else 4
    entries = []
    for j, o in subbands(levels):
        psi, kc = canonical_kernel(j, o, bank, S)
        roi, u_abs, cov, pts = dominant_lobe(psi, tau)
        w = ridge_weight(psi, roi, pts, u_abs, cov, ridge_rel)
        u = u_abs - (1 << j) * kc
        log_scale, quat = splat_shape(cov)
        entries.append(dict(j=j, o=o, u=u, cov=cov, w=w, log_scale=log_scale, quat=quat,
                            roi_size=int(roi.sum())))
    return entries


def ablate(entries, isotropic=False, unit_weight=False):
    """Bank of the ablation variants of Sec. 5.4 (entries are not modified).

    isotropic (w/o transition bank): every covariance becomes sigma_iso^2 I, with
    sigma_iso the average spatial extent of the full bank, read as the mean over
    its 7J+1 subbands of det(Sigma_{j,o})^(1/6) (the geometric-mean standard
    deviation of each subband's Gaussian); centres and weights are kept.
    unit_weight (w/o energy projection): w_{j,o} = 1.
    """
    out = [dict(e) for e in entries]
    if isotropic:
        sigma = float(np.mean([np.linalg.det(e["cov"]) ** (1.0 / 6.0) for e in entries]))
        for e in out:
            e["cov"] = sigma * sigma * np.eye(3)
            e["log_scale"] = np.full(3, np.log(sigma))
            e["quat"] = np.array([1.0, 0.0, 0.0, 0.0])
    if unit_weight:
        for e in out:
            e["w"] = 1.0
    return out

