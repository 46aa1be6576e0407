"""Coefficient -> Gaussian construction, the whole volume-to-Gaussians build (oracle).

Test infrastructure only.  Sec. 4.3:
  * multichannel DWT of RF = TF(F) (Eq. 20-21);
  * per kept coefficient: p = |A_{j,o,k,(R,G,B,alpha)}| (.) w_{j,o} (Eq. 22),
    amplitude s_{j,o} p with s = 2^{-3j/2} (Eq. 23), centre
    u_{j,o,k} = T_{2^j k + delta} u_{j,o} (Eq. 24), covariance Sigma_{j,o};
  * the union over subbands (Eq. 31-32).
Readings (the paper leaves the 3DGS parameterisation implicit, Eq. 32):
  * delta = (1/2, 1/2, 1/2) is the voxel-centre offset: centre (world) =
    u_{j,o} + 2^j k + 1/2.
  * amplitude -> opacity: logit(clamp(s p_alpha, 2/255, 0.99)) so that the
    sigmoid-activated 3DGS opacity reproduces it; colour = s p_rgb (raw, no
    activation, view independent).  The floor 2/255 keeps every retained
    coefficient visible: the fine-tuning renderer never composites a splat
    whose opacity is below 1/255 (such a Gaussian would get no gradient and
    stay invisible), while the adaptive filter kept the coefficient as
    significant (Sec. 4.3).
  * log_scale and rotation come from the bank entry of the subband.
  * s is applied by default (energy_comp); it can be switched off.
Gaussians are emitted subband by subband (oracle.dwt.subbands order) and,
within a subband, in raster order of k (x fastest, then y, then z).
"""

import numpy as np

from .bank import build_bank
from .dwt import dwt3d, subband_slices, subbands
from .filters import filter_bank
from .select import allocate_budget, select_subband
from .tf import apply_tf_vectorised


def radiance_pyramid(F, levels, knots_x, knots_rgba, wavelet="bior4.4"):
    """A[c] = DWT(TF(F)[..., c]) for c = R, G, B, alpha: shape (4, nz, ny, nx)."""
    RF = apply_tf_vectorised(F, knots_x, knots_rgba)
    bank = filter_bank(wavelet)
    return np.stack([dwt3d(RF[..., c], levels, bank) for c in range(4)])


def select_all(A, levels, K_tot, alpha_E=0.5, beta_N=0.5, lam=3.0, min_per_band=10,
               dtype=np.float64):
    """Budget allocation and per-subband keep masks (Supp. Sec. 1).

    Returns (masks, Ks, E, N) lists in subband order.
    """
    shape = A.shape[1:]
    bands = subbands(levels)
    E, N = [], []
    for j, o in bands:
        sub = np.asarray(A[3][subband_slices(shape, j, o)], dtype=np.float64)
        E.append(float((sub * sub).sum()))
        N.append(sub.size)
    Ks = allocate_budget(E, N, K_tot, alpha_E, beta_N, min_per_band)
    masks = []
    for (j, o), K in zip(bands, Ks):
        sl = subband_slices(shape, j, o)
        mask, _ = select_subband(A[(slice(None),) + sl], K, lam, dtype)
        masks.append(mask)
    return masks, Ks, E, N


def map_coefficients(A, masks, levels, bank_entries, energy_comp=True):
    """Gaussian parameters P[14][N] (float64) for the kept coefficients (Eq. 22-24)."""
    shape = A.shape[1:]
    cols = []
    for (j, o), mask, entry in zip(subbands(levels), masks, bank_entries):
        assert entry["j"] == j and tuple(entry["o"]) == tuple(o)
        sl = subband_slices(shape, j, o)
        kz, ky, kx = np.nonzero(mask)
        if kx.size == 0:
            continue
        coefs = np.asarray(A[(slice(None),) + sl], dtype=np.float64)[:, kz, ky, kx]
        s = 2.0 ** (-1.5 * j) if energy_comp else 1.0
        amp = s * np.abs(coefs) * entry["w"]                       # (4, n)
        P = np.zeros((14, kx.size))
        step = float(1 << j)
        P[0] = entry["u"][0] + step * kx + 0.5
        P[1] = entry["u"][1] + step * ky + 0.5
        P[2] = entry["u"][2] + step * kz + 0.5
        P[3:6] = np.asarray(entry["log_scale"])[:, None]
        P[6:10] = np.asarray(entry["quat"])[:, None]
        op = np.clip(amp[3], 2.0 / 255.0, 0.99)
        P[10] = np.log(op / (1.0 - op))
        P[11:14] = amp[0:3]
        cols.append(P)
    if not cols:
        return np.zeros((14, 0))
    return np.concatenate(cols, axis=1)


def vbm_build(F, levels, knots_x, knots_rgba, K_tot, wavelet="bior4.4", tau=0.1,
              ridge_rel=1e-6, alpha_E=0.5, beta_N=0.5, lam=3.0, energy_comp=True,
              bank_entries=None):
    """Volume -> Gaussian parameters, the map F -> RF -> Phi -> G of Sec. 4.1."""
    A = radiance_pyramid(F, levels, knots_x, knots_rgba, wavelet)
    if bank_entries is None:
        bank_entries = build_bank(levels, wavelet, tau, ridge_rel)
    masks, Ks, E, N = select_all(A, levels, K_tot, alpha_E, beta_N, lam)
    P = map_coefficients(A, masks, levels, bank_entries, energy_comp)
    return P, dict(A=A, masks=masks, Ks=Ks, E=E, N=N, bank=bank_entries)
