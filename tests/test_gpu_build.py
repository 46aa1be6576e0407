"""GPU parity of the volume -> Gaussians build (Sec. 4.2-4.3, Supp. Sec. 1) and of the DVR
target renderer (Sec. 4.4) against the FP64 oracle."""

import numpy as np
import pytest
import torch

from _helpers import oracle_bank, read_device
from oracle import dvr as odvr
from oracle.dwt import dwt3d, subband_slices, subbands
from oracle.filters import filter_bank
from oracle.mapping import map_coefficients, select_all
from oracle.tf import apply_tf_vectorised
from vbm_inputs import TF_KNOTS_RGBA, TF_KNOTS_X, blob_volume, orbit_cameras
from vbm_inputs.cameras import camera_array, cameras_as_float32

pytestmark = pytest.mark.gpu


def _tf(vbm):
    return vbm.make_tf(TF_KNOTS_X, TF_KNOTS_RGBA)


def _tf32():
    return TF_KNOTS_X.astype(np.float32).astype(np.float64), TF_KNOTS_RGBA.astype(np.float32).astype(np.float64)


def test_tf_apply(cuda_lib):
    F = np.random.default_rng(0).uniform(-0.2, 1.2, 10007).astype(np.float32)
    out = torch.zeros(4 * F.size, device="cuda")
    cuda_lib.tf_apply(torch.from_numpy(F).cuda(), _tf(cuda_lib), out)
    x, rgba = _tf32()
    ref = apply_tf_vectorised(F.astype(np.float64), x, rgba)
    assert np.abs(out.cpu().numpy().reshape(4, -1).T - ref).max() < 1e-6


@pytest.mark.parametrize("wavelet,levels,dims", [(0, 2, (32, 32, 32)), (0, 3, (48, 32, 64)), (1, 2, (16, 24, 8))])
def test_dwt3d(cuda_lib, wavelet, levels, dims):
    nx, ny, nz = dims
    x = np.random.default_rng(1).standard_normal((2, nz, ny, nx)).astype(np.float32)
    d = torch.from_numpy(x.copy()).cuda()
    tmp = torch.zeros(2 * x[0].size, device="cuda")
    cuda_lib.dwt3d(d, 2, dims, levels, wavelet, tmp)
    bank = filter_bank(wavelet)
    for c in range(2):
        ref = dwt3d(x[c].astype(np.float64), levels, bank)
        assert np.abs(d.cpu().numpy()[c] - ref).max() < 2e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("levels,wavelet", [(3, 0), (5, 0), (2, 1)])
def test_bank_matches_oracle(cuda_lib, levels, wavelet):
    """Host FP64 bank of the library against the oracle's, every entry (five levels:
    the 512^3 workload's bank)."""
    lib_bank = cuda_lib.bank_to_dicts(cuda_lib.bank_build(levels, wavelet))
    ref = oracle_bank(levels, wavelet)
    assert len(lib_bank) == len(ref) == 7 * levels + 1
    for e, r in zip(lib_bank, ref):
        assert (e["j"], tuple(e["o"])) == (r["j"], tuple(r["o"]))
        assert np.allclose(e["u"], r["u"], atol=1e-9)
        assert np.allclose(e["cov"], r["cov"], atol=1e-9 * np.abs(r["cov"]).max())
        assert abs(e["w"] - r["w"]) < 1e-9 * r["w"]
        assert np.allclose(e["log_scale"], r["log_scale"], atol=1e-6)
        assert np.allclose(e["quat"], r["quat"], atol=1e-6)


def _build(vbm, F, J, K_tot, wavelet=0, energy_comp=True, ablation=0, knots=None):
    dims = F.shape[::-1]
    bank = vbm.bank_build(J, wavelet)
    if ablation:
        vbm.bank_ablate(bank, ablation)
    sel = vbm.make_select(K_tot, energy_comp=energy_comp)
    n = F.size
    coef = torch.zeros(4 * n, device="cuda")
    keep = torch.zeros(n, dtype=torch.uint8, device="cuda")
    tf = _tf(vbm) if knots is None else vbm.make_tf(*knots)
    params, count = vbm.build(torch.from_numpy(F).cuda(), dims, tf, bank, sel, capacity=n, coef=coef, keep=keep)
    torch.cuda.synchronize()
    return (params.cpu().numpy()[:, :count], count, coef.cpu().numpy().reshape(4, *F.shape),
            keep.cpu().numpy().reshape(F.shape).astype(bool), bank)


@pytest.mark.parametrize("G,J,K_tot,seed,ablation,mode,wavelet", [
    (32, 2, 4096, 0, 0, None, 0), (64, 3, 20000, 1, 0, None, 0),
    (32, 2, 4096, 0, 1, None, 0), (32, 2, 4096, 0, 2, None, 0),
    (32, 2, 4096, 0, 0, 1, 0), (64, 3, 20000, 1, 0, 3, 0),
    (32, 2, 4096, 0, 0, None, 1), (64, 3, 20000, 1, 0, None, 1), (64, 3, 20000, 1, 3, None, 1)])
def test_build_matches_oracle(cuda_lib, G, J, K_tot, seed, ablation, mode, wavelet):
    """vbm_build against the oracle: pyramid, kept indices (bit-exact), Gaussians mapped
    with the oracle's own bank; also with the ablated banks of Sec. 5.4 (isotropic
    covariance, unit weight), with the Haar basis of the same ablation study, and with two
    of the TF modes of Sec. 4.4 (non-zero over one value interval only)."""
    from vbm_inputs import tf_mode
    F = blob_volume(G, 4 if G == 32 else 12, seed=seed)
    knots = None if mode is None else tf_mode(mode)
    P, count, A_gpu, keep_gpu, bank = _build(cuda_lib, F, J, K_tot, wavelet=wavelet, ablation=ablation, knots=knots)
    # 1. coefficient pyramid vs the FP64 oracle pipeline (TF + DWT)
    if knots is None:
        x, rgba = _tf32()
    else:     # the library holds the knots in float32
        x, rgba = (k.astype(np.float32).astype(np.float64) for k in knots)
    RF = apply_tf_vectorised(F.astype(np.float64), x, rgba)
    fb = filter_bank(wavelet)
    A_ref = np.stack([dwt3d(RF[..., c], J, fb) for c in range(4)])
    assert np.abs(A_gpu - A_ref).max() < 2e-6 * np.abs(A_ref).max()
    # 2. selection: same decisions in the same precision (float32) on the GPU's pyramid
    masks, Ks, E, N = select_all(A_gpu, J, K_tot, dtype=np.float32)
    for (j, o), m in zip(subbands(J), masks):
        assert np.array_equal(keep_gpu[subband_slices(F.shape, j, o)], m), (j, o)
    assert count == sum(int(m.sum()) for m in masks)
    if mode is None:
        assert 0.5 * K_tot < count < 1.5 * K_tot
    else:
        assert count > 100
    # 3. mapping on the GPU's pyramid and masks with the oracle's own bank
    ref = map_coefficients(A_gpu.astype(np.float64), masks, J, oracle_bank(J, wavelet, ablation))
    assert ref.shape == P.shape
    assert np.allclose(P[0:3], ref[0:3], atol=1e-5 * G)
    assert np.allclose(P[3:10], ref[3:10], atol=1e-6)
    assert np.allclose(P[10], ref[10], atol=2e-5 * np.abs(ref[10]).max())
    assert np.allclose(P[11:14], ref[11:14], rtol=1e-5, atol=1e-9)


def test_build_capacity_error(cuda_lib):
    vbm = cuda_lib
    F = blob_volume(16, 2, seed=3)
    bank = vbm.bank_build(2, 0)
    with pytest.raises(vbm.VbmError) as e:
        vbm.build(torch.from_numpy(F).cuda(), F.shape[::-1], _tf(vbm), bank, vbm.make_select(500), capacity=3)
    assert e.value.status == vbm.VBM_ERR_CAPACITY


@pytest.mark.parametrize("G,W,H,V", [(32, 64, 48, 2), (24, 37, 29, 1)])
def test_dvr_matches_oracle(cuda_lib, G, W, H, V):
    F = blob_volume(G, 3, seed=G)
    cams = orbit_cameras((G, G, G), V, W, H)
    cams_dev = cuda_lib.cameras_to_device(camera_array(cams))
    out = torch.zeros((V, 4, H, W), device="cuda")
    cuda_lib.render_dvr(torch.from_numpy(F).cuda(), F.shape[::-1], _tf(cuda_lib), cams_dev, V, W, H, 0.5, out)
    torch.cuda.synchronize()
    x, rgba = _tf32()
    c32 = cameras_as_float32(cams)
    for v in range(V):
        ref = odvr.render_dvr(F.astype(np.float64), x, rgba, c32[v], step=0.5)
        assert np.abs(out.cpu().numpy()[v] - ref).max() <= 1e-4
    assert out.max().item() > 0.01
