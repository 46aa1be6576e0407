"""Pins for the oracle's transition bank (Sec. 4.2), adaptive filtering (Supp. Sec. 1)
and coefficient-to-Gaussian mapping (Sec. 4.3)."""

import statistics

import numpy as np
import pytest

from oracle import bank as obank
from oracle.dwt import dwt3d, idwt3d, subband_slices, subbands
from oracle.filters import bior44, haar
from oracle.mapping import map_coefficients, select_all
from oracle.select import allocate_budget, joint_magnitude, median, select_subband


# ------------------------------------------------------------------ bank

@pytest.mark.parametrize("j", [1, 2, 3])
def test_haar_bank_closed_form(j):
    """Haar atoms are boxes of side 2^j with magnitude 2^{-3j/2}: centroid (2^j - 1)/2,
    covariance (4^j - 1)/12 I, and w from separable 1D sums."""
    entries = obank.build_bank(j, "haar")
    n = 1 << j
    var = (4.0 ** j - 1.0) / 12.0
    c = (n - 1) / 2.0
    g1 = np.exp(-0.5 * (np.arange(n) - c) ** 2 / var)
    sumG, sumG2 = g1.sum() ** 3, (g1 ** 2).sum() ** 3
    w_expect = 2.0 ** (-1.5 * j) * sumG / (sumG2 * (1 + 1e-6))
    for e in entries:
        if e["j"] != j:
            continue
        assert np.allclose(e["u"], c, atol=1e-12)
        assert np.allclose(e["cov"], var * np.eye(3), atol=1e-12)
        assert e["roi_size"] == n ** 3
        assert abs(e["w"] - w_expect) < 1e-12 * w_expect
        assert np.allclose(e["quat"], [1, 0, 0, 0]) and np.allclose(np.exp(2 * e["log_scale"]), var)


def test_ablated_banks_haar_closed_form():
    """Ablation variants (Sec. 5.4) of the Haar bank, whose subband covariances are
    (4^j - 1)/12 I: isotropic gives every subband sigma_iso^2 I with sigma_iso the mean
    over the 7J + 1 subbands of sqrt((4^j - 1)/12), keeping centres and weights; unit
    weight sets every w to 1 and changes nothing else."""
    J = 2
    entries = obank.build_bank(J, "haar")
    sig = [np.sqrt((4.0 ** e["j"] - 1.0) / 12.0) for e in entries]
    sigma_iso = float(np.mean(sig))
    assert len(entries) == 7 * J + 1
    assert sigma_iso == pytest.approx((7 * 0.5 + 8 * np.sqrt(15.0 / 12.0)) / 15.0, abs=1e-12)
    iso = obank.ablate(entries, isotropic=True)
    for e, a in zip(entries, iso):
        assert np.allclose(a["cov"], sigma_iso ** 2 * np.eye(3), atol=1e-12)
        assert np.allclose(a["log_scale"], np.log(sigma_iso), atol=1e-12)
        assert np.array_equal(a["quat"], [1.0, 0.0, 0.0, 0.0])
        assert np.array_equal(a["u"], e["u"]) and a["w"] == e["w"]
    unit = obank.ablate(entries, unit_weight=True)
    for e, a in zip(entries, unit):
        assert a["w"] == 1.0 and np.array_equal(a["cov"], e["cov"]) and np.array_equal(a["u"], e["u"])
    assert entries[0]["w"] != 1.0          # the input is not modified


def test_bior44_bank_symmetry():
    """Symmetric 9/7 filters: low-pass atoms centred on 2^j k, high-pass atoms on
    2^j k + 2^{j-1} per axis; symmetric magnitude makes every covariance diagonal."""
    for e in obank.build_bank(2, "bior4.4"):
        j, o = e["j"], e["o"]
        expect = np.array([o[d] * 2.0 ** (j - 1) for d in range(3)])
        assert np.allclose(e["u"], expect, atol=1e-10)
        off = e["cov"] - np.diag(np.diag(e["cov"]))
        assert np.abs(off).max() < 1e-12 * np.abs(np.diag(e["cov"])).max()
        assert e["w"] > 0


@pytest.mark.parametrize("o", [(0, 0, 0), (1, 0, 1), (1, 1, 1)])
def test_kernel_paths_agree(o):
    b = bior44()
    a, kc = obank.canonical_kernel(2, o, b, 16, max_3d=64)
    c, kc2 = obank.canonical_kernel(2, o, b, 16, max_3d=0)
    assert kc == kc2 and np.abs(a - c).max() < 1e-14


def test_dominant_lobe_hand_example():
    psi = np.zeros((5, 5, 5))
    psi[2, 2, 1], psi[2, 2, 2], psi[2, 2, 3] = 1.0, -2.0, 0.5
    psi[0, 0, 0] = 0.1          # below tau * max = 0.2: outside the ROI
    roi, u, cov, pts = obank.dominant_lobe(psi, 0.1)
    assert roi.sum() == 3
    # weights 1, 2, 0.5 at x = 1, 2, 3: centroid 6.5 / 3.5 = 13/7, variance 20/49
    assert np.allclose(u, [13.0 / 7.0, 2.0, 2.0], atol=1e-14)
    expect = np.zeros((3, 3))
    expect[0, 0] = 20.0 / 49.0
    assert np.allclose(cov, expect, atol=1e-14)


def test_dominant_lobe_strict_threshold():
    psi = np.zeros((3, 3, 3))
    psi[1, 1, 1] = 2.0
    psi[0, 1, 1] = 0.5          # |psi| = tau * max exactly (tau = 0.25) -> excluded
    psi[2, 1, 1] = 0.75         # above -> included
    roi, u, cov, pts = obank.dominant_lobe(psi, 0.25)
    assert roi.sum() == 2 and not roi[0, 1, 1] and roi[2, 1, 1]


def test_ridge_weight_is_the_minimiser():
    b = bior44()
    psi, kc = obank.canonical_kernel(1, (1, 1, 0), b)
    roi, u, cov, pts = obank.dominant_lobe(psi, 0.1)
    w = obank.ridge_weight(psi, roi, pts, u, cov, 1e-6)
    Y = np.abs(psi[roi])
    d = pts - u
    G = np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, np.linalg.inv(cov), d))
    lam = 1e-6 * (G * G).sum()

    def obj(x):
        return ((Y - x * G) ** 2).sum() + lam * x * x
    for eps in (1e-3, 1e-6):
        assert obj(w) <= obj(w + eps) and obj(w) <= obj(w - eps)


def test_splat_shape_general_covariance():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((3, 3))
    cov = M @ M.T + 0.5 * np.eye(3)
    ls, q = obank.splat_shape(cov)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    assert np.allclose(R @ np.diag(np.exp(2 * ls)) @ R.T, cov, atol=1e-12)


# ------------------------------------------------------------------ select

def test_allocate_budget_hand_example():
    # S = sqrt(E N) = [20, 10, 0, 15], sum 45: floor(1000 S / 45) = [444, 222, 0, 333], min 10
    assert allocate_budget([4, 1, 0, 9], [100, 100, 100, 25], 1000) == [444, 222, 10, 333]


@pytest.mark.parametrize("n", [1, 2, 7, 10, 101])
def test_median_matches_library(n):
    x = np.random.default_rng(n).standard_normal(n)
    assert median(x) == pytest.approx(statistics.median(x.tolist()), abs=0)


def test_select_hand_example():
    vals = np.array([0, 0, 0.1, 0.2, 0.3, 5, 6, 7, 0.15, 0.25, 0.05])
    A = np.zeros((4, vals.size))
    A[0] = vals
    # median 0.2, MAD 0.15, T = 3 * 0.15 / 0.6745 = 0.667...; candidates {5, 6, 7}
    m2, info = select_subband(A, 2)
    assert info["n_candidates"] == 3 and info["K_eff"] == 2
    assert set(vals[m2]) == {6.0, 7.0}
    m10, _ = select_subband(A, 10)
    assert set(vals[m10]) == {5.0, 6.0, 7.0}
    assert info["T"] == pytest.approx(3 * 0.15 / 0.6745, rel=1e-12)


def test_select_ties_and_zeros():
    vals = np.array([0.0] * 9 + [1.0, 2.0, 2.0, 3.0])
    A = np.zeros((4, vals.size))
    A[2] = vals
    m, info = select_subband(A, 2)          # T = 0, v_(2) = 2: ties keep three
    assert info["T"] == 0 and sorted(vals[m]) == [2.0, 2.0, 3.0]
    m, _ = select_subband(A, 100)           # zeros are never kept
    assert sorted(vals[m]) == [1.0, 2.0, 2.0, 3.0]
    m, _ = select_subband(np.zeros((4, 6)), 3)
    assert not m.any()


def _brute_select(A, K, lam=3.0):
    """Rank formulation: keep k iff v_k >= T, v_k > 0 and fewer than K' candidates beat it."""
    v = np.sqrt((np.asarray(A, dtype=np.float64) ** 2).sum(axis=0)).reshape(-1)
    med = statistics.median(v.tolist())
    T = lam * statistics.median(np.abs(v - med).tolist()) / 0.6745
    cand = [i for i in range(v.size) if v[i] >= T]
    Kp = min(K, len(cand))
    keep = np.zeros(v.size, dtype=bool)
    for i in cand:
        greater = sum(1 for m in cand if v[m] > v[i])
        keep[i] = greater < Kp and v[i] > 0
    return keep.reshape(A.shape[1:])


@pytest.mark.parametrize("seed,K", [(0, 5), (1, 40), (2, 1000)])
def test_select_matches_brute_force(seed, K):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((4, 6, 5, 4)) * rng.exponential(1.0, size=(1, 6, 5, 4)) ** 3
    mask, _ = select_subband(A, K)
    assert np.array_equal(mask, _brute_select(A, K))


def test_select_float32_mode_is_float32():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((4, 300)).astype(np.float32)
    v = joint_magnitude(A, np.float32)
    assert v.dtype == np.float32
    manual = np.sqrt(((A[0] * A[0] + A[1] * A[1]) + A[2] * A[2]) + A[3] * A[3])
    assert np.array_equal(v, manual)
    m32, info = select_subband(A, 20, dtype=np.float32)
    assert isinstance(info["T"], np.float32)
    assert m32.sum() >= min(20, info["n_candidates"])


# ------------------------------------------------------------------ mapping

def test_single_atom_maps_to_its_lobe():
    """A volume that is one wavelet atom (IDWT of one impulse at k, subband (j, o)) maps to a
    Gaussian centred on the atom's own dominant-lobe centroid + 1/2 (translation rule,
    Eq. 19 and 24) with amplitude |A| w (s switched off)."""
    b = bior44()
    G, J = 32, 2
    entries = obank.build_bank(J, "bior4.4")
    for (j, o), k in [((1, (1, 0, 1)), (5, 9, 3)), ((2, (0, 1, 1)), (2, 6, 5)), ((2, (0, 0, 0)), (4, 3, 2))]:
        coef = np.zeros((G, G, G))
        sl = subband_slices(coef.shape, j, o)
        amp = np.array([0.3, -0.2, 0.1, 0.8])
        coef[sl[0].start + k[2], sl[1].start + k[1], sl[2].start + k[0]] = 1.0
        atom = idwt3d(coef, J, b)
        A = np.stack([dwt3d(atom * a, J, b) for a in amp])
        masks, Ks, E, N = select_all(A, J, K_tot=50)
        P = map_coefficients(A, masks, J, entries, energy_comp=False)
        best = np.argmax(P[11])          # largest red amplitude: the atom's own coefficient
        roi, u, cov, pts = obank.dominant_lobe(atom, 0.1)
        assert np.allclose(P[0:3, best], u + 0.5, atol=1e-9)
        assert np.allclose(np.exp(2 * P[3:6, best]), np.diag(cov), rtol=1e-9)
        e = [x for x in entries if x["j"] == j and tuple(x["o"]) == o][0]
        assert np.allclose(P[11:14, best], np.abs(amp[:3]) * e["w"], rtol=1e-12)
        op = 1 / (1 + np.exp(-P[10, best]))
        assert op == pytest.approx(min(0.99, max(2 / 255, abs(amp[3]) * e["w"])), rel=1e-12)


def test_mapping_structure_and_energy_compensation():
    rng = np.random.default_rng(7)
    J = 2
    A = rng.standard_normal((4, 16, 16, 16)) * 0.05
    entries = obank.build_bank(J, "bior4.4")
    masks, Ks, E, N = select_all(A, J, K_tot=300)
    P1 = map_coefficients(A, masks, J, entries, energy_comp=True)
    P0 = map_coefficients(A, masks, J, entries, energy_comp=False)
    col = 0
    for (j, o), mask, e in zip(subbands(J), masks, entries):
        n = int(mask.sum())
        blk = slice(col, col + n)
        assert np.allclose(P1[11:14, blk], 2.0 ** (-1.5 * j) * P0[11:14, blk], rtol=1e-13)
        assert np.allclose(P1[3:6, blk], e["log_scale"][:, None])
        frac = (P1[0:3, blk] - e["u"][:, None] - 0.5) / (1 << j)
        assert np.allclose(frac, np.round(frac), atol=1e-12)
        col += n
    assert col == P1.shape[1]


def test_opacity_clamp_values():
    """logit(clamp(.)): a huge alpha amplitude gives logit(0.99) = ln 99, a tiny one logit(2/255)."""
    entries = obank.build_bank(1, "haar")
    bands = subbands(1)
    masks = [np.zeros((4, 4, 4), dtype=bool) for _ in bands]
    masks[bands.index((1, (1, 0, 0)))][0, 0, 0] = True      # x-detail octant, k = 0
    A = np.zeros((4, 8, 8, 8))
    A[3, 0, 0, 4] = 1e6
    P = map_coefficients(A, masks, 1, entries)
    assert P.shape[1] == 1 and P[10, 0] == pytest.approx(np.log(99.0), rel=1e-12)
    A[3, 0, 0, 4] = 1e-9
    P = map_coefficients(A, masks, 1, entries)
    assert P[10, 0] == pytest.approx(np.log(2.0 / 253.0), rel=1e-12)
