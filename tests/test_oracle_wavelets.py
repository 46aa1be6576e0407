"""Pins for the oracle's filter bank and periodised DWT (Sec. 3, Sec. 4.2, Supp. Sec. 2)."""

import os

import numpy as np
import pytest

from oracle.dwt import (analysis_1d, dwt3d, idwt3d, impulse_response, impulse_response_1d,
                        subband_slices, subbands, synthesis_1d)
from oracle.filters import bior44, filter_bank, haar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cdf97_filters.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, tap, v = line.split()
        vals.setdefault(name, {})[int(tap)] = float(v)
    return vals


def test_bior44_matches_published_cdf97():
    g = _golden()
    b = bior44()
    for n, v in g["lowpass9"].items():
        assert abs(b["ht"][n] - v) < 1e-9 and abs(b["ht"][-n] - v) < 1e-9
    for n, v in g["lowpass7"].items():
        assert abs(b["h"][n] - v) < 1e-9 and abs(b["h"][-n] - v) < 1e-9


@pytest.mark.parametrize("name", ["bior4.4", "haar"])
def test_filter_identities(name):
    b = filter_bank(name)
    s2 = np.sqrt(2.0)
    assert abs(sum(b["ht"].values()) - s2) < 1e-13
    assert abs(sum(b["h"].values()) - s2) < 1e-13
    # biorthogonality of the low-pass pair: sum_n h[n] ht[n + 2l] = delta_l
    for l in range(-5, 6):
        acc = sum(hv * b["ht"].get(n + 2 * l, 0.0) for n, hv in b["h"].items())
        assert abs(acc - (1.0 if l == 0 else 0.0)) < 1e-13, l
    # high-pass filters annihilate constants
    assert abs(sum(b["gt"].values())) < 1e-13 and abs(sum(b["g"].values())) < 1e-13


def test_bior44_four_vanishing_moments_and_symmetry():
    b = bior44()
    for key in ("gt", "g"):
        for p in range(4):
            assert abs(sum(v * float(n) ** p for n, v in b[key].items())) < 1e-12, (key, p)
        # the fifth moment does not vanish (exactly four)
        assert abs(sum(v * float(n) ** 4 for n, v in b[key].items())) > 1e-3
    for key in ("ht", "h", "gt", "g"):
        for n, v in b[key].items():
            assert abs(b[key][-n] - v) < 1e-15
    assert len(b["ht"]) == 9 and len(b["h"]) == 7


def _fft_analysis(x, filt, parity):
    """Brute force: circular correlation via FFT, then keep samples 2k + parity."""
    L = x.size
    f = np.zeros(L)
    for n, v in filt.items():
        f[(-n) % L] += v       # correlation kernel: c[m] = sum_n f[n] x[m + n]
    c = np.real(np.fft.ifft(np.fft.fft(x) * np.fft.fft(f)))
    return c[parity::2]


@pytest.mark.parametrize("name", ["bior4.4", "haar"])
def test_1d_analysis_matches_fft_correlation(name):
    b = filter_bank(name)
    rng = np.random.default_rng(3)
    for L in (16, 24):
        x = rng.standard_normal(L)
        out = analysis_1d(x, 0, b)
        assert np.allclose(out[:L // 2], _fft_analysis(x, b["ht"], 0), atol=1e-13)
        assert np.allclose(out[L // 2:], _fft_analysis(x, b["gt"], 1), atol=1e-13)


@pytest.mark.parametrize("name,levels,shape", [("bior4.4", 3, (16, 32, 24)), ("haar", 2, (8, 8, 12)),
                                               ("bior4.4", 2, (32, 32, 32))])
def test_perfect_reconstruction(name, levels, shape):
    b = filter_bank(name)
    x = np.random.default_rng(1).standard_normal(shape)
    assert np.abs(idwt3d(dwt3d(x, levels, b), levels, b) - x).max() < 1e-12


def test_haar_closed_form_and_energy():
    b = haar()
    x = np.random.default_rng(2).standard_normal((8, 8, 8))
    p = dwt3d(x, 1, b)
    blocks = x.reshape(4, 2, 4, 2, 4, 2).sum(axis=(1, 3, 5)) / 2 ** 1.5
    assert np.allclose(p[:4, :4, :4], blocks, atol=1e-14)
    # x-detail (o = H, L, L): (x_even - x_odd) summed over y, z pairs
    dx = (x[:, :, 0::2] - x[:, :, 1::2]).reshape(4, 2, 4, 2, 4).sum(axis=(1, 3)) / 2 ** 1.5
    assert np.allclose(p[subband_slices(x.shape, 1, (1, 0, 0))], dx, atol=1e-14)
    p3 = dwt3d(x, 3, b)
    assert abs((p3 ** 2).sum() - (x ** 2).sum()) < 1e-11   # orthogonal transform


def test_constant_field_has_no_detail():
    b = bior44()
    x = np.full((16, 16, 16), 0.37)
    p = dwt3d(x, 2, b)
    for j, o in subbands(2):
        sub = p[subband_slices(x.shape, j, o)]
        if o == (0, 0, 0):
            assert np.allclose(sub, 0.37 * 2 ** (3 * j / 2), atol=1e-12)
        else:
            assert np.abs(sub).max() < 1e-13


@pytest.mark.parametrize("j,o,k", [(1, (1, 0, 0), (2, 3, 1)), (1, (1, 1, 1), (5, 0, 7)),
                                   (2, (0, 1, 1), (1, 2, 3)), (2, (0, 0, 0), (3, 0, 2))])
def test_translation_theorem(j, o, k):
    """Supp. Sec. 2: H delta_k = T_{2^j k} H delta_0 exactly on the periodic grid."""
    b = bior44()
    shape = (32, 32, 32)
    r0 = impulse_response(shape, 2, j, o, (0, 0, 0), b)
    rk = impulse_response(shape, 2, j, o, k, b)
    step = 1 << j
    shifted = np.roll(r0, (step * k[2], step * k[1], step * k[0]), axis=(0, 1, 2))
    assert np.abs(rk - shifted).max() < 1e-14


@pytest.mark.parametrize("j,o", [(1, (1, 0, 1)), (2, (0, 1, 0)), (2, (0, 0, 0))])
def test_separability(j, o):
    """Supp. Sec. 2, Step 1: the 3D canonical kernel is an outer product of 1D responses."""
    b = bior44()
    L = 32
    r3 = impulse_response((L, L, L), j, j, o, (3, 2, 1), b)
    rx = impulse_response_1d(L, j, o[0], 3, b)
    ry = impulse_response_1d(L, j, o[1], 2, b)
    rz = impulse_response_1d(L, j, o[2], 1, b)
    assert np.abs(r3 - rz[:, None, None] * ry[None, :, None] * rx[None, None, :]).max() < 1e-14


def test_synthesis_is_adjoint_free_inverse_1d():
    b = bior44()
    c = np.random.default_rng(5).standard_normal(20)
    assert np.abs(analysis_1d(synthesis_1d(c, 0, b), 0, b) - c).max() < 1e-13


def test_subband_count():
    for J in (1, 2, 3, 5):
        assert len(subbands(J)) == 7 * J + 1
