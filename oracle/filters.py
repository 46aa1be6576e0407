"""Wavelet filter banks for the oracle (test infrastructure only).

The paper uses the biorthogonal 4.4 wavelet through PyWavelets (Sec. 4.2,
"Translation Consistency"; Sec. 5.2) and Haar in its ablation (Sec. 5.4, item
3).  PyWavelets is not available, so bior4.4 is derived here from its
published construction: the Cohen-Daubechies-Feauveau spline variant with
four vanishing moments on both sides (the "9/7" pair).  With x = sin^2(w/2),
the product of the two low-pass responses is cos^8(w/2) P(x), where
P(x) = sum_{k<4} C(3+k, k) x^k = 1 + 4x + 10x^2 + 20x^3.  P has one real root
x_r and a complex pair; the 7-tap filter takes cos^4(w/2) (1 - x / x_r), the
9-tap filter takes cos^4(w/2) times the quadratic with the complex pair.  Both
are scaled to sum sqrt(2).

Filter convention (periodised, length L even), used by oracle.dwt:
  analysis   a[k] = sum_n ht[n] x[2k + n],      d[k] = sum_n gt[n] x[2k + 1 + n]
  synthesis  x[m] = sum_k h[m - 2k] a[k] + sum_k g[m - 2k - 1] d[k]
Each filter is a dict {n: coefficient}.  For the symmetric 9/7 pair,
ht = 9-tap (n = -4..4), h = 7-tap (n = -3..3), and the high-pass filters are
the modulated low-pass filters gt[n] = (-1)^n h[n], g[n] = (-1)^n ht[n], which
makes the bank perfectly reconstructing and alias free.
"""

import numpy as np


def _laurent_mul(a, b):
    """Product of two centred Laurent polynomials given as odd-length arrays."""
    return np.convolve(a, b)


def _cdf_97_lowpass():
    """(9-tap, 7-tap) symmetric low-pass filters, each summing to sqrt(2)."""
    # P(x) = 20x^3 + 10x^2 + 4x + 1 (highest power first for numpy.roots).
    P = np.array([20.0, 10.0, 4.0, 1.0])
    roots = np.roots(P)
    xr = float(np.real(roots[np.argmin(np.abs(np.imag(roots)))]))
    for _ in range(5):  # Newton polish of the real root in FP64
        xr -= np.polyval(P, xr) / np.polyval(np.polyder(P), xr)
    # Quadratic factor with the complex pair: P(x) / (20 (x - xr)) = x^2 + p x + q.
    quad, rem = np.polydiv(P, np.array([20.0, -20.0 * xr]))
    assert abs(rem[-1]) < 1e-12
    p, q = quad[1] / quad[0], quad[2] / quad[0]
    # Laurent polynomials in z = e^{-iw}, centred: index 0 of the middle entry.
    sin2 = np.array([-0.25, 0.5, -0.25])       # sin^2(w/2) = (2 - z - 1/z) / 4
    cos2 = np.array([0.25, 0.5, 0.25])         # cos^2(w/2) = (2 + z + 1/z) / 4
    one = np.array([0.0, 1.0, 0.0])
    cos4 = _laurent_mul(cos2, cos2)            # 5 taps
    f7 = _laurent_mul(cos4, one - sin2 / xr)   # cos^4 (1 - x / xr): 7 taps
    x2 = _laurent_mul(sin2, sin2)              # 5 taps
    quad_l = x2 + np.pad(p * sin2 + q * one, 1)
    f9 = _laurent_mul(cos4, quad_l / q)        # cos^4 (x^2 + p x + q) / q: 9 taps
    f9 = np.trim_zeros(f9)
    f7 = np.trim_zeros(f7)
    assert f9.size == 9 and f7.size == 7
    f9 = f9 * (np.sqrt(2.0) / f9.sum())
    f7 = f7 * (np.sqrt(2.0) / f7.sum())
    return f9, f7


def _centred_dict(arr):
    half = arr.size // 2
    return {n - half: float(v) for n, v in enumerate(arr)}


def bior44():
    """bior4.4 (CDF 9/7) bank: dict(ht, gt, h, g) in the convention above."""
    f9, f7 = _cdf_97_lowpass()
    ht = _centred_dict(f9)
    h = _centred_dict(f7)
    gt = {n: (-1.0) ** (n % 2) * v for n, v in h.items()}
    g = {n: (-1.0) ** (n % 2) * v for n, v in ht.items()}
    return dict(name="bior4.4", ht=ht, gt=gt, h=h, g=g)


def haar():
    """Haar bank in the same convention: a = (x0 + x1)/sqrt2, d = (x0 - x1)/sqrt2."""
    s = 1.0 / np.sqrt(2.0)
    return dict(name="haar", ht={0: s, 1: s}, gt={-1: s, 0: -s},
                h={0: s, 1: s}, g={-1: s, 0: -s})


def filter_bank(wavelet):
    """Bank by name or code: 'bior4.4' / 0, 'haar' / 1."""
    if wavelet in ("bior4.4", 0):
        return bior44()
    if wavelet in ("haar", 1):
        return haar()
    raise ValueError(wavelet)
