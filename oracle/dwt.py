"""Periodised separable 3D discrete wavelet transform (oracle, test infrastructure only).

Follows the multiresolution expansion of Sec. 3 (Eq. 1-3) and the multichannel
J-level transform of Sec. 4.3 (Eq. 20-21).  Readings taken where the paper is
silent or inconsistent:
  * Boundary: periodisation.  Sec. 4.2 allows "symmetric or periodic"
    extensions; periodisation keeps every subband exactly size n / 2^j and
    makes the translation theorem of Supp. Sec. 2 exact on the grid.
  * Level index: j = 1..J with j = 1 the finest level, so a level-j
    coefficient has stride 2^j on the input grid, matching the translation
    T_{2^j k} of Eq. 12 / Eq. 19.  The approximation band LLL exists only at
    j = J (the paper's count "8(J+1)" in Sec. 4.2 includes LLL bands that a
    J-level transform does not keep).
  * Layout: Mallat.  After level j the array region [0, n/2^(j-1))^3 holds
    eight octants indexed by o = (o_x, o_y, o_z) in {L=0, H=1}^3; octant o
    occupies [o_d n/2^j, (o_d + 1) n/2^j) along axis d.  Level j+1 recurses
    into the LLL octant.
Arrays are indexed [z, y, x]; axis 2 is x.

The filter convention (analysis and synthesis sums) is stated in oracle.filters.
"""

import numpy as np

AXIS_OF = {0: 2, 1: 1, 2: 0}  # spatial dimension d (x, y, z) -> numpy axis


def analysis_1d(x, axis, bank):
    """One periodised analysis step along an axis: returns [a | d] concatenated.

    a[k] = sum_n ht[n] x[(2k + n) mod L],  d[k] = sum_n gt[n] x[(2k + 1 + n) mod L].
    """
    L = x.shape[axis]
    assert L % 2 == 0, "periodised DWT needs an even length"
    k = np.arange(L // 2)
    a = 0.0
    for n, c in bank["ht"].items():
        a = a + c * np.take(x, (2 * k + n) % L, axis=axis)
    d = 0.0
    for n, c in bank["gt"].items():
        d = d + c * np.take(x, (2 * k + 1 + n) % L, axis=axis)
    return np.concatenate([a, d], axis=axis)


def synthesis_1d(c, axis, bank):
    """Inverse of analysis_1d: x[m] = sum_k h[m-2k] a[k] + sum_k g[m-2k-1] d[k].

    Written as a scatter: every a[k] adds h[n] a[k] at 2k + n, every d[k] adds
    g[n] d[k] at 2k + 1 + n (indices mod L).  For a fixed tap n the targets
    (2k + n) mod L are distinct over k, so each tap is one indexed add.
    """
    L = c.shape[axis]
    half = L // 2
    a = np.take(c, np.arange(half), axis=axis)
    d = np.take(c, np.arange(half, L), axis=axis)
    out_shape = list(c.shape)
    x = np.zeros(out_shape, dtype=np.result_type(c, np.float64))
    k = np.arange(half)
    xm = np.moveaxis(x, axis, 0)
    am = np.moveaxis(a, axis, 0)
    dm = np.moveaxis(d, axis, 0)
    for n, hv in bank["h"].items():
        xm[(2 * k + n) % L] += hv * am
    for n, gv in bank["g"].items():
        xm[(2 * k + 1 + n) % L] += gv * dm
    return x


def dwt3d(vol, levels, bank):
    """J-level 3D DWT of a (nz, ny, nx) array into a same-shape Mallat pyramid."""
    out = np.array(vol, dtype=np.float64, copy=True)
    nz, ny, nx = out.shape
    for j in range(1, levels + 1):
        sz, sy, sx = nz >> (j - 1), ny >> (j - 1), nx >> (j - 1)
        block = out[:sz, :sy, :sx]
        for axis in (2, 1, 0):           # x, then y, then z
            block = analysis_1d(block, axis, bank)
        out[:sz, :sy, :sx] = block
    return out


def idwt3d(pyr, levels, bank):
    """Inverse of dwt3d."""
    out = np.array(pyr, dtype=np.float64, copy=True)
    nz, ny, nx = out.shape
    for j in range(levels, 0, -1):
        sz, sy, sx = nz >> (j - 1), ny >> (j - 1), nx >> (j - 1)
        block = out[:sz, :sy, :sx]
        for axis in (0, 1, 2):           # undo z, then y, then x
            block = synthesis_1d(block, axis, bank)
        out[:sz, :sy, :sx] = block
    return out


def subbands(levels):
    """All kept subbands as (j, o) with o = (o_x, o_y, o_z), 0 = L, 1 = H.

    Seven detail bands per level j = 1..J plus the approximation band LLL at
    j = J: 7J + 1 in total.  Order: j ascending, o in binary order o_x + 2 o_y
    + 4 o_z, with LLL (o = 0) present only at j = J.
    """
    out = []
    for j in range(1, levels + 1):
        for code in range(8):
            o = (code & 1, (code >> 1) & 1, (code >> 2) & 1)
            if code == 0 and j != levels:
                continue
            out.append((j, o))
    return out


def subband_slices(shape, j, o):
    """numpy slices (z, y, x) of subband (j, o) inside a Mallat pyramid."""
    nz, ny, nx = shape
    sl = []
    for d, n in ((2, nz), (1, ny), (0, nx)):
        m = n >> j
        sl.append(slice(o[d] * m, (o[d] + 1) * m))
    return tuple(sl)


def impulse_response(shape, levels, j, o, k, bank):
    """IDWT of a unit impulse at index k = (kx, ky, kz) of subband (j, o) (Eq. 9-11)."""
    pyr = np.zeros(shape, dtype=np.float64)
    sl = subband_slices(shape, j, o)
    pyr[sl[0].start + k[2], sl[1].start + k[1], sl[2].start + k[0]] = 1.0
    return idwt3d(pyr, levels, bank)


def impulse_response_1d(length, j, band, k, bank):
    """1D IDWT (j levels) of a unit impulse at index k of the level-j band.

    band 0 = approximation (low-pass chain), 1 = detail.  Used for the
    separability check of the 3D canonical kernels (Supp. Sec. 2, Step 1).
    """
    c = np.zeros(length, dtype=np.float64)
    m = length >> j
    c[band * m + k] = 1.0
    for lev in range(j, 0, -1):
        n = length >> (lev - 1)
        c[:n] = synthesis_1d(c[:n], 0, bank)
    return c
