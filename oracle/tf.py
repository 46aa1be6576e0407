"""Transfer function (oracle, test infrastructure only).

Sec. 3 ("Transfer Function"): TF maps the scalar field to an RGBA radiance
field, RF = TF(F).  The paper does not give the interpolation; the reading
here is piecewise-linear in each channel between ascending knots, with the
scalar clamped to [0, 1] and constant extrapolation outside the knot range.
"""

import numpy as np


def apply_tf(F, knots_x, knots_rgba):
    """RGBA = TF(F) for an array F of any shape; returns shape F.shape + (4,), float64.

    For f in [x_i, x_{i+1}]: value = (1 - t) rgba_i + t rgba_{i+1},
    t = (f - x_i) / (x_{i+1} - x_i).
    """
    x = np.asarray(knots_x, dtype=np.float64)
    v = np.asarray(knots_rgba, dtype=np.float64)
    f = np.clip(np.asarray(F, dtype=np.float64), 0.0, 1.0)
    out = np.empty(f.shape + (4,), dtype=np.float64)
    flat = f.reshape(-1)
    res = out.reshape(-1, 4)
    for idx in range(flat.size):
        fi = flat[idx]
        if fi <= x[0]:
            res[idx] = v[0]
            continue
        if fi >= x[-1]:
            res[idx] = v[-1]
            continue
        i = np.searchsorted(x, fi, side="right") - 1
        t = (fi - x[i]) / (x[i + 1] - x[i])
        res[idx] = (1.0 - t) * v[i] + t * v[i + 1]
    return out


def apply_tf_vectorised(F, knots_x, knots_rgba):
    """Same map as apply_tf, evaluated channel by channel with whole-array ops."""
    x = np.asarray(knots_x, dtype=np.float64)
    v = np.asarray(knots_rgba, dtype=np.float64)
    f = np.clip(np.asarray(F, dtype=np.float64), 0.0, 1.0)
    i = np.clip(np.searchsorted(x, f, side="right") - 1, 0, x.size - 2)
    t = np.clip((f - x[i]) / (x[i + 1] - x[i]), 0.0, 1.0)
    return (1.0 - t)[..., None] * v[i] + t[..., None] * v[i + 1]
