"""Seeded random Gaussian parameter sets for splatting tests.

Parameter layout (shared with the C ABI): a float array P[14][stride], one row
per scalar attribute, column i = Gaussian i:
  rows 0-2   mean (x, y, z), world units (voxels)
  rows 3-5   log of the per-axis standard deviation
  rows 6-9   rotation quaternion (w, x, y, z), not necessarily unit length
  row  10    opacity logit
  rows 11-13 colour (r, g, b)
"""

import numpy as np

N_ROWS = 14
ROW_MEAN, ROW_LOG_SCALE, ROW_QUAT, ROW_OPACITY, ROW_COLOR = 0, 3, 6, 10, 11


def random_gaussians(n, box_lo, box_hi, seed, scale_range=(0.4, 3.0),
                     opacity_logit_range=(-3.0, 2.0), stride=None, dtype=np.float64):
    """n random Gaussians with means uniform in the box [box_lo, box_hi]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    stride = n if stride is None else stride
    P = np.zeros((N_ROWS, stride), dtype=np.float64)
    P[0:3, :n] = rng.uniform(box_lo, box_hi, size=(3, n))
    P[3:6, :n] = np.log(rng.uniform(scale_range[0], scale_range[1], size=(3, n)))
    q = rng.standard_normal((4, n))
    q *= rng.uniform(0.5, 2.0, size=(1, n)) / np.linalg.norm(q, axis=0, keepdims=True)
    P[6:10, :n] = q
    P[10, :n] = rng.uniform(opacity_logit_range[0], opacity_logit_range[1], size=n)
    P[11:14, :n] = rng.uniform(0.0, 1.0, size=(3, n))
    return P.astype(dtype)


def gaussians_in_view(n, G, seed, **kw):
    """Random Gaussians inside the central 80% of a G^3 volume box."""
    return random_gaussians(n, 0.1 * G, 0.9 * G, seed, **kw)
