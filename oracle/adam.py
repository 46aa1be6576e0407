"""Adam update of the Gaussian parameters (oracle, test infrastructure only).

Sec. 5.2 states that Adam is used; its hyper-parameters are not given.
Readings (3D Gaussian Splatting ranges, fixed learning rates, no schedule):
beta1 = 0.9, beta2 = 0.999, eps = 1e-15, bias correction as in Kingma & Ba
(2015), learning rate per parameter row group of the P[14][N] layout:
  mean 1.6e-4 * extent (extent = largest volume edge), log_scale 5e-3,
  quaternion 1e-3, opacity logit 5e-2, colour 2.5e-3.
"""

import numpy as np

ROW_GROUPS = [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]


def default_lrs(extent):
    return [1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3]


def adam_step(P, grad, m, v, step, lrs, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step in place on float64 arrays of shape (14, N); step = t (1-based)."""
    for (lo, hi), lr in zip(ROW_GROUPS, lrs):
        g = grad[lo:hi]
        m[lo:hi] = beta1 * m[lo:hi] + (1.0 - beta1) * g
        v[lo:hi] = beta2 * v[lo:hi] + (1.0 - beta2) * g * g
        mhat = m[lo:hi] / (1.0 - beta1 ** step)
        vhat = v[lo:hi] / (1.0 - beta2 ** step)
        P[lo:hi] -= lr * mhat / (np.sqrt(vhat) + eps)
    return P, m, v
