"""The 8-knot RGBA transfer-function table used by every workload.

A transfer function maps the scalar field to colour and opacity (Sec. 3,
"Transfer Function").  The paper's own TFs are not printed; this table is a
typical one that is zero-opacity near 0 and non-zero only over part of the
value range, as the fine-tuning section describes for its TF modes
(Sec. 4.4).  Knots sit at x = i/7, i = 0..7.
"""

import numpy as np

TF_KNOTS_X = np.arange(8, dtype=np.float64) / 7.0
TF_KNOTS_RGBA = np.array([
    [0.00, 0.00, 0.00, 0.00],
    [0.10, 0.10, 0.60, 0.00],
    [0.10, 0.50, 0.90, 0.02],
    [0.20, 0.80, 0.60, 0.06],
    [0.60, 0.90, 0.20, 0.12],
    [0.95, 0.75, 0.10, 0.25],
    [0.95, 0.35, 0.10, 0.45],
    [1.00, 1.00, 1.00, 0.70],
], dtype=np.float64)


def transfer_function(x=None, rgba=None):
    """The knot table as a dict {x: (K,), rgba: (K, 4)} (float64 copies)."""
    return dict(x=(TF_KNOTS_X if x is None else np.asarray(x, np.float64)).copy(),
                rgba=(TF_KNOTS_RGBA if rgba is None else np.asarray(rgba, np.float64)).copy())
