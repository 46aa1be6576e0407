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


# Transfer-function modes (Sec. 4.4: one TF per visual mode, each non-zero only
# over its own interval of the field's values): five hats over adjacent,
# disjoint intervals of [0.10, 0.95], each with its own colour and peak
# opacity, zero at and beyond the interval's ends.
TF_MODE_EDGES = np.array([0.10, 0.27, 0.44, 0.61, 0.78, 0.95], dtype=np.float64)
TF_MODE_RGBA = np.array([
    [0.15, 0.35, 0.95, 0.06],
    [0.10, 0.85, 0.85, 0.10],
    [0.25, 0.90, 0.25, 0.16],
    [0.95, 0.65, 0.10, 0.28],
    [0.95, 0.15, 0.10, 0.45],
], dtype=np.float64)


def tf_mode(h):
    """Knots (x, rgba) of mode h: zero up to the interval's start, the mode's
    colour and opacity at its midpoint, zero from its end on."""
    a, b = TF_MODE_EDGES[h], TF_MODE_EDGES[h + 1]
    x = np.array([0.0, a, 0.5 * (a + b), b, 1.0])
    rgba = np.zeros((5, 4))
    rgba[2] = TF_MODE_RGBA[h]
    return x, rgba


def tf_modes_union():
    """One TF equal to the sum of the five modes (their supports are disjoint):
    knots at every interval edge and midpoint."""
    xs, rgbas = [0.0], [np.zeros(4)]
    for h in range(len(TF_MODE_RGBA)):
        a, b = TF_MODE_EDGES[h], TF_MODE_EDGES[h + 1]
        if h == 0:
            xs.append(a)
            rgbas.append(np.zeros(4))
        xs += [0.5 * (a + b), b]
        rgbas += [TF_MODE_RGBA[h].copy(), np.zeros(4)]
    xs.append(1.0)
    rgbas.append(np.zeros(4))
    return np.array(xs), np.array(rgbas)
