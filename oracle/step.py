"""One image-space fine-tuning step, composed from the oracle parts (test infrastructure only).

Sec. 4.4: render the current Gaussians for a batch of views, compare with the
volume-rendered targets through the 3DGS image loss, back-propagate to every
Gaussian parameter and apply Adam (Sec. 5.2).
"""

import numpy as np

from .adam import adam_step
from .loss import loss_and_grad
from .raster import splat_backward, splat_forward


def finetune_step(P, m, v, step, cams, targets, lrs, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
                  lam=0.2, scene_offset=None, view_scene=None):
    """Updates P, m, v in place; returns (loss, grad, forward record)."""
    fwd = splat_forward(P, cams, tile_w, tile_h, bg, scene_offset, view_scene)
    L, dimg = loss_and_grad(fwd["img"], targets, lam)
    grad, _, _ = splat_backward(fwd, P, cams, dimg)
    adam_step(P, grad, m, v, step, lrs)
    return L, grad, fwd
