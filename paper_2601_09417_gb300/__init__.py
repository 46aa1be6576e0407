"""GB300 (sm_103a) implementation of Variable Basis Mapping (arXiv 2601.09417).

The compute path is the C-ABI library libvbm.so (include/vbm.h), built from the
CUDA sources in csrc/ by build_ext.  `vbm` is its thin ctypes binding,
`autograd` wraps the splatting forward/backward as a torch.autograd.Function
and `finetune` composes the image-space fine-tuning step (plain and batched,
CUDA-graph captured).
"""

from . import vbm  # noqa: F401

__all__ = ["vbm"]
