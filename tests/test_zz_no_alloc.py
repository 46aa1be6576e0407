"""vbm_loss_static, the allocation-free variant of vbm_loss.

Callers that cannot allocate device memory when they need the loss (for
example while a CUDA graph is being captured, or under a memory budget fixed
at start-up) use this entry point; its scratch is a static array inside the
library.  The test calls it through the C ABI twice in a row, each time
against vbm_loss with a workspace on different inputs, and checks the
size limit.  It lives in a file that pytest collects last.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(seed, V, H, W):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1).astype(np.float32)
    return torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()


def test_static_loss_matches_workspace_loss_twice(cuda_lib):
    vbm = cuda_lib
    for seed, (V, H, W) in [(1, (2, 96, 80)), (2, (3, 57, 131))]:
        x, y = _inputs(seed, V, H, W)
        scale = 1.0 / x.numel()
        ws = vbm.loss_workspace(V, H, W)
        L_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        g_ref = torch.empty_like(x)
        vbm.loss(x, y, V, H, W, 0.2, scale, L_ref, g_ref, ws)
        L = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
        g = torch.full_like(x, 7.0)
        vbm.loss_static(x, y, V, H, W, 0.2, scale, L, g)
        torch.cuda.synchronize()
        assert abs(L.item() - L_ref.item()) <= 1e-6 * abs(L_ref.item())
        err = (g - g_ref).abs().max().item()
        assert err <= 1e-3 * g_ref.abs().max().item(), err


def test_static_loss_rejects_oversized_batches(cuda_lib):
    vbm = cuda_lib
    x = torch.zeros((8, 3, 512, 512), device="cuda")
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(vbm.VbmError) as e:
        vbm.loss_static(x, x, 8, 512, 512, 0.2, 1.0, L, torch.empty_like(x))
    assert e.value.status == vbm.VBM_ERR_CAPACITY
    assert "static" in str(e.value)
