"""vbm_loss_static, the allocation-free variant of vbm_loss.

Callers that cannot allocate device memory when they need the loss (for
example while a CUDA graph is being captured, or under a memory budget fixed
at start-up) use this entry point; its scratch is a static array inside the
library.  Both entry points run the same kernels on the same inputs, so the
results must be bit-identical: the tests call it through the C ABI twice in a
row against vbm_loss with a workspace on different inputs (a stale scratch
word would show), replay it from a captured CUDA graph after a warm-up call,
split a batch into per-image calls with accumulate, and check the size limits.
This file is collected last.
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


def _reference(vbm, x, y, scale):
    V, _, H, W = x.shape
    ws = vbm.loss_workspace(V, H, W)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    vbm.loss(x, y, V, H, W, 0.2, scale, L, g, ws)
    return L, g


def test_static_loss_matches_workspace_loss_twice(cuda_lib):
    vbm = cuda_lib
    for seed, (V, H, W) in [(1, (2, 96, 80)), (2, (3, 57, 131))]:
        x, y = _inputs(seed, V, H, W)
        scale = 1.0 / x.numel()
        L_ref, g_ref = _reference(vbm, x, y, scale)
        L = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
        g = torch.full_like(x, 7.0)
        vbm.loss_static(x, y, V, H, W, 0.2, scale, L, g)
        torch.cuda.synchronize()
        assert L.item() == L_ref.item()
        assert torch.equal(g, g_ref)


def test_static_loss_replayed_from_a_captured_graph(cuda_lib):
    """After one warm-up call on the device, the call is captured into a CUDA graph; new
    inputs are copied into the captured buffers and the replay equals vbm_loss on them."""
    vbm = cuda_lib
    V, H, W = 2, 64, 72
    x, y = _inputs(5, V, H, W)
    scale = 1.0 / x.numel()
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    vbm.loss_static(x, y, V, H, W, 0.2, scale, L, g)      # warm-up: symbol lookup, window upload
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        vbm.loss_static(x, y, V, H, W, 0.2, scale, L, g)
    for seed in (6, 7):
        x2, y2 = _inputs(seed, V, H, W)
        x.copy_(x2)
        y.copy_(y2)
        graph.replay()
        torch.cuda.synchronize()
        L_ref, g_ref = _reference(vbm, x2, y2, scale)
        torch.cuda.synchronize()
        assert L.item() == L_ref.item()
        assert torch.equal(g, g_ref)


def test_static_loss_per_image_accumulate(cuda_lib):
    """A batch split into one call per image with accumulate gives the whole batch's
    gradient bit for bit and its loss up to the FP64 summation order."""
    vbm = cuda_lib
    V, H, W = 4, 50, 66
    x, y = _inputs(9, V, H, W)
    scale = 1.0 / x.numel()
    L_ref, g_ref = _reference(vbm, x, y, scale)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for v in range(V):
        vbm.loss_static(x[v:v + 1], y[v:v + 1], 1, H, W, 0.2, scale, L, g[v:v + 1], accumulate=v > 0)
    torch.cuda.synchronize()
    assert abs(L.item() - L_ref.item()) <= 1e-12 * abs(L_ref.item())
    assert torch.equal(g, g_ref)


def test_static_loss_rejects_oversized_batches(cuda_lib):
    vbm = cuda_lib
    x = torch.zeros((8, 3, 512, 512), device="cuda")
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(vbm.VbmError) as e:
        vbm.loss_static(x, x, 8, 512, 512, 0.2, 1.0, L, torch.empty_like(x))
    assert e.value.status == vbm.VBM_ERR_CAPACITY
    assert "static" in str(e.value)
    # more images than the grid's z-slices hold: an argument error before any launch,
    # from both entry points
    n = 65535 // 3 + 1
    x = torch.zeros((n, 3, 1, 1), device="cuda")
    with pytest.raises(vbm.VbmError) as e:
        vbm.loss_static(x, x, n, 1, 1, 0.2, 1.0, L, torch.empty_like(x))
    assert e.value.status == vbm.VBM_ERR_ARG
    with pytest.raises(vbm.VbmError) as e:
        vbm.loss(x, x, n, 1, 1, 0.2, 1.0, L, torch.empty_like(x), vbm.loss_workspace(n, 1, 1))
    assert e.value.status == vbm.VBM_ERR_ARG
