"""Image-space fine-tuning of the Gaussians (Sec. 4.4), one step = render all views,
L1 + D-SSIM loss against the targets, backward to every parameter, Adam.

Two forms of the same step:
  * plain   -- one view per launch sequence: for each view, its forward,
               its loss term and its backward (accumulating the gradient),
               then one Adam update;
  * batched -- every view (and every scene of an uneven batch) in one
               launch per kernel, the whole step captured once as a CUDA
               graph and replayed.
Both run only the library's kernels; this module allocates the buffers,
sequences the C-ABI calls and owns the graph.
"""

import numpy as np
import torch

from . import vbm


def default_lrs(extent):
    """Per-row-group learning rates: mean, log-scale, quaternion, opacity, colour."""
    return [1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3]


# Share of the device memory free at plan creation that the stored per-pixel
# compositing state (final transmittance and last contributor, 8 bytes per
# pixel of the batch) may take before recompute="auto" chooses to recompute it
# in the backward instead.
STATE_MEMORY_SHARE = 0.05


def choose_recompute(n_pixels, free_bytes, share=STATE_MEMORY_SHARE):
    """True when storing the per-pixel state of n_pixels would take more than `share` of
    the free device memory: the backward then replays the forward's walk (only short
    lists in persistent plans) instead of reading stored state."""
    return 8 * int(n_pixels) > share * float(free_bytes)


class FineTuner:
    def __init__(self, params, cam_records, targets, scene_offset=None, view_scene=None, tile=(16, 16), ppt=0,
                 persistent=False, pair_capacity=None, lrs=None, lam=0.2, bg=(0.0, 0.0, 0.0), extent=None,
                 device="cuda", group_lanes=0, recompute=False, segment_len=0, radix_sort=False, bwd_ppt=0,
                 bwd_group_lanes=0, fused_adam=True):
        self.device = torch.device(device)
        self.params = params
        self.n = params.shape[1] if scene_offset is None else int(scene_offset[-1])
        self.V, _, self.H, self.W = targets.shape
        self.targets = targets
        self.cams = vbm.cameras_to_device(cam_records, self.device)
        self.bg = tuple(float(b) for b in bg)
        self.lam = float(lam)
        self.scene_offset = np.asarray([0, self.n] if scene_offset is None else scene_offset, dtype=np.int64)
        self.view_scene = view_scene
        if pair_capacity is None:
            pair_capacity = vbm.default_pair_capacity(vbm.batch_items(self.scene_offset, self.V, view_scene))
        self.tile, self.ppt, self.persistent = tuple(tile), int(ppt), bool(persistent)
        self.group_lanes = int(group_lanes)
        if recompute == "auto":
            free, _ = torch.cuda.mem_get_info(self.device)
            recompute = choose_recompute(self.V * self.H * self.W, free)
        self.recompute = bool(recompute)
        self.plan = vbm.Plan(self.scene_offset, self.V, self.W, self.H, view_scene=view_scene, tile_w=tile[0],
                             tile_h=tile[1], pair_capacity=min(pair_capacity, vbm.MAX_PAIR_CAPACITY), pixels_per_thread=ppt,
                             flags=(vbm.PLAN_PERSISTENT if persistent else 0) |
                             (vbm.PLAN_RECOMPUTE if recompute else 0) |
                             (vbm.PLAN_RADIX_SORT if radix_sort else 0), group_lanes=group_lanes,
                             segment_len=segment_len, bwd_pixels_per_thread=bwd_ppt,
                             bwd_group_lanes=bwd_group_lanes)
        self.img = torch.zeros((self.V, 3, self.H, self.W), device=self.device)
        self.dimg = torch.zeros_like(self.img)
        self.grad = torch.zeros_like(params)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.nonfinite = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.ws = vbm.loss_workspace(self.V, self.H, self.W, self.device)
        self.scale = 1.0 / (self.V * 3 * self.H * self.W)
        ext = extent if extent is not None else 1.0
        self.lrs = list(lrs) if lrs is not None else default_lrs(ext)
        self.fused_adam = bool(fused_adam)
        self.graph = None

    # -------------------------------------------------------------- steps
    def step_plain(self):
        """One view per launch sequence, then Adam (no graph)."""
        for v in range(self.V):
            self.plan.forward(self.params, self.cams, self.img, view_begin=v, view_count=1, bg=self.bg)
            vbm.loss(self.img[v], self.targets[v], 1, self.H, self.W, self.lam, self.scale, self.loss, self.dimg[v],
                     self.ws, accumulate=v > 0)
            self.plan.backward(self.params, self.cams, self.dimg, self.grad, view_begin=v, view_count=1,
                               bg=self.bg, accumulate=v > 0)
        vbm.adam(self.params, self.grad, self.m, self.v, self.n, self.step_count, self.lrs,
                 nonfinite=self.nonfinite)

    def _backward_and_adam(self):
        """The backward of the batched forward and the Adam step: fused (no gradient array
        written), or, with fused_adam = False, the separate calls (self.grad then holds the
        step's gradient)."""
        if self.fused_adam:
            self.plan.backward_adam(self.params, self.cams, self.dimg, self.m, self.v, self.n, self.step_count,
                                    self.lrs, bg=self.bg, nonfinite=self.nonfinite)
            return
        self.plan.backward(self.params, self.cams, self.dimg, self.grad, bg=self.bg)
        vbm.adam(self.params, self.grad, self.m, self.v, self.n, self.step_count, self.lrs,
                 nonfinite=self.nonfinite)

    def step_batched(self):
        """All views in one launch per kernel, then Adam."""
        self.plan.forward(self.params, self.cams, self.img, bg=self.bg)
        vbm.loss(self.img, self.targets, self.V, self.H, self.W, self.lam, self.scale, self.loss, self.dimg,
                 self.ws)
        self._backward_and_adam()

    def capture(self):
        """Capture step_batched as a CUDA graph (run it once first on a side stream)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            snapshot = [t.clone() for t in (self.params, self.m, self.v, self.step_count)]
            self.step_batched()
            for dst, src in zip((self.params, self.m, self.v, self.step_count), snapshot):
                dst.copy_(src)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step_batched()
        return self.graph

    def step_graph(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def _step_from_host(self, host_targets, host_loss, side):
        """The batched step with this step's targets copied from pinned host memory on a
        side branch (overlapping projection, binning and the forward compositing, joined
        before the loss) and the loss copied back to pinned host memory at the end."""
        main = torch.cuda.current_stream(self.device)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            self.targets.copy_(host_targets, non_blocking=True)
        self.plan.forward(self.params, self.cams, self.img, bg=self.bg)
        main.wait_stream(side)
        vbm.loss(self.img, self.targets, self.V, self.H, self.W, self.lam, self.scale, self.loss, self.dimg,
                 self.ws)
        self._backward_and_adam()
        host_loss.copy_(self.loss, non_blocking=True)

    def capture_host(self, host_targets, host_loss):
        """Capture the end-to-end step (host targets in, host loss out) as a CUDA graph."""
        side = torch.cuda.Stream(device=self.device)
        warm = torch.cuda.Stream(device=self.device)
        warm.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(warm):
            snapshot = [t.clone() for t in (self.params, self.m, self.v, self.step_count)]
            self._step_from_host(host_targets, host_loss, side)
            for dst, src in zip((self.params, self.m, self.v, self.step_count), snapshot):
                dst.copy_(src)
        torch.cuda.current_stream(self.device).wait_stream(warm)
        torch.cuda.synchronize(self.device)
        self.host_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.host_graph):
            self._step_from_host(host_targets, host_loss, side)
        self._host_bufs = (host_targets, host_loss)
        return self.host_graph

    def step_host(self, host_targets, host_loss):
        """End-to-end step through host memory: this step's targets are copied from pinned
        host memory and its loss read back to pinned host memory, inside one replayed
        graph (the target copy overlaps the forward)."""
        if getattr(self, "host_graph", None) is None or self._host_bufs[0] is not host_targets \
                or self._host_bufs[1] is not host_loss:
            self.capture_host(host_targets, host_loss)
        self.host_graph.replay()

    def check(self):
        """(ok, pairs_needed, nonfinite): synchronises."""
        ok, need = self.plan.check()
        return ok, need, int(self.nonfinite.item())
