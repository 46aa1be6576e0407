"""Autotuner of the splatting launch configuration.

Candidates are (tile shape, pixels per thread, lanes per group, persistent).
The tile shape sets how finely splats are binned (smaller tiles: more pairs
to sort, fewer wasted evaluations per pixel); pixels per thread sets how many
pixels of a tile column one thread composites and therefore the number of
threads per block, which is also the number of list entries staged in shared
memory per round; lanes per group sets the pixel block whose own entry list a
lane group walks (smaller groups: fewer idle lanes, more reductions per
pixel in the backward); persistent runs the compositing kernels as one grid
of resident blocks taking tiles longest-list-first from a work queue instead
of one block per tile.
Each candidate runs the batch's forward and backward calls on the caller's
own Gaussians and cameras (median of a few timed repetitions, CUDA events on
the current stream), the two calls timed apart; for each tile shape and
persistence the fastest forward configuration is paired with the fastest
backward one (the backward's warp regions are its own), and the best few
pairs are timed again together, in turns, with more repetitions.  For a
persistent winner a last stage times the per-warp list length: the number of
list entries beyond which the backward walks a tile's list as separate
segments (SEGMENT_LENGTHS; -1 never splits).  Results are cached in a
JSON file keyed by device name and workload signature.
"""

import hashlib
import json
import os

import numpy as np
import torch

from . import vbm

CANDIDATES = [(tile, ppt, gl, pers)
              for tile in ((16, 16), (16, 8), (8, 16), (8, 8), (16, 4), (8, 4))
              for ppt in (1, 2, 4)
              for gl in (4, 8, 16, 32)
              for pers in (False, True)
              if tile[1] % (4 * ppt) == 0]   # a warp region is 4 thread rows of ppt pixels
SEGMENT_LENGTHS = (64, 128, 256, 512, -1)
DEFAULT = ((16, 16), 2, 32, False, 0)
CACHE_FORMAT = "v7"


def _cache_path():
    return os.environ.get("VBM_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json"))


def _signature(params, n, cam_bytes, W, H, scene_offset, view_scene):
    h = hashlib.sha256()
    h.update(np.asarray([n, W, H], dtype=np.int64).tobytes())
    h.update(cam_bytes)
    h.update(np.asarray(scene_offset, dtype=np.int64).tobytes())
    if view_scene is not None:
        h.update(np.asarray(view_scene, dtype=np.int32).tobytes())
    return h.hexdigest()[:16]


class _Trial:
    """A plan and buffers for one candidate; times forward + backward calls of the batch."""

    def __init__(self, params, cams_dev, n_views, W, H, scene_offset, view_scene, tile, ppt, gl, persistent,
                 pair_capacity, segment_len=0, bwd_ppt=0, bwd_gl=0, recompute=False):
        self.params, self.cams = params, cams_dev
        self.plan = vbm.Plan(scene_offset, n_views, W, H, view_scene=view_scene, tile_w=tile[0], tile_h=tile[1],
                             pair_capacity=pair_capacity, pixels_per_thread=ppt,
                             flags=(vbm.PLAN_PERSISTENT if persistent else 0) |
                             (vbm.PLAN_RECOMPUTE if recompute else 0), group_lanes=gl,
                             segment_len=segment_len, bwd_pixels_per_thread=bwd_ppt, bwd_group_lanes=bwd_gl)
        self.img = torch.zeros((n_views, 3, H, W), device=params.device)
        self.dimg = torch.full_like(self.img, 1e-6)
        self.grad = torch.zeros_like(params)

    def run(self, iters, split=False):
        """ms of `iters` forward + backward calls; with split, (forward ms, backward ms) pairs."""
        times = []
        for _ in range(iters):
            s, m, e = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            s.record()
            self.plan.forward(self.params, self.cams, self.img)
            m.record()
            self.plan.backward(self.params, self.cams, self.dimg, self.grad)
            e.record()
            e.synchronize()
            times.append((s.elapsed_time(m), m.elapsed_time(e)) if split else s.elapsed_time(e))
        return times

    def close(self):
        ok, need = self.plan.check()
        self.plan.close()
        return ok, need


def time_config(params, cams_dev, n_views, W, H, scene_offset, view_scene, tile, ppt, gl, persistent, pair_capacity,
                iters=5, recompute=False):
    """Median ms of one forward + backward call of the whole batch with this configuration, and
    the medians of the forward and the backward call alone; plus the pairs needed."""
    t = _Trial(params, cams_dev, n_views, W, H, scene_offset, view_scene, tile, ppt, gl, persistent, pair_capacity,
               recompute=recompute)
    times = t.run(iters + 2, split=True)[2:]
    ok, need = t.close()
    if not ok:
        return float("inf"), float("inf"), float("inf"), need
    return (float(np.median([a + b for a, b in times])), float(np.median([a for a, _ in times])),
            float(np.median([b for _, b in times])), need)


def retime(params, cams_dev, n_views, W, H, scene_offset, view_scene, configs, pair_capacity, rounds=8, iters=3,
           recompute=False):
    """Median ms of each configuration (tile, ppt, group lanes, persistent[, segment length[,
    backward ppt, backward group lanes]]),
    timed in turns (rounds x iters calls each) so that clock or thermal drift affects them
    alike."""
    trials = [_Trial(params, cams_dev, n_views, W, H, scene_offset, view_scene, *c[:4], pair_capacity, *c[4:],
                     recompute=recompute) for c in configs]
    for t in trials:
        t.run(2)
    times = [[] for _ in trials]
    for _ in range(rounds):
        for k, t in enumerate(trials):
            times[k] += t.run(iters)
    out = []
    for t, ts in zip(trials, times):
        ok, _ = t.close()
        out.append(float(np.median(ts)) if ok else float("inf"))
    return out


def autotune(params, cam_records, n_views, W, H, scene_offset=None, view_scene=None, pair_capacity=None,
             candidates=None, use_cache=True, recompute=False):
    """Best ((tile_w, tile_h), ppt, group_lanes, persistent, segment_len, bwd_ppt, bwd_group_lanes)
    for this workload, plus the table of timings (segment_len 0: the library's default; only
    persistent plans split lists; bwd_* 0: the forward's).
    recompute: time plans that keep no per-pixel state (VBM_PLAN_RECOMPUTE), as the caller will run."""
    n = int(params.shape[1] if scene_offset is None else scene_offset[-1])
    so = [0, n] if scene_offset is None else list(scene_offset)
    raw = np.ascontiguousarray(cam_records).view(np.uint8).tobytes()
    dev = torch.cuda.get_device_name(params.device)
    key = "%s|%s|%s|%d" % (CACHE_FORMAT, dev, _signature(params, n, raw, W, H, so, view_scene), int(recompute))
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        ent = cache[key]
        return (tuple(ent["tile"]), ent["ppt"], ent["group_lanes"], ent["persistent"], ent["segment_len"],
                ent["bwd_ppt"], ent["bwd_group_lanes"]), ent["table"]
    cams_dev = vbm.cameras_to_device(cam_records, params.device)
    cap = pair_capacity if pair_capacity is not None else vbm.default_pair_capacity(
        vbm.batch_items(so, n_views, view_scene))
    cap = min(cap, vbm.MAX_PAIR_CAPACITY)
    table = []
    for tile, ppt, gl, persistent in (candidates or CANDIDATES):
        ms, ms_f, ms_b, need = time_config(params, cams_dev, n_views, W, H, so, view_scene, tile, ppt, gl,
                                           persistent, cap, recompute=recompute)
        table.append({"tile": list(tile), "ppt": ppt, "group_lanes": gl, "persistent": persistent, "ms": ms,
                      "ms_fwd": ms_f, "ms_bwd": ms_b, "pairs_needed": need})
    # per (tile, persistence): the fastest forward configuration with the fastest
    # backward one; the best few of these pairs again, in turns, together
    combos = []
    for tp in sorted({(tuple(r["tile"]), r["persistent"]) for r in table}):
        rows = [r for r in table if (tuple(r["tile"]), r["persistent"]) == tp]
        f = min(rows, key=lambda r: r["ms_fwd"])
        b = min(rows, key=lambda r: r["ms_bwd"])
        combos.append((f["ms_fwd"] + b["ms_bwd"], tp[0], f["ppt"], f["group_lanes"], tp[1], b["ppt"],
                       b["group_lanes"]))
    combos = sorted(c for c in combos if np.isfinite(c[0]))[:4] or [(0.0,) + tuple(DEFAULT[:4]) + (0, 0)]
    finals = retime(params, cams_dev, n_views, W, H, so, view_scene,
                    [(c[1], c[2], c[3], c[4], 0, c[5], c[6]) for c in combos], cap, recompute=recompute)
    for c, ms in zip(combos, finals):
        table.append({"tile": list(c[1]), "ppt": c[2], "group_lanes": c[3], "persistent": c[4], "bwd_ppt": c[5],
                      "bwd_group_lanes": c[6], "ms": c[0], "ms_final": ms, "stage": "combination"})
    _, tile, ppt_b, gl_b, pers_b, bwd_ppt, bwd_gl = combos[int(np.argmin(finals))]
    best = {"tile": list(tile), "ppt": ppt_b, "group_lanes": gl_b, "persistent": pers_b}
    seg = 0
    if pers_b:
        segs = retime(params, cams_dev, n_views, W, H, so, view_scene,
                      [(tile, ppt_b, gl_b, True, s_len, bwd_ppt, bwd_gl) for s_len in SEGMENT_LENGTHS], cap,
                      recompute=recompute)
        for s_len, ms in zip(SEGMENT_LENGTHS, segs):
            table.append({"tile": list(tile), "ppt": ppt_b, "group_lanes": gl_b, "persistent": True,
                          "bwd_ppt": bwd_ppt, "bwd_group_lanes": bwd_gl, "segment_len": s_len, "ms": ms,
                          "ms_final": ms, "stage": "segment"})
        seg = SEGMENT_LENGTHS[int(np.argmin(segs))]
    if use_cache:
        cache[key] = {"tile": best["tile"], "ppt": best["ppt"], "group_lanes": best["group_lanes"],
                      "persistent": best["persistent"], "segment_len": seg, "bwd_ppt": bwd_ppt,
                      "bwd_group_lanes": bwd_gl, "table": table}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".%d.tmp" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return (tuple(best["tile"]), best["ppt"], best["group_lanes"], best["persistent"], seg, bwd_ppt, bwd_gl), table
