"""Synthetic fine-tuning workloads built entirely through the C ABI.

A workload is one entry of vbm_inputs.configs: a seeded synthetic volume (or
several, for uneven batches) turned into Gaussians by vbm_build and rendered
to DVR target images by vbm_render_dvr on the GPU.
"""

import numpy as np
import torch

from vbm_inputs import TF_KNOTS_RGBA, TF_KNOTS_X, config, orbit_cameras, tf_mode, tf_modes_union, volume_for_config
from vbm_inputs.cameras import camera_array

from . import vbm


class Workload:
    """Gaussians P[14][n], packed cameras, target images [V][3][H][W] (device)."""

    def __init__(self, cfg, params, n, cam_records, cams, targets, scene_offset=None, view_scene=None, volumes=None,
                 union_targets=None):
        self.cfg = cfg
        self.params = params
        self.n = n
        self.cam_records = cam_records
        self.cams = cams
        self.targets = targets
        self.scene_offset = scene_offset
        self.view_scene = view_scene
        self.volumes = volumes
        # TF-mode workloads: DVR of the sum of the modes' TFs on one mode's
        # cameras, the target of the concatenated Gaussian sets
        self.union_targets = union_targets

    @property
    def views(self):
        return self.targets.shape[0]


def _build_one(F, levels, K_tot, device, tf, wavelet=0, ablation=0):
    G = F.shape
    dims = (G[2], G[1], G[0])
    bank = vbm.bank_build(levels, wavelet)
    if ablation:
        vbm.bank_ablate(bank, ablation)
    Fd = torch.from_numpy(F).to(device)
    params, n = vbm.build(Fd, dims, tf, bank, vbm.make_select(K_tot), capacity=2 * K_tot + 1024)
    return Fd, dims, params[:, :n].contiguous(), n


def _render_targets(Fd, dims, tf, cams, width, height, device):
    recs = camera_array(cams)
    cams_dev = vbm.cameras_to_device(recs, device)
    rgba = torch.zeros((len(cams), 4, height, width), device=device)
    vbm.render_dvr(Fd, dims, tf, cams_dev, len(cams), width, height, 0.5, rgba)
    return recs, rgba[:, :3].contiguous()


def make_workload(key, device="cuda", wavelet=0, ablation=0):
    """Build workload `key`; wavelet 1 (Haar) and the bank ablation flags give the
    ablation variants of Sec. 5.4 (the targets are the same DVR images)."""
    cfg = config(key)
    tf = vbm.make_tf(TF_KNOTS_X, TF_KNOTS_RGBA)
    if "edges" in cfg:                      # uneven batch of independent volumes
        Ps, so, recs_all, cams_all, tgts, vs = [], [0], [], [], [], []
        for i, G in enumerate(cfg["edges"]):
            F = volume_for_config(cfg, i)
            K = int(cfg["K_tot_frac"] * G ** 3)
            Fd, dims, P, n = _build_one(F, cfg["levels"], K, device, tf, wavelet, ablation)
            cams = orbit_cameras(dims, cfg["views_per_volume"], cfg["width"], cfg["height"])
            recs, tgt = _render_targets(Fd, dims, tf, cams, cfg["width"], cfg["height"], device)
            Ps.append(P)
            so.append(so[-1] + n)
            recs_all.append(recs)
            cams_all.extend(cams)
            tgts.append(tgt)
            vs.extend([i] * len(cams))
        params = torch.cat(Ps, dim=1).contiguous()
        torch.cuda.synchronize()
        return Workload(cfg, params, int(so[-1]), np.concatenate(recs_all), cams_all, torch.cat(tgts),
                        scene_offset=np.asarray(so, dtype=np.int64), view_scene=np.asarray(vs, dtype=np.int32))
    if "modes" in cfg:                      # one Gaussian set per TF mode (Sec. 4.4)
        F = volume_for_config(cfg)
        Ps, so, tgts, vs = [], [0], [], []
        cams = recs = None
        for h in range(cfg["modes"]):
            tf_h = vbm.make_tf(*tf_mode(h))
            Fd, dims, P, n = _build_one(F, cfg["levels"], cfg["K_tot"], device, tf_h, wavelet, ablation)
            cams = orbit_cameras(dims, cfg["views"], cfg["width"], cfg["height"])
            recs, tgt = _render_targets(Fd, dims, tf_h, cams, cfg["width"], cfg["height"], device)
            Ps.append(P)
            so.append(so[-1] + n)
            tgts.append(tgt)
            vs.extend([h] * len(cams))
        _, union = _render_targets(Fd, dims, vbm.make_tf(*tf_modes_union()), cams, cfg["width"], cfg["height"],
                                   device)
        params = torch.cat(Ps, dim=1).contiguous()
        torch.cuda.synchronize()
        H = cfg["modes"]
        return Workload(cfg, params, int(so[-1]), np.concatenate([recs] * H), cams * H, torch.cat(tgts),
                        scene_offset=np.asarray(so, dtype=np.int64), view_scene=np.asarray(vs, dtype=np.int32),
                        volumes=[F], union_targets=union)
    F = volume_for_config(cfg)
    Fd, dims, params, n = _build_one(F, cfg["levels"], cfg["K_tot"], device, tf, wavelet, ablation)
    cams = orbit_cameras(dims, cfg["views"], cfg["width"], cfg["height"])
    recs, targets = _render_targets(Fd, dims, tf, cams, cfg["width"], cfg["height"], device)
    torch.cuda.synchronize()
    return Workload(cfg, params, n, recs, cams, targets, volumes=[F])
