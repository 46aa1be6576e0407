"""Convergence of the image-space fine-tuning from the VBM initialisation versus a
random initialisation with the same number of Gaussians (the comparison behind the
paper's fine-tuning experiments, Sec. 5.3 / Table 1, run here on a synthetic workload),
and the ablation variants of Sec. 5.4: the bank's covariances collapsed to one
isotropic one, unit energy weights, and the Haar wavelet instead of bior4.4.

Both runs use the same targets (vbm_render_dvr), cameras, loss, learning rates and
launch configuration; only the initial Gaussians differ.  The random initialisation
follows the usual 3DGS recipe for a volume: means uniform in the volume box,
isotropic scale equal to half the mean spacing (G^3 / N)^(1/3) / 2, identity
rotation, opacity 0.1, colour uniform in [0, 1] (seeded).

Every `every` steps the views are rendered and scored against the targets: PSNR from
the mean squared error over all views and channels, and the mean SSIM from the
library's own loss kernel (11 x 11 Gaussian window, sigma 1.5).  For the TF-mode
workload (one Gaussian set per mode, Sec. 4.4) the sets are also rendered together,
as one scene, and scored against the DVR of the sum of the modes' TFs.

    python -m paper_2601_09417_gb300.convergence --config c1 --steps 2000 --every 250
    python -m paper_2601_09417_gb300.convergence --variants full,isotropic,unit_weight,haar,random
"""

import argparse
import json
import math

import numpy as np
import torch

from . import vbm
from .finetune import FineTuner
from .workloads import make_workload


def random_init(n, G, seed=0):
    """P[14][n] (float32): the random initialisation described in the module docstring."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.zeros((14, n), dtype=np.float64)
    P[0:3] = rng.uniform(0.0, G, size=(3, n))
    P[3:6] = math.log(0.5 * (G ** 3 / n) ** (1.0 / 3.0))
    P[6] = 1.0
    P[10] = math.log(0.1 / 0.9)
    P[11:14] = rng.uniform(0.0, 1.0, size=(3, n))
    return P.astype(np.float32)


def image_score(img, tgt, ws):
    """(PSNR in dB, mean SSIM) of images [V][3][H][W] against targets of the same shape."""
    V, _, H, W = img.shape
    loss = torch.zeros(1, dtype=torch.float64, device=img.device)
    dimg = torch.empty_like(img)
    vbm.loss(img, tgt, V, H, W, 1.0, 1.0 / img.numel(), loss, dimg, ws)   # lambda = 1: 1 - SSIM
    torch.cuda.synchronize(img.device)
    a = img.cpu().numpy().astype(np.float64)
    b = tgt.cpu().numpy().astype(np.float64)
    mse = float(np.mean((a - b) ** 2))
    psnr = 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf")
    return psnr, 1.0 - float(loss.item())


def score(ft):
    """(PSNR in dB, mean SSIM) of the current Gaussians' renders against the targets."""
    ft.plan.forward(ft.params, ft.cams, ft.img, bg=ft.bg)
    return image_score(ft.img, ft.targets, ft.ws)


class ConcatScore:
    """Renders every Gaussian set of a TF-mode batch together, as one scene, on the first
    mode's cameras and scores it against the DVR of the modes' summed TF."""

    def __init__(self, ft, w, tile):
        self.targets = w.union_targets
        V, _, H, W = self.targets.shape
        n = ft.params.shape[1]
        self.cams = vbm.cameras_to_device(w.cam_records[:V], ft.device)
        self.plan = vbm.Plan([0, n], V, W, H, tile_w=tile[0], tile_h=tile[1],
                             pair_capacity=vbm.default_pair_capacity(n * V))
        self.img = torch.zeros_like(self.targets)
        self.ft = ft

    def __call__(self):
        self.plan.forward(self.ft.params, self.cams, self.img, bg=self.ft.bg)
        return image_score(self.img, self.targets, self.ft.ws)


def run(ft, steps, every, extra=None):
    """[(step, PSNR, SSIM[, concatenated PSNR, SSIM])] every `every` steps."""
    def point(k):
        return (k,) + score(ft) + (extra() if extra else ())
    curve = [point(0)]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        for _ in range(k):
            ft.step_graph()
        done += k
        curve.append(point(done))
    return curve


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c1")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--tile", default="8x8")
    ap.add_argument("--ppt", type=int, default=1)
    ap.add_argument("--gl", type=int, default=16)
    ap.add_argument("--variants", default="full,random",
                    help="comma list of full, isotropic, unit_weight, haar, random")
    args = ap.parse_args()
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w = make_workload(args.config, device)
    if "edges" in w.cfg:
        raise SystemExit("convergence runs take a single-volume workload")
    G = w.cfg["G"]
    tile = tuple(int(x) for x in args.tile.split("x"))
    launch = dict(tile=tile, ppt=args.ppt, group_lanes=args.gl, persistent=True, extent=G)
    builds = {"full": dict(), "isotropic": dict(ablation=vbm.BANK_ISOTROPIC),
              "unit_weight": dict(ablation=vbm.BANK_UNIT_WEIGHT), "haar": dict(wavelet=1)}
    inits = {}         # name -> (initial Gaussians, scene offsets)
    for name in args.variants.split(","):
        if name == "random":
            inits[name] = (torch.from_numpy(random_init(w.n, G)).to(device), w.scene_offset)
        elif name == "full":
            inits[name] = (w.params.clone(), w.scene_offset)
        else:
            wv = make_workload(args.config, device, **builds[name])
            inits[name] = (wv.params.clone(), wv.scene_offset)
    out = {"config": args.config, "gaussians": {k: int(v[0].shape[1]) for k, v in inits.items()},
           "views": int(w.targets.shape[0]), "steps": args.steps, "curves": {}}
    for name, (P, so) in inits.items():
        ft = FineTuner(P.contiguous(), w.cam_records, w.targets, scene_offset=so, view_scene=w.view_scene, **launch)
        concat = ConcatScore(ft, w, tile) if w.union_targets is not None else None
        curve = run(ft, args.steps, args.every, concat)
        ok, need, bad = ft.check()
        out["curves"][name] = [dict(zip(("step", "psnr", "ssim", "concat_psnr", "concat_ssim"), c)) for c in curve]
        out["curves"][name + "_pairs_ok"] = bool(ok)
        for c in curve:
            rec = {"init": name, "step": c[0], "psnr_db": round(c[1], 3), "ssim": round(c[2], 4)}
            if len(c) > 3:
                rec.update(concat_psnr_db=round(c[3], 3), concat_ssim=round(c[4], 4))
            print(json.dumps(rec), flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
