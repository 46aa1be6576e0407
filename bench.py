"""Benchmark of the VBM image-space fine-tuning step on GB300.

Workload (default "c1"): a 128^3 synthetic volume (32 random blobs plus
k^-2 band-limited noise), 3-level bior4.4 DWT, ~1e5 Gaussians built on the
GPU by vbm_build, 8 orbit views at 512x512 rendered by vbm_render_dvr as
targets.  One step = forward splatting of all views, L1 + D-SSIM loss,
backward to every Gaussian parameter, Adam (Sec. 4.4).

value      steps/s of the batched step (all views per launch, CUDA graph),
           device time from CUDA events, L2 flushed between steps
plain      steps/s of the same step run one view per launch sequence
e2e        steps/s through FineTuner.step_host: targets copied from pinned
           host memory every step, loss read back every step
roofline   the dominant kernel (forward or backward compositing) timed live
           with CUDA events recorded by the library on its launch stream
cpu_baseline  the FP64 oracle on the host, one view of the step (scaled)

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun with N > 1 every rank runs an independent replica (the step
has no cross-GPU exchange in this build); rank 0 prints the line.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fine-tune steps/sec (fwd+bwd, batched vs plain) on 1 GB300; raster Gpixel/s; %roofline"
FWD_FLOP_PER_PAIR = 20     # dx, dy, quadratic form, o*G, min, 1-a, T(1-a), a*T, 3 colour FMAs
BWD_FLOP_PER_PAIR = 60     # T recovery, colour and alpha partials, exponent chain, 9 partial sums
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c1")
    ap.add_argument("--plain-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default=None, help="WxH, skips the autotuner (with --ppt)")
    ap.add_argument("--ppt", type=int, default=1, help="pixels per thread with --tile")
    ap.add_argument("--persistent", action="store_true", help="persistent compositing kernels with --tile")
    ap.add_argument("--gl", type=int, default=32, help="lanes per compositing group with --tile (8, 16, 32)")
    ap.add_argument("--bwd-ppt", type=int, default=0, help="backward pixels per thread (0 = the forward's)")
    ap.add_argument("--bwd-gl", type=int, default=0, help="backward lanes per group (0 = the forward's)")
    ap.add_argument("--radix", action="store_true",
                    help="order the pairs by device radix sorts (items by depth, pairs by tile)")
    ap.add_argument("--seg", type=int, default=0,
                    help="list segment length of the persistent backward (0 = library default, -1 = never split)")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warmup + steps of the batched step without timing (for ncu captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ workload

def make_workload(cfg_key, device):
    """Volume(s) -> Gaussians (vbm_build) and DVR targets (vbm_render_dvr), all on the GPU."""
    from paper_2601_09417_gb300.workloads import make_workload as build
    return build(cfg_key, device)


def workload_extent(cfg):
    """Scene extent for the learning rate of the means (largest volume edge)."""
    return max(cfg["edges"]) if "edges" in cfg else cfg["G"]


# Fine-tuning steps run (with a fixed launch configuration) before the autotuner times its candidates.
TUNE_WARM_STEPS = 30

# Oracle timing window for workloads whose full view would take minutes on one core.
CPU_CROP = {"c4": 256}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- timing

def time_steps(fn, steps, flush):
    """Per-step CUDA-event times (ms) with an L2 flush before each step."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s, e in evs:
        flush()
        s.record()
        fn()
        e.record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in evs]


def kernel_source_hash():
    """Hash of the compositing kernels' code (raster.cu and vbm_internal.h with // comments
    and blank lines removed, so that a comment edit keeps a capture of unchanged code)."""
    h = hashlib.sha256()
    for name in ("raster.cu", "vbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2601_09417_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch from a committed ncu capture of the current kernel source, else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------- cpu baseline

def cpu_baseline(cfg, w, P_host, targets_host):
    """FP64 oracle on the host: one view of the step (projection, binning, compositing, loss,
    backward; a centred window of it for the largest workloads, scaled by pixel count) times
    the number of views, plus Adam over all Gaussians."""
    from oracle import adam as oadam
    from oracle import loss as oloss
    from oracle import raster as oraster
    from vbm_inputs.cameras import cameras_as_float32
    V = len(w.cams)
    so = [0, w.n] if w.scene_offset is None else [int(x) for x in w.scene_offset]
    s0 = 0 if w.view_scene is None else int(w.view_scene[0])
    P64 = P_host[:, so[s0]:so[s0 + 1]].astype(np.float64)
    cam = dict(cameras_as_float32(w.cams)[0])
    H, W = targets_host.shape[2], targets_host.shape[3]
    tgt = targets_host[:1].astype(np.float64)
    crop = CPU_CROP.get(cfg["key"])
    scale = 1.0
    if crop and crop < min(W, H):
        x0, y0 = (W - crop) // 2, (H - crop) // 2
        cam["cx"] -= x0
        cam["cy"] -= y0
        cam["width"] = cam["height"] = crop
        tgt = tgt[:, :, y0:y0 + crop, x0:x0 + crop]
        scale = (W * H) / float(crop * crop)
    t0 = time.perf_counter()
    fwd = oraster.splat_forward(P64, [cam])
    _, dimg = oloss.loss_and_grad(fwd["img"], tgt)
    dimg *= 1.0 / V
    oraster.splat_backward(fwd, P64, [cam], dimg)
    t_view = (time.perf_counter() - t0) * scale
    t1 = time.perf_counter()
    P_all = P_host.astype(np.float64)
    oadam.adam_step(P_all, np.zeros_like(P_all), np.zeros_like(P_all), np.zeros_like(P_all), 1,
                    oadam.default_lrs(workload_extent(cfg)))
    t_adam = time.perf_counter() - t1
    t_step = V * t_view + t_adam
    what = ("a %dx%d window of 1 of %d views (x%.0f for the full view)" % (crop, crop, V, scale)
            if scale != 1.0 else "1 of %d views" % V)
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": "%s (projection, binning, compositing, loss, backward) timed, x%d, plus Adam over all %d "
                      "Gaussians; %.2f s per view" % (what, V, P_host.shape[1], t_view)}


def _gpu_id(torch, device, local):
    """nvidia-smi id of the device (its UUID when torch reports one)."""
    uuid = str(getattr(torch.cuda.get_device_properties(device), "uuid", "") or "")
    if not uuid:
        return str(local)
    return uuid if uuid.startswith("GPU-") else "GPU-" + uuid


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the same workload, bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    device = torch.device("cuda", 0) if torch.cuda.is_available() else None
    if device is None:
        print(json.dumps({"impl": "reference", "unavailable": "workload inputs are built on the GPU"}))
        return
    torch.cuda.set_device(device)
    w = make_workload(args.config, device)
    cfg, n = w.cfg, w.n
    P = w.params.cpu().numpy()
    T = w.targets.cpu().numpy()
    vals = []
    for _ in range(max(1, min(args.steps, 3))):
        vals.append(cpu_baseline(cfg, w, P, T))
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": len(vals), "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "gaussians": int(n)},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------- main

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_2601_09417_gb300 import vbm
    from paper_2601_09417_gb300.finetune import FineTuner

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    vbm.load()

    w = make_workload(args.config, device)
    cfg, params, n, recs, cams, targets = w.cfg, w.params, w.n, w.cam_records, w.cams, w.targets
    V, H, W = targets.shape[0], targets.shape[2], targets.shape[3]
    batch = dict(scene_offset=w.scene_offset, view_scene=w.view_scene, extent=workload_extent(cfg),
                 recompute=bool(cfg.get("recompute", False)))
    if args.tile:
        tile, ppt, gl, pers = tuple(int(x) for x in args.tile.split("x")), args.ppt, args.gl, args.persistent
        seg = args.seg
        bppt, bgl = args.bwd_ppt, args.bwd_gl
        tune_table = []
    else:
        from paper_2601_09417_gb300.autotune import autotune
        # tune on the Gaussians as they are a few dozen steps into fine-tuning:
        # the first steps shrink the initial footprints, and the timed steps run
        # in that regime
        ftw = FineTuner(params.clone(), recs, targets, **batch, tile=(16, 16), ppt=1, group_lanes=16,
                        persistent=True)
        for _ in range(TUNE_WARM_STEPS):
            ftw.step_batched()
        torch.cuda.synchronize()
        (tile, ppt, gl, pers, seg, bppt, bgl), tune_table = autotune(ftw.params, recs, V, W, H, scene_offset=w.scene_offset,
                                                           view_scene=w.view_scene, recompute=batch["recompute"])
        del ftw
    if args.seg:
        seg = args.seg
    if args.bwd_ppt or args.bwd_gl:
        bppt, bgl = args.bwd_ppt, args.bwd_gl
    launch = dict(tile=tile, ppt=ppt, persistent=pers, group_lanes=gl, segment_len=seg, radix_sort=args.radix,
                  bwd_ppt=bppt, bwd_group_lanes=bgl)
    if args.profile_only:
        ftp = FineTuner(params, recs, targets, **batch, **launch)
        for _ in range(args.warmup + args.steps):
            ftp.step_batched()
        torch.cuda.synchronize()
        print(json.dumps({"profile_only": True, "tile": "%dx%d" % tile, "ppt": ppt, "group_lanes": gl,
                          "persistent": pers, "steps": args.steps}))
        return
    params0 = params.clone()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    def flush():
        flush_buf.fill_(1)

    # ---------------------------------------------------------- batched form
    ft = FineTuner(params0.clone(), recs, targets, **batch, **launch)
    # profiling hooks: events around the compositing kernels (recorded inside the
    # graph) and the per-pixel evaluated-entry count of every forward
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in kev:          # torch creates the underlying cudaEvent on the first record
        e.record()
    torch.cuda.synchronize()
    n_eval = torch.zeros((V, H, W), dtype=torch.int32, device=device)
    bufs = ft.plan.buffers()
    if bufs.n_contrib:
        ft.plan.set_profile(kev, n_eval)
        n_contrib = vbm.device_tensor(bufs.n_contrib, (V, H, W), np.int32)
    else:   # recompute mode keeps no contributor counts: the profiling hook writes them
        n_contrib = torch.zeros((V, H, W), dtype=torch.int32, device=device)
        ft.plan.set_profile(kev, n_eval, n_contrib)
    n_pairs_dev = vbm.device_tensor(bufs.n_pairs, (1,), np.int64)
    ft.capture()
    for _ in range(args.warmup):
        ft.step_graph()
    torch.cuda.synchronize()
    ok, need, bad = ft.check()
    if not ok:
        raise RuntimeError("pair capacity too small: %d needed" % need)
    launches0 = vbm.kernel_launches()
    ft.step_batched()
    torch.cuda.synchronize()
    launches_per_step = vbm.kernel_launches() - launches0

    clocks = ClockSampler(_gpu_id(torch, device, local))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms, fwd_ms, bwd_ms, p_fwd, p_bwd, pairs = [], [], [], 0, 0, []
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush()
        s_ev.record()
        ft.step_graph()
        e_ev.record()
        e_ev.synchronize()
        step_ms.append(s_ev.elapsed_time(e_ev))
        fwd_ms.append(kev[0].elapsed_time(kev[1]))
        bwd_ms.append(kev[2].elapsed_time(kev[3]))
        p_fwd += int(n_eval.sum().item())
        p_bwd += int(n_contrib.sum().item())
        pairs.append(int(n_pairs_dev.item()))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    from paper_2601_09417_gb300.replicas import job_rate
    total_ms, value = job_rate(sum(step_ms), args.steps, device)
    ms_per_step = total_ms / args.steps
    ok, need, bad = ft.check()

    # forward alone (projection, binning, sort, compositing) and forward + loss +
    # backward, all views in one call each, no graph: the Gpixel/s figures
    def fwd_only():
        ft.plan.forward(ft.params, ft.cams, ft.img, bg=ft.bg)

    def fwd_bwd():
        ft.plan.forward(ft.params, ft.cams, ft.img, bg=ft.bg)
        vbm.loss(ft.img, ft.targets, V, H, W, ft.lam, ft.scale, ft.loss, ft.dimg, ft.ws)
        ft.plan.backward(ft.params, ft.cams, ft.dimg, ft.grad, bg=ft.bg)
    n_px = min(args.steps, 100)
    fo = time_steps(fwd_only, n_px, flush)
    fb = time_steps(fwd_bwd, n_px, flush)
    del ft

    # ------------------------------------------ plain form: one view per launch
    # sequence, default tile settings, no graph; same initial state and steps
    plain_steps = args.plain_steps if args.plain_steps is not None else args.steps
    ftp = FineTuner(params0.clone(), recs, targets, **batch)
    for _ in range(args.warmup):
        ftp.step_plain()
    plain = time_steps(ftp.step_plain, plain_steps, flush)
    plain_ms = sum(plain) / len(plain)
    del ftp

    # ------------------------------------------------------------ end to end
    fte = FineTuner(params0.clone(), recs, targets, **batch, **launch)
    host_t = torch.empty(targets.shape, dtype=torch.float32, pin_memory=True)
    host_t.copy_(targets)
    host_l = torch.empty(1, dtype=torch.float64, pin_memory=True)
    fte.capture_host(host_t, host_l)
    for _ in range(args.warmup):
        fte.step_host(host_t, host_l)
    e2e = time_steps(lambda: fte.step_host(host_t, host_l), args.steps, flush)
    e2e_ms = sum(e2e) / len(e2e)
    del fte

    # --------------------------------------- forward-only frames (single view)
    fwd_only = None
    if cfg.get("fwd_only") and w.scene_offset is None:
        from vbm_inputs import orbit_cameras
        from vbm_inputs.cameras import camera_array
        fw, fh = cfg["fwd_only"]
        cams1 = orbit_cameras((cfg["G"],) * 3, 1, fw, fh)
        cd1 = vbm.cameras_to_device(camera_array(cams1), device)
        plan1 = vbm.Plan([0, n], 1, fw, fh, tile_w=tile[0], tile_h=tile[1], pixels_per_thread=ppt, group_lanes=gl,
                         flags=vbm.PLAN_PERSISTENT if pers else 0, pair_capacity=vbm.default_pair_capacity(n))
        img1 = torch.zeros((1, 3, fh, fw), device=device)

        def frame():
            plan1.forward(params0, cd1, img1)
        for _ in range(max(3, args.warmup)):
            frame()
        fo_ms = time_steps(frame, min(args.steps, 100), flush)
        ok1, need1 = plan1.check()
        fwd_only = {"image": "%dx%d" % (fw, fh), "frames_per_s": 1e3 / float(np.median(fo_ms)),
                    "ms_per_frame": float(np.median(fo_ms)), "pairs_ok": bool(ok1),
                    "form": "projection + binning + sort + compositing of one view, one call"}
        plan1.close()

    # ------------------------------------------------------------- roofline
    f_fwd = sum(fwd_ms) / len(fwd_ms)
    f_bwd = sum(bwd_ms) / len(bwd_ms)
    peak_tflops = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    if f_bwd >= f_fwd:
        kname, flops, kms = "raster_bwd", p_bwd * BWD_FLOP_PER_PAIR, sum(bwd_ms)
    else:
        kname, flops, kms = "raster_fwd", p_fwd * FWD_FLOP_PER_PAIR, sum(fwd_ms)
    achieved = flops / (kms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": profiled_traffic(kname), "kernel": kname,
                "kernel_ms": kms / args.steps, "fwd_kernel_ms": f_fwd, "bwd_kernel_ms": f_bwd,
                "pairs_fwd_per_step": p_fwd / args.steps, "pairs_bwd_per_step": p_bwd / args.steps,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP (FMA) x 2070 MHz max SM clock",
                "flop_per_pair": {"fwd": FWD_FLOP_PER_PAIR, "bwd": BWD_FLOP_PER_PAIR}}
    n_pairs = int(np.mean(pairs))

    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["workload"], "gaussians": int(n), "views": V, "image": "%dx%d" % (W, H),
                       "tile": "%dx%d" % tile, "pixels_per_thread": ppt, "group_lanes": gl, "persistent": pers,
                       "segment_len": (seg if seg else 256) if pers else None,
                       "bwd_pixels_per_thread": bppt or ppt, "bwd_group_lanes": bgl or gl,
                       "pair_order": "device radix sorts" if args.radix else "bucketed per-tile sort",
                       "compositing_state": "recomputed in the backward" if batch["recompute"] else "stored",
                       "pairs_mean": n_pairs,
                       "form": "batched, CUDA graph, autotuned",
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "plain": {"value": 1e3 / plain_ms, "unit": "steps/s", "ms_per_step": plain_ms,
                      "form": "one view per launch sequence, no graph, 16x16 tiles, default settings"},
            "autotune": {"candidates": len(tune_table),
                         "fastest": [{"tile": "%dx%d" % tuple(r["tile"]), "ppt": r["ppt"],
                                      "group_lanes": r["group_lanes"], "persistent": r["persistent"],
                                      "ms_fwd_bwd": r["ms"], "ms_fwd": r.get("ms_fwd"), "ms_bwd": r.get("ms_bwd")}
                                     for r in sorted((r for r in tune_table if r.get("stage") is None),
                                                     key=lambda r: r["ms"])[:6]],
                         "pairs_retimed": [{"tile": "%dx%d" % tuple(r["tile"]), "fwd": [r["ppt"], r["group_lanes"]],
                                            "bwd": [r["bwd_ppt"], r["bwd_group_lanes"]], "persistent": r["persistent"],
                                            "ms_estimate": r["ms"], "ms_fwd_bwd_retimed": r["ms_final"]}
                                           for r in tune_table if r.get("stage") == "combination"],
                         "segment_len": [{"segment_len": r["segment_len"], "ms_fwd_bwd": r["ms"]}
                                         for r in tune_table if r.get("stage") == "segment"],

                         "tuned_after_steps": TUNE_WARM_STEPS if tune_table else 0},
            "batched_over_plain": plain_ms / ms_per_step,
            "step_ms_percentiles": {"p10": float(np.percentile(step_ms, 10)),
                                    "p50": float(np.percentile(step_ms, 50)),
                                    "p90": float(np.percentile(step_ms, 90))},
            "gpixel_per_s": {"fwd": V * H * W / (float(np.median(fo)) * 1e-3) / 1e9,
                             "fwd_loss_bwd": V * H * W / (float(np.median(fb)) * 1e-3) / 1e9,
                             "raster_fwd_kernel": V * H * W / (f_fwd * 1e-3) / 1e9,
                             "note": "fwd = projection + binning + sort + compositing of all views, one call, "
                                     "median of %d; raster_fwd_kernel = the compositing kernel alone" % n_px},
            "e2e": {"value": 1e3 / e2e_ms, "unit": "steps/s", "h2d_bytes_per_step": int(targets.numel() * 4),
                    "d2h_bytes_per_step": 8},
            "roofline": roofline, "gpu_launches": int(launches_per_step * args.steps),
            "wall_s_timed": wall}
    if fwd_only is not None:
        line["fwd_only"] = fwd_only
    if clk is not None:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, w, params0.cpu().numpy(), targets.cpu().numpy())
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
