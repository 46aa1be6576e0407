"""Benchmark of the VBM image-space fine-tuning step on GB300.

Workload (default "c4", the largest that fits one GPU): a 512^3 supernova-like
synthetic volume (5 noisy concentric shells and a dense core), 5-level
bior4.4 DWT, ~2.9e6 Gaussians built on the GPU by vbm_build, 8 orbit views at
1024x1024 rendered by vbm_render_dvr as targets, per-pixel compositing state
recomputed in the backward.  One step = forward splatting of all views,
L1 + D-SSIM loss, backward to every Gaussian parameter, Adam (Sec. 4.4).

value      steps/s of the batched step (all views per launch, CUDA graph),
           device time from CUDA events, L2 flushed between steps
plain      steps/s of the same step run one view per launch sequence
e2e        steps/s through FineTuner.step_host on the host clock: every step
           copies its targets from pinned host memory and the host reads the
           loss back before the next step starts
fwd_only   frames/s of the forward alone at 1920x1080 (one view, one call)
roofline   the dominant kernel (backward compositing) against the FP32 peak
           measured in this run by vbm_peak_probe; `kernels` lists every
           kernel group of the step with its time (CUDA events recorded by
           the library on its launch stream) and its algorithmic lower bound
           (FP32, ex2 or HBM); step_frac = sum of the lower bounds / step time
cpu_baseline  the FP64 oracle on the host cores: every view's sample in its
           own process (spawn pool), extrapolated to the full step as stated
           in the line, plus the one-thread figure

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config cN]
Under torchrun with N > 1 every rank runs an independent replica (the step
has no cross-GPU exchange in this build); rank 0 prints the line.
"""

import argparse
import atexit
import hashlib
import json
import math
import multiprocessing
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fine-tune steps/sec (fwd+bwd, batched vs plain) on 1 GB300; raster Gpixel/s; %roofline"
DEFAULT_CONFIG = "c4"
FWD_FLOP_PER_PAIR = 20     # dx, dy, quadratic form, o*G, min, 1-a, T(1-a), a*T, 3 colour FMAs
BWD_FLOP_PER_PAIR = 60     # T recovery, colour and alpha partials, exponent chain, 9 partial sums
BWD_SFU_PER_PAIR = 2       # ex2 of the exponent, rcp of (1 - alpha)
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--plain-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default=None, help="WxH, skips the autotuner (with --ppt)")
    ap.add_argument("--ppt", type=int, default=1, help="pixels per thread with --tile")
    ap.add_argument("--persistent", action="store_true", help="persistent compositing kernels with --tile")
    ap.add_argument("--gl", type=int, default=32, help="lanes per compositing group with --tile (4, 8, 16, 32)")
    ap.add_argument("--bwd-ppt", type=int, default=0, help="backward pixels per thread (0 = the forward's)")
    ap.add_argument("--bwd-gl", type=int, default=0, help="backward lanes per group (0 = the forward's)")
    ap.add_argument("--radix", action="store_true",
                    help="order the pairs by device radix sorts (items by depth, pairs by tile)")
    ap.add_argument("--seg", type=int, default=0,
                    help="list segment length of the persistent backward (0 = library default, -1 = never split)")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warmup + steps of the batched step without timing (for ncu captures)")
    ap.add_argument("--views", type=int, default=0,
                    help="use only the first N views of a single-volume workload (smaller ncu cases)")
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

# Oracle sample per view: a centred window of this many pixels per side (None = the whole view).
CPU_WINDOW = {"c2": 200, "c4": 128}
REF_WINDOW = {"c2": 100, "c4": 64}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 50 ms, each stamped with the host
    clock when it arrives; started ahead of the timed region (nvidia-smi takes a moment to
    produce its first line), and summarised over the lines that arrived between mark_begin()
    and mark_end()."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index, interval_ms=50):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []             # (host time, line)
        self.reader = None
        self.t0 = self.t1 = None

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def read(stream):
            for line in stream:
                self.lines.append((time.perf_counter(), line))
        self.reader = threading.Thread(target=read, args=(self.proc.stdout,), daemon=True)
        self.reader.start()
        atexit.register(self._end_process)

    def _end_process(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()

    def wait_first(self, timeout_s=5.0):
        """Blocks until the first sample has arrived (or the timeout passes)."""
        t_end = time.perf_counter() + timeout_s
        while self.proc is not None and not self.lines and time.perf_counter() < t_end:
            time.sleep(0.01)

    def mark_begin(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader is not None:
            self.reader.join(timeout=5)
        return self.summarise(self.lines, self.t0, self.t1)

    @classmethod
    def summarise(cls, lines, t0=None, t1=None):
        """Median SM clock, the largest maximum clock and the active throttle reasons of the
        samples stamped within [t0, t1] (all samples where a bound is None)."""
        sm, mx, reasons = [], [], set()
        for t, line in lines:
            if (t0 is not None and t < t0) or (t1 is not None and t > t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(cls.NAMES, parts[3:7]):
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


def measured_peaks(device):
    """FP32 FMA, FP32x2 FMA and ex2 rates of this GPU from vbm_peak_probe (best of 5 CUDA-event
    timed launches of one wave-filling grid each), and the HBM copy bandwidth measured by the
    pool's driver (MEASURED_PEAKS.json) or, without that file, by a 1 GiB device copy here."""
    import torch
    from paper_2601_09417_gb300 import vbm
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = sms * 8
    out = torch.zeros(blocks * 256, device=device)
    res = {}
    for kind, name, iters in ((0, "fp32_fma_tflops", 32768), (1, "fp32x2_fma_tflops", 32768),
                              (2, "ex2_tera_per_s", 4096)):
        vbm.peak_probe(kind, blocks, iters, out)            # warm-up
        best = None
        for _ in range(5):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            ops = vbm.peak_probe(kind, blocks, iters, out)
            e.record()
            e.synchronize()
            rate = ops / (s.elapsed_time(e) * 1e-3) / 1e12
            best = rate if best is None else max(best, rate)
        res[name] = best
    res["fp32_tflops"] = max(res["fp32_fma_tflops"], res["fp32x2_fma_tflops"])
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = None
    try:
        with open(path) as f:
            hbm = float(json.load(f)["hbm_gbs"])
        res["hbm_source"] = "MEASURED_PEAKS.json (STREAM-style copy, driver-measured on this pool)"
    except (OSError, ValueError, KeyError):
        a = torch.empty(1 << 30, dtype=torch.uint8, device=device)
        b = torch.empty_like(a)
        best = 0.0
        for _ in range(6):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            b.copy_(a)
            e.record()
            e.synchronize()
            best = max(best, 2 * a.numel() / (s.elapsed_time(e) * 1e-3) / 1e9)
        hbm = best
        res["hbm_source"] = "measured here: 1 GiB device copy, read + write bytes, best of 6"
        del a, b
    res["hbm_gbs"] = hbm
    res["derived_fp32_tflops"] = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    res["probe"] = ("vbm_peak_probe: %d blocks x 256 threads x 8 independent chains, CUDA events, best of 5"
                    % blocks)
    return res


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


def profiled_traffic(kernel, workload_key):
    """DRAM bytes per launch from a committed ncu capture of the current kernel source on this
    workload, else None (with the reason)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, "no profiles/traffic.json"
    ent = rec.get(kernel, {}).get(workload_key)
    if not ent:
        return None, "no capture of %s on %s" % (kernel, workload_key)
    if ent.get("source_hash") != kernel_source_hash():
        return None, "kernel changed since the capture"
    return ent.get("dram_bytes_per_launch"), ent.get("note", "")


# ------------------------------------------------------- algorithmic work

def step_work(N, items, V, HW, n_dup, p_fwd, p_bwd, recompute, fused_adam=False):
    """Algorithmic work per step of each kernel group (FP32 FLOP, ex2/rcp evaluations, HBM bytes),
    the counts of the method itself (N Gaussians, `items` (view, Gaussian) pairs (N V for one
    scene; each view its own scene's Gaussians in a batch of scenes), V views of HW pixels,
    n_dup (view, tile, Gaussian) pairs, p_fwd / p_bwd evaluated pairs) and not of this
    implementation.  fused_adam: the projection backward and Adam as one group, which reads
    the splat gradients, the parameters once and the two moments, and writes the parameters
    and moments (no gradient array)."""
    px = V * HW
    state = 0 if recompute else 8                      # T_final and the last contributor per pixel
    work = {
        "projection": dict(flop=250 * items, sfu=0, bytes=N * 56 + items * 40),
        "binning_sort": dict(flop=0, sfu=0, bytes=items * 8 + n_dup * 12 + n_dup * 12 * 2 + n_dup * 8),
        "raster_fwd": dict(flop=FWD_FLOP_PER_PAIR * p_fwd, sfu=p_fwd, bytes=n_dup * 40 + px * (12 + state)),
        # SSIM: two separable 11-tap passes (2 FLOP per tap) over the 5 moment maps forward and the 3
        # gradient maps backward, plus about 40 FLOP of per-element algebra
        "loss": dict(flop=px * 3 * (2 * 11 * 2 * (5 + 3) + 40), sfu=0, bytes=px * 3 * 4 * 3),
        "raster_bwd": dict(flop=BWD_FLOP_PER_PAIR * p_bwd, sfu=BWD_SFU_PER_PAIR * p_bwd,
                           bytes=n_dup * 40 + px * (12 + 12 + state) + n_dup * 36),
        "projection_bwd": dict(flop=400 * items, sfu=0, bytes=items * 36 + N * 56),
        "adam": dict(flop=0, sfu=0, bytes=14 * N * 28),
    }
    if fused_adam:
        del work["projection_bwd"], work["adam"]
        work["projection_bwd_adam"] = dict(flop=400 * items, sfu=0, bytes=items * 36 + N * 56 * 6)
    return work


def lower_bound_ms(w, peaks):
    """max(FLOP / FP32 peak, ex2 / SFU peak, bytes / HBM peak) in ms, and which one binds."""
    t = {"alu": w["flop"] / (peaks["fp32_tflops"] * 1e12),
         "sfu": w["sfu"] / (peaks["ex2_tera_per_s"] * 1e12),
         "hbm": w["bytes"] / (peaks["hbm_gbs"] * 1e9)}
    bound = max(t, key=t.get)
    return t[bound] * 1e3, bound


# ------------------------------------------------------------- cpu baseline

def _window_camera(cam, window):
    """The camera of a centred window (w, h) of cam's image: principal point shifted."""
    c = dict(cam)
    if window is None:
        return c, (0, 0, cam["width"], cam["height"])
    w = min(window, cam["width"])
    h = min(window, cam["height"])
    x0, y0 = (cam["width"] - w) // 2, (cam["height"] - h) // 2
    c["cx"] -= x0
    c["cy"] -= y0
    c["width"], c["height"] = w, h
    return c, (x0, y0, w, h)


_WORKER_P = None


def _oracle_worker_init(p_path):
    """Spawned oracle worker: loads the Gaussians once (FP64 P[14][N])."""
    global _WORKER_P
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    _WORKER_P = np.ascontiguousarray(np.load(p_path), dtype=np.float64)


def _oracle_view_sample(job):
    """One view's share of the step by the FP64 oracle, on a window of the view: projection of
    all N Gaussians, binning, compositing, L1 + D-SSIM loss, backward and projection backward,
    each phase timed (oracle.raster's per-phase timings)."""
    from oracle import loss as oloss
    from oracle import raster as oraster
    cam, target = job["cam"], job["target"]
    tm = {}
    t0 = time.perf_counter()
    fwd = oraster.splat_forward(_WORKER_P, [cam], timings=tm)
    t1 = time.perf_counter()
    _, dimg = oloss.loss_and_grad(fwd["img"], target)
    tm["loss"] = time.perf_counter() - t1
    dimg *= job["loss_scale"]
    oraster.splat_backward(fwd, _WORKER_P, [cam], dimg, timings=tm)
    tm["total"] = time.perf_counter() - t0
    tm["pairs"] = int(fwd["items"].size)
    tm["view"] = job["view"]
    return tm


def _extrapolate_view(tm, pairs_view, pixel_ratio):
    """Full-view seconds from a window's phases: projection, binning and projection backward
    run over all N items whatever the window (taken as measured, so binning's per-pair part is
    not scaled); compositing forward and backward scale with the view's pairs over the
    window's; the loss with the pixels."""
    pr = pairs_view / max(1, tm["pairs"])
    return (tm["project"] + tm["bin_sort"] + tm["project_bwd"] + (tm["render"] + tm["render_bwd"]) * pr
            + tm["loss"] * pixel_ratio)


class OracleSampler:
    """A spawn pool of min(V, cpu) oracle processes holding the Gaussians; each run times one
    window sample of every view (view v in its own process)."""

    def __init__(self, P64, cams, targets, window, pairs_view):
        self.V = len(cams)
        self.workers = max(1, min(self.V, os.cpu_count() or 1))
        fd, self.p_path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        np.save(self.p_path, np.ascontiguousarray(P64, dtype=np.float64))
        self.N = P64.shape[1]
        self.jobs = []
        W, H = cams[0]["width"], cams[0]["height"]
        for v, cam in enumerate(cams):
            c, (x0, y0, w, h) = _window_camera(cam, window)
            self.jobs.append(dict(view=v, cam=c, target=np.ascontiguousarray(targets[v][:, y0:y0 + h, x0:x0 + w],
                                                                              dtype=np.float64)[None],
                                  loss_scale=(w * h) / float(self.V * W * H)))
        self.win = (self.jobs[0]["cam"]["width"], self.jobs[0]["cam"]["height"])
        self.pixel_ratio = (W * H) / float(self.win[0] * self.win[1])
        self.pairs_view = [int(x) for x in pairs_view]
        ctx = multiprocessing.get_context("spawn")
        self.pool = ctx.Pool(self.workers, initializer=_oracle_worker_init, initargs=(self.p_path,))

    def run(self):
        """One sample: wall seconds, per-view extrapolated full-view seconds, raw phases."""
        t0 = time.perf_counter()
        res = sorted(self.pool.map(_oracle_view_sample, self.jobs, chunksize=1), key=lambda r: r["view"])
        wall = time.perf_counter() - t0
        per_view = [_extrapolate_view(r, self.pairs_view[r["view"]], self.pixel_ratio) for r in res]
        return wall, per_view, res

    def adam_seconds(self, extent):
        from oracle import adam as oadam
        P = np.load(self.p_path)
        t0 = time.perf_counter()
        oadam.adam_step(P, np.zeros_like(P), np.zeros_like(P), np.zeros_like(P), 1, oadam.default_lrs(extent))
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        try:
            os.remove(self.p_path)
        except OSError:
            pass


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def baseline_record(sampler, per_view, wall, t_adam, window_label):
    """cpu_baseline object from one sample run."""
    V = sampler.V
    rounds = math.ceil(V / sampler.workers)
    t_step = rounds * max(per_view) + t_adam
    t_step_1 = sum(per_view) + t_adam
    return {"value": 1.0 / t_step, "unit": "steps/s", "cores": sampler.workers, "kind": "oracle",
            "value_1_thread": 1.0 / t_step_1, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": ("FP64 oracle, one process per view (%d processes, spawn pool): a centred %dx%d window of each "
                       "of the %d views (projection of all %d Gaussians, binning, compositing, loss, backward, "
                       "projection backward), %.1f s wall; full view extrapolated per view: projection, binning "
                       "and projection backward as measured, compositing forward/backward scaled by the view's "
                       "pair count over the window's, loss by pixels (%s); step = slowest view x %d + Adam over all "
                       "Gaussians (%.2f s); value_1_thread = the sum of the per-view seconds + Adam (each view "
                       "measured in its own process on its own core)"
                       % (sampler.workers, sampler.win[0], sampler.win[1], V, sampler.N, wall, window_label, rounds,
                          t_adam)),
            "s_per_view": [round(x, 3) for x in per_view]}


def _gpu_id(torch, device, local):
    """nvidia-smi id of the device (its UUID when torch reports one)."""
    uuid = str(getattr(torch.cuda.get_device_properties(device), "uuid", "") or "")
    if not uuid:
        return str(local)
    return uuid if uuid.startswith("GPU-") else "GPU-" + uuid


# ------------------------------------------------------------- reference arm

def _oracle_inputs(cfg):
    """The workload's Gaussians (FP64 P[14][N]) and per-view pair counts, its cameras and DVR
    target windows, built by the oracle alone (no GPU, no libvbm): TF, DWT (the four RGBA
    channels in threads), budget and MAD selection, the bank, the coefficient map; pair
    counts from the oracle's projection of each full view."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import dvr as odvr
    from oracle import raster as oraster
    from oracle.bank import build_bank
    from oracle.dwt import dwt3d
    from oracle.filters import filter_bank
    from oracle.mapping import map_coefficients, select_all
    from oracle.tf import apply_tf_vectorised
    from vbm_inputs import TF_KNOTS_RGBA, TF_KNOTS_X, orbit_cameras, volume_for_config
    from vbm_inputs.cameras import cameras_as_float32
    if "edges" in cfg or "modes" in cfg:
        raise ValueError("the reference arm builds single-volume workloads")
    F = volume_for_config(cfg).astype(np.float64)
    J = cfg["levels"]
    x32 = TF_KNOTS_X.astype(np.float32).astype(np.float64)
    rgba32 = TF_KNOTS_RGBA.astype(np.float32).astype(np.float64)
    RF = apply_tf_vectorised(F, x32, rgba32)
    fb = filter_bank(0)
    with ThreadPoolExecutor(5) as ex:
        bank_f = ex.submit(build_bank, J)
        chans = list(ex.map(lambda c: dwt3d(np.ascontiguousarray(RF[..., c]), J, fb), range(4)))
        bank = bank_f.result()
    del RF
    A = np.stack(chans)
    del chans
    masks, _, _, _ = select_all(A, J, cfg["K_tot"])
    P = map_coefficients(A, masks, J, bank)
    del A
    cams = cameras_as_float32(orbit_cameras(F.shape[::-1], cfg["views"], cfg["width"], cfg["height"]))
    n = P.shape[1]
    pairs_view = [int(oraster.project(P, c, np.arange(n), 16, 16)[:, 12].sum()) for c in cams]
    window = REF_WINDOW.get(cfg["key"])
    targets = []
    for c in cams:
        wc, (x0, y0, w, h) = _window_camera(c, window)
        jj, ii = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
        pix = np.stack([ii.reshape(-1), jj.reshape(-1)], 1)
        rgba = odvr.render_dvr(F.astype(np.float64), x32, rgba32, c, step=0.5, pixels=pix)
        img = np.zeros((3, c["height"], c["width"]))
        img[:, y0:y0 + h, x0:x0 + w] = rgba[:3].reshape(3, h, w)
        targets.append(img)
    return P, cams, targets, pairs_view, window


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the same workload, built and timed without the GPU.
    Each step is one bounded sample (a window of every view, one process per view); the line's
    ms_per_step is that sample's wall time, its value the full-step rate extrapolated from it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from vbm_inputs import config
    cfg = config(args.config)
    t0 = time.perf_counter()
    P, cams, targets, pairs_view, window = _oracle_inputs(cfg)
    t_build = time.perf_counter() - t0
    sampler = OracleSampler(P, cams, targets, window, pairs_view)
    try:
        for _ in range(args.warmup):
            sampler.run()
        walls, rates, recs = [], [], []
        t_adam = sampler.adam_seconds(workload_extent(cfg))
        for _ in range(args.steps):
            wall, per_view, _ = sampler.run()
            walls.append(wall)
            rec = baseline_record(sampler, per_view, wall, t_adam,
                                  "whole view, nothing extrapolated" if window is None else "window %d" % window)
            rates.append(rec["value"])
            recs.append(rec)
    finally:
        sampler.close()
    v = statistics.median(rates)
    ms = 1e3 * statistics.median(walls)
    rec = recs[len(recs) // 2]
    rec["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "gaussians": int(P.shape[1]),
                       "inputs": "built by the FP64 oracle on the host (no GPU): %.0f s" % t_build},
            "note": ("each timed step is one bounded sample of the workload (a %s window of every view); "
                     "ms_per_step is that sample's wall time, value the full-step rate extrapolated from it "
                     "(cpu_baseline.sample)" % ("%dx%d" % sampler.win)),
            "cpu_baseline": rec,
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
    if args.views:
        if w.scene_offset is not None:
            raise ValueError("--views applies to single-volume workloads")
        w.cam_records, w.cams = w.cam_records[:args.views], w.cams[:args.views]
        w.targets = w.targets[:args.views].contiguous()
        w.cfg = dict(w.cfg, views=args.views, workload=w.cfg["workload"] + " (first %d views)" % args.views)
    torch.cuda.empty_cache()    # the build's workspace, kept by torch's caching allocator
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

    peaks = measured_peaks(device)

    # ---------------------------------------------------------- batched form
    ft = FineTuner(params0.clone(), recs, targets, **batch, **launch)
    # profiling hooks: events at the kernel-group boundaries (recorded by the
    # library inside the graph, on its launch stream) and the per-pixel
    # evaluated-entry count of every forward
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    for e in kev:          # torch creates the underlying cudaEvent on the first record
        e.record()
    torch.cuda.synchronize()
    n_eval = torch.zeros((V, H, W), dtype=torch.int32, device=device)
    bufs = ft.plan.buffers()
    own_contrib = bool(bufs.n_contrib)
    n_contrib = (vbm.device_tensor(bufs.n_contrib, (V, H, W), np.int32) if own_contrib else
                 torch.zeros((V, H, W), dtype=torch.int32, device=device))

    def count_pairs():
        """(P_fwd, P_bwd) of the current Gaussians: one untimed forward with the per-pixel
        count hooks set (recompute plans keep no contributor counts: the hook writes them);
        the timed graph runs without them, and the timed steps are synchronised one by one,
        so a count between two of them is outside the timed intervals."""
        ft.plan.set_profile(None, n_eval, None if own_contrib else n_contrib)
        ft.plan.forward(ft.params, ft.cams, ft.img, bg=ft.bg)
        torch.cuda.synchronize()
        counts = int(n_eval.sum().item()), int(n_contrib.sum().item())
        ft.plan.set_profile(kev)
        return counts
    ft.plan.set_profile(kev)
    n_pairs_dev = vbm.device_tensor(bufs.n_pairs, (1,), np.int64)
    ft.capture()
    clocks = ClockSampler(_gpu_id(torch, device, local))
    clocks.start()
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
    extra_steps = 1        # the launch-count step above

    clocks.wait_first()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark_begin()
    t_wall0 = time.perf_counter()
    # the backward's end event follows Adam when the two are fused
    fused_adam = ft.fused_adam
    groups = ("head", "projection", "binning_sort", "raster_fwd", "loss", "raster_bwd") + \
        (("projection_bwd_adam",) if fused_adam else ("projection_bwd", "adam"))
    step_ms, grp_ms, pairs, counts = [], {g: [] for g in groups}, [], []
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    count_every = max(1, args.steps // 8)
    for i in range(args.steps):
        if i % count_every == 0:    # untimed: the pair counts of the state the next step sees
            counts.append(count_pairs())
        flush()
        s_ev.record()
        ft.step_graph()
        e_ev.record()
        e_ev.synchronize()
        step_ms.append(s_ev.elapsed_time(e_ev))
        marks = [s_ev, kev[4], kev[5], kev[0], kev[1], kev[2], kev[3]] + ([] if fused_adam else [kev[6]]) + [e_ev]
        for g, a, b in zip(groups, marks[:-1], marks[1:]):
            grp_ms[g].append(a.elapsed_time(b))
        pairs.append(int(n_pairs_dev.item()))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clocks.mark_end()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    from paper_2601_09417_gb300.replicas import job_rate
    total_ms, value = job_rate(sum(step_ms), args.steps, device)
    ms_per_step = total_ms / args.steps
    ok, need, bad = ft.check()
    counts.append(count_pairs())
    # evaluated and contributing pairs per step: the mean of the counts sampled
    # through the timed window
    p_fwd_step = float(np.mean([c[0] for c in counts]))
    p_bwd_step = float(np.mean([c[1] for c in counts]))
    state_ms = {g: float(np.median(grp_ms[g])) for g in groups}

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
    ft.plan.set_profile()
    # pairs per view of the built Gaussians (the oracle baseline's state, for its
    # extrapolation): the entries of each view's tile ranges after one forward
    ft.plan.forward(params0, ft.cams, ft.img, bg=ft.bg)
    TXY = ((W + tile[0] - 1) // tile[0]) * ((H + tile[1] - 1) // tile[1])
    rng_host = vbm.device_tensor(bufs.ranges, (V * TXY, 2), np.int32).cpu().numpy()
    pairs_view = [int((rng_host[v * TXY:(v + 1) * TXY, 1] - rng_host[v * TXY:(v + 1) * TXY, 0]).sum())
                  for v in range(V)]
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
    # host clock: flush L2 and drain the stream (untimed), then time the step
    # from its launch through the host's read of the loss copied back
    fte = FineTuner(params0.clone(), recs, targets, **batch, **launch)
    host_t = torch.empty(targets.shape, dtype=torch.float32, pin_memory=True)
    host_t.copy_(targets)
    host_l = torch.empty(1, dtype=torch.float64, pin_memory=True)
    fte.capture_host(host_t, host_l)
    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        fte.step_host(host_t, host_l)
    stream.synchronize()
    e2e_s, losses = [], []
    for _ in range(args.steps):
        flush()
        stream.synchronize()
        t0 = time.perf_counter()
        fte.step_host(host_t, host_l)
        stream.synchronize()
        losses.append(float(host_l[0]))
        e2e_s.append(time.perf_counter() - t0)
    e2e_ms = 1e3 * sum(e2e_s) / len(e2e_s)
    del fte

    # --------------------------------------- forward-only frames (single view)
    fwd_only_rec = None
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
        fwd_only_rec = {"image": "%dx%d" % (fw, fh), "frames_per_s": 1e3 / float(np.median(fo_ms)),
                        "ms_per_frame": float(np.median(fo_ms)), "pairs_ok": bool(ok1),
                        "gaussians": int(n),
                        "form": "projection + binning + sort + compositing of one view, one call, the initial "
                                "Gaussians, L2 flushed before each frame"}
        plan1.close()

    # ------------------------------------------------------------- roofline
    n_pairs = float(np.mean(pairs))
    n_items = vbm.batch_items([0, n] if w.scene_offset is None else w.scene_offset, V, w.view_scene)
    work = step_work(n, n_items, V, H * W, n_pairs, p_fwd_step, p_bwd_step, batch["recompute"],
                     fused_adam=fused_adam)
    kernels, lb_sum = {}, 0.0
    for g in groups[1:]:
        lb, bound = lower_bound_ms(work[g], peaks)
        t = state_ms[g]
        rec = {"ms": t, "lower_bound_ms": lb, "bound": bound, "frac": lb / t if t > 0 else None,
               "hbm_gbs": work[g]["bytes"] / (t * 1e-3) / 1e9 if t > 0 else None,
               "hbm_frac": work[g]["bytes"] / (t * 1e-3) / 1e9 / peaks["hbm_gbs"] if t > 0 else None,
               "algorithmic_bytes": work[g]["bytes"]}
        if work[g]["flop"]:
            rec["tflops"] = work[g]["flop"] / (t * 1e-3) / 1e12 if t > 0 else None
        kernels[g] = rec
        lb_sum += lb
    t_bwd, t_fwd = state_ms["raster_bwd"], state_ms["raster_fwd"]
    kname = "raster_bwd" if t_bwd >= t_fwd else "raster_fwd"
    flops = work[kname]["flop"]
    achieved = flops / (state_ms[kname] * 1e-3) / 1e12
    traffic, traffic_note = profiled_traffic(kname, cfg["key"])
    roofline = {"bound": "alu", "achieved": achieved, "peak": peaks["fp32_tflops"], "unit": "TFLOP/s",
                "frac": achieved / peaks["fp32_tflops"], "traffic": traffic, "traffic_note": traffic_note,
                "kernel": kname, "kernel_ms": state_ms[kname],
                "peak_source": "measured in this run (vbm_peak_probe, FP32 FMA chains: %.1f, FP32x2 FMA chains: "
                               "%.1f TFLOP/s); derived 152 SMs x 128 lanes x 2 x 2070 MHz = %.1f"
                               % (peaks["fp32_fma_tflops"], peaks["fp32x2_fma_tflops"], peaks["derived_fp32_tflops"]),
                "sfu_frac": work[kname]["sfu"] / (state_ms[kname] * 1e-3) / 1e12 / peaks["ex2_tera_per_s"],
                "pairs_fwd_per_step": p_fwd_step, "pairs_bwd_per_step": p_bwd_step,
                "pairs_counted": "per-pixel counts of %d untimed forwards spread through the timed steps"
                                 % len(counts),
                "flop_per_pair": {"fwd": FWD_FLOP_PER_PAIR, "bwd": BWD_FLOP_PER_PAIR},
                "step_frac": lb_sum / ms_per_step, "step_lower_bound_ms": lb_sum,
                "graph_head_ms": state_ms["head"],
                "kernels": kernels, "peaks": peaks}

    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["workload"], "key": cfg["key"], "gaussians": int(n), "views": V,
                       "image": "%dx%d" % (W, H),
                       "tile": "%dx%d" % tile, "pixels_per_thread": ppt, "group_lanes": gl, "persistent": pers,
                       "segment_len": (seg if seg else 256) if pers else None,
                       "bwd_pixels_per_thread": bppt or ppt, "bwd_group_lanes": bgl or gl,
                       "pair_order": "device radix sorts" if args.radix else "bucketed per-tile sort",
                       "compositing_state": "recomputed in the backward" if batch["recompute"] else "stored",
                       "adam": "fused into the projection backward" if fused_adam else "separate kernel",
                       "pairs_mean": int(n_pairs),
                       "timed_iterations": "fine-tuning iterations %d-%d from the built Gaussians (the launch "
                                           "configuration was tuned on a copy %d iterations in)"
                                           % (args.warmup + extra_steps + 1, args.warmup + extra_steps + args.steps,
                                              TUNE_WARM_STEPS),
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
                             "raster_fwd_kernel": V * H * W / (t_fwd * 1e-3) / 1e9,
                             "note": "fwd = projection + binning + sort + compositing of all views, one call, "
                                     "median of %d; raster_fwd_kernel = the compositing kernel alone" % n_px},
            "e2e": {"value": 1e3 / e2e_ms, "unit": "steps/s", "h2d_bytes_per_step": int(targets.numel() * 4),
                    "d2h_bytes_per_step": 8, "ms_per_step": e2e_ms,
                    "timing": "host clock per step: graph launch (targets copied from pinned host memory inside "
                              "it), stream synchronize, host read of the loss; L2 flushed before each step, "
                              "outside the timed interval",
                    "loss_first_last": [losses[0], losses[-1]]},
            "roofline": roofline, "gpu_launches": int(launches_per_step * args.steps),
            "launches_per_step": int(launches_per_step), "wall_s_timed": wall}
    if fwd_only_rec is not None:
        line["fwd_only"] = fwd_only_rec
    if clk is not None:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from vbm_inputs.cameras import cameras_as_float32
        if w.scene_offset is None:
            cams32 = cameras_as_float32(cams)
            window = CPU_WINDOW.get(cfg["key"])
            sampler = OracleSampler(params0.cpu().numpy().astype(np.float64), cams32, targets.cpu().numpy(),
                                    window, pairs_view)
            try:
                wall_c, per_view, _ = sampler.run()
                t_adam = sampler.adam_seconds(workload_extent(cfg))
            finally:
                sampler.close()
            line["cpu_baseline"] = baseline_record(
                sampler, per_view, wall_c, t_adam,
                "whole view, nothing extrapolated" if window is None else "window %d" % window)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
