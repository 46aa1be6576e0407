"""GPU parity of the image loss, Adam and a whole fine-tuning step (Sec. 4.4, Sec. 5.2),
plus a central finite-difference check of the GPU gradient."""

import numpy as np
import pytest
import torch

from _helpers import read_device, rel_group_error, scene, split_place, split_records, to_device
from oracle import adam as oadam
from oracle import loss as oloss
from oracle import raster as oraster

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(2, 40, 50), (1, 128, 128), (3, 17, 33)])
def test_loss_and_gradient(cuda_lib, shape):
    vbm = cuda_lib
    V, H, W = shape
    rng = np.random.default_rng(V * 100 + H)
    x = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1).astype(np.float32)
    x[0, 0, :3, :3] = y[0, 0, :3, :3]         # exact ties: sign(0) = 0
    L_ref, g_ref = oloss.loss_and_grad(x.astype(np.float64), y.astype(np.float64))
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ws = vbm.loss_workspace(V, H, W)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(xt)
    vbm.loss(xt, yt, V, H, W, 0.2, 1.0 / x.size, L, g, ws)
    torch.cuda.synchronize()
    assert abs(L.item() - L_ref) <= 1e-6 * L_ref
    nrm, elt = rel_group_error(g.cpu().numpy(), g_ref)
    assert nrm < 1e-3 and elt < 1e-3, (nrm, elt)
    # accumulate: per-image calls add up to the batched value
    L2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for v in range(V):
        vbm.loss(xt[v], yt[v], 1, H, W, 0.2, 1.0 / x.size, L2, g[v], ws, accumulate=v > 0)
    torch.cuda.synchronize()
    assert abs(L2.item() - L.item()) <= 1e-12 * max(1.0, L.item())


@pytest.mark.parametrize("n, stride", [(1000, 1003), (1001, 1001), (513, 513), (3, 3)])
def test_adam_matches_oracle(cuda_lib, n, stride):
    """Padded rows (stride > n): one scalar per thread and row; packed rows: four scalars per
    thread over the flat array, quads crossing rows, a ragged last quad (14 n not a multiple
    of 4), and n < 4 (a quad spanning three rows)."""
    vbm = cuda_lib
    rng = np.random.default_rng(3)
    P = rng.standard_normal((14, stride)).astype(np.float32)
    lrs = oadam.default_lrs(64.0)
    Pt = torch.from_numpy(P.copy()).cuda()
    m, v = torch.zeros_like(Pt), torch.zeros_like(Pt)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    P64, m64, v64 = P[:, :n].astype(np.float64), np.zeros((14, n)), np.zeros((14, n))
    for t in range(1, 4):
        G = (rng.standard_normal((14, stride)) * 10.0 ** rng.uniform(-4, 0, (14, 1))).astype(np.float32)
        vbm.adam(Pt, torch.from_numpy(G).cuda(), m, v, n, step, lrs, nonfinite=bad)
        oadam.adam_step(P64, G[:, :n].astype(np.float64), m64, v64, t, lrs)
    torch.cuda.synchronize()
    out = Pt.cpu().numpy()
    assert step.item() == 3 and bad.item() == 0
    assert np.abs(out[:, :n] - P64).max() < 2e-5 * max(1.0, np.abs(P64).max())
    assert np.array_equal(out[:, n:], P[:, n:])      # columns beyond n untouched
    # a non-finite gradient element is counted and leaves its parameter alone
    G = np.zeros((14, stride), dtype=np.float32)
    G[2, 5 % n] = np.nan
    G[3, 6 % n] = np.inf
    G[4, 7 % n] = -np.inf
    G[13, n - 1] = np.nan
    before = Pt.cpu().numpy()
    vbm.adam(Pt, torch.from_numpy(G).cuda(), m, v, n, step, lrs, nonfinite=bad)
    torch.cuda.synchronize()
    after = Pt.cpu().numpy()
    bad_at = ((2, 5 % n), (3, 6 % n), (4, 7 % n), (13, n - 1))
    assert bad.item() == 4
    for r, c in bad_at:
        assert after[r, c] == before[r, c]
    ok = np.ones((14, n), dtype=bool)
    for r, c in bad_at:
        ok[r, c] = False
    assert np.all(after[:, :n][ok] != before[:, :n][ok])   # finite scalars of the same quads move


def test_gradient_central_differences(cuda_lib):
    """Autograd backward (torch.autograd.Function over vbm_raster_fwd/bwd) of L = sum w * img
    on 64 sampled parameters against central differences of the GPU forward (FP32, h = 1e-3).
    The two FP32 images are differenced in FP64 and the step is the exact float32 difference
    of the perturbed parameters; the tolerance is 5e-2 relative plus ten times the rounding
    noise of the differenced images.  A sample is skipped when the FP64 oracle shows that a
    compositing decision differs between theta + h and theta - h (per pixel: the number of
    blended Gaussians or the position of the last one) or a tile rectangle moves: the loss is
    discontinuous across such a flip."""
    from paper_2601_09417_gb300.autograd import render
    vbm = cuda_lib
    W, H, V = 64, 64, 2
    P, cams, cams32 = scene(seed=21, n=300, V=V, W=W, H=H, scale_range=(0.8, 2.5))
    params, cams_dev = to_device(P, cams)
    plan = vbm.Plan([0, P.shape[1]], V, W, H, pair_capacity=1 << 20)
    w_np = np.random.default_rng(5).uniform(0.5, 1.5, (V, 3, H, W)).astype(np.float32)
    w = torch.from_numpy(w_np).cuda()
    p = params.clone().requires_grad_(True)
    (render(p, plan, cams_dev) * w).sum().backward()
    g = p.grad.cpu().numpy()
    img = torch.zeros((V, 3, H, W), device="cuda")

    def render_np(Pn):
        plan.forward(torch.from_numpy(Pn).cuda(), cams_dev, img)
        return img.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(2000):
        if checked == 64:
            break
        r, c = int(rng.integers(0, 14)), int(rng.integers(0, P.shape[1]))
        if abs(g[r, c]) < 1e-2 * np.abs(g[r]).max():
            continue
        Pp, Pm = P.copy(), P.copy()
        Pp[r, c] += np.float32(1e-3)
        Pm[r, c] -= np.float32(1e-3)
        fp = oraster.splat_forward(Pp.astype(np.float64), cams32)
        fm = oraster.splat_forward(Pm.astype(np.float64), cams32)
        if not (np.array_equal(fp["n_blend"], fm["n_blend"]) and np.array_equal(fp["n_contrib"], fm["n_contrib"])
                and np.array_equal(fp["rect"], fm["rect"])):
            continue
        two_h = float(np.float64(Pp[r, c]) - np.float64(Pm[r, c]))
        diff = render_np(Pp) - render_np(Pm)
        fd = float((diff * w_np).sum()) / two_h
        noise = np.sqrt(max(1, int((diff != 0).sum()))) * 2 * 6e-8 * 1.5 / two_h
        assert abs(fd - g[r, c]) <= 5e-2 * abs(g[r, c]) + 10 * noise, (r, c, fd, g[r, c], noise)
        checked += 1
    assert checked == 64, checked


def test_full_step_matches_oracle_step(cuda_lib):
    """One whole fine-tuning step (forward, L1 + D-SSIM, backward, Adam) against the FP64
    oracle's step.  The scene is one whose every pixel stays at least 2e-5 (relative) from
    each compositing cut-off in the oracle and whose image differs from the target by more
    than 1e-5 everywhere (asserted), so FP32 takes the same decisions as FP64 and no pixel
    is excluded.  Bars: loss 1e-6 relative; gradient 1e-3 per parameter group in norm and
    element-wise; Adam element-wise: against the oracle's Adam on the GPU's own gradient,
    and against the oracle's step wherever the gradient's sign is decided (|g_ref| above
    1e-2 of its group's rms; elsewhere the update is bounded by the learning rate)."""
    vbm = cuda_lib
    from oracle.step import finetune_step
    W, H, V, G = 64, 48, 2, 32
    P, cams, cams32 = scene(seed=40, n=800, V=V, W=W, H=H)
    target = np.random.default_rng(2).uniform(0, 0.4, (V, 3, H, W)).astype(np.float32)
    params, cams_dev = to_device(P, cams)
    plan = vbm.Plan([0, P.shape[1]], V, W, H, pair_capacity=1 << 20)
    img = torch.zeros((V, 3, H, W), device="cuda")
    dimg = torch.empty_like(img)
    ws = vbm.loss_workspace(V, H, W)
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros_like(params)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    lrs = oadam.default_lrs(G)
    tgt = torch.from_numpy(target).cuda()
    plan.forward(params, cams_dev, img)
    vbm.loss(img, tgt, V, H, W, 0.2, 1.0 / img.numel(), L, dimg, ws)
    plan.backward(params, cams_dev, dimg, grad)
    vbm.adam(params, grad, m, v, P.shape[1], step, lrs)
    torch.cuda.synchronize()
    P64 = P.astype(np.float64)
    m64, v64 = np.zeros_like(P64), np.zeros_like(P64)
    L_ref, g_ref, fwd = finetune_step(P64, m64, v64, 1, cams32, target.astype(np.float64), lrs)
    assert fwd["margin"].min() > 2e-5
    assert np.abs(fwd["img"] - target).min() > 1e-5
    assert np.abs(img.cpu().numpy() - fwd["img"]).max() <= 1e-4
    assert abs(L.item() - L_ref) <= 1e-6 * L_ref
    g = grad.cpu().numpy()
    for lo, hi in oadam.ROW_GROUPS:
        nrm, elt = rel_group_error(g[lo:hi], g_ref[lo:hi])
        assert nrm < 1e-3 and elt < 1e-3, (lo, nrm, elt)
    P_gpu = params.cpu().numpy().astype(np.float64)
    # Adam itself, element-wise, on the GPU's gradient
    P_own = P.astype(np.float64)
    oadam.adam_step(P_own, g.astype(np.float64), np.zeros_like(P_own), np.zeros_like(P_own), 1, lrs)
    lr_row = np.concatenate([np.full(hi - lo, lr) for (lo, hi), lr in zip(oadam.ROW_GROUPS, lrs)])[:, None]
    assert (np.abs(P_gpu - P_own) <= 1e-6 * np.abs(P_own) + 1e-5 * lr_row).all()
    # the step against the oracle's step
    decided = np.zeros_like(g_ref, dtype=bool)
    for lo, hi in oadam.ROW_GROUPS:
        rms = np.sqrt(np.mean(g_ref[lo:hi] ** 2))
        decided[lo:hi] = np.abs(g_ref[lo:hi]) > 1e-2 * rms
    tol = 1e-6 * np.abs(P64) + 1e-5 * lr_row
    assert (np.abs(P_gpu - P64) <= tol)[decided].all()
    step_gpu = P_gpu - P.astype(np.float64)
    assert (np.abs(step_gpu) <= lr_row * (1 + 1e-5) + 1e-6 * np.abs(P64)).all()
    assert decided.mean() > 0.5


def test_gradient_central_differences_c1_full_size(cuda_lib):
    """Full-size workload (128^3 volume -> ~5e4 Gaussians by vbm_build, 8 views of
    512 x 512, DVR targets, 8 x 8 tiles): the gradient of the fine-tuning loss
    (L1 + D-SSIM, lambda = 0.2) through the autograd Function against central
    differences of the GPU loss on 64 sampled parameters (h = 1e-3, exact float32 step).
    A sample is skipped where the loss is discontinuous between theta - h and theta + h:
    the depth order of any tile's list changes, a tile rectangle moves, any pixel's
    contributor count changes, or the perturbed Gaussian's own alpha crosses (or comes
    within 1e-4 of) the 1/255 cut-off at a pixel of its tiles.  Tolerance: 5e-2 relative,
    plus ten times the FP32 rounding noise of the changed pixels, plus twice the bound
    on the L1 kink error from pixels whose residual changes sign."""
    from paper_2601_09417_gb300.autograd import render
    from paper_2601_09417_gb300.workloads import make_workload
    vbm = cuda_lib
    lam = 0.2
    w = make_workload("c1")
    V, H, W = w.targets.shape[0], w.targets.shape[2], w.targets.shape[3]
    n = w.n
    cams_dev = vbm.cameras_to_device(w.cam_records)
    plan = vbm.Plan([0, n], V, W, H, tile_w=8, tile_h=8, pixels_per_thread=1, pair_capacity=1 << 25)
    ws = vbm.loss_workspace(V, H, W)
    scale = 1.0 / (V * 3 * H * W)

    class Loss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, img):
            L = torch.zeros(1, dtype=torch.float64, device="cuda")
            d = torch.empty_like(img)
            vbm.loss(img.contiguous(), w.targets, V, H, W, lam, scale, L, d, ws)
            ctx.save_for_backward(d)
            return L

        @staticmethod
        def backward(ctx, gL):
            (d,) = ctx.saved_tensors
            return d * gL.to(d.dtype)

    P = w.params.detach().clone()
    p = P.clone().requires_grad_(True)
    Loss.apply(render(p, plan, cams_dev)).sum().backward()
    g = p.grad.cpu().numpy()

    def evaluate(Pt):
        img = torch.zeros((V, 3, H, W), device="cuda")
        plan.forward(Pt, cams_dev, img)
        L = float(Loss.apply(img).item())
        b = plan.buffers()
        n_pairs = int(read_device(b.n_pairs, (1,), np.int64)[0])
        st = dict(img=img, n_contrib=vbm.device_tensor(b.n_contrib, (V, H, W), np.int32).clone(),
                  pair_item=vbm.device_tensor(b.pair_item, (n_pairs,), np.int32).clone(),
                  pair_tile=vbm.device_tensor(b.pair_tile, (n_pairs,), np.int32).clone(),
                  rect=split_place(read_device(b.place, (b.n_items, 4), np.uint32))["rect"],
                  **split_records(read_device(b.rec, (b.n_items, 16), np.float32)))
        return L, st

    def own_alpha(st, item):
        x0, y0, x1, y1 = st["rect"][item]
        if x1 <= x0 or y1 <= y0:
            return np.zeros(0)
        xs = np.arange(x0 * 8, min(x1 * 8, W)) + 0.5
        ys = np.arange(y0 * 8, min(y1 * 8, H)) + 0.5
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        u, v_, A, B = st["geo"][item].astype(np.float64)
        C, o = float(st["conic_c"][item]), float(st["col"][item][3])
        dx, dy = u - X, v_ - Y
        return o * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)

    def same(a, b):
        return a.shape == b.shape and bool(torch.equal(a, b))

    rng = np.random.default_rng(11)
    checked, tried = 0, 0
    while checked < 64 and tried < 3000:
        tried += 1
        r, c = int(rng.integers(0, 14)), int(rng.integers(0, n))
        if abs(g[r, c]) < 1e-2 * np.abs(g[r]).max():
            continue
        h = np.float32(1e-3)
        Pp, Pm = P.clone(), P.clone()
        Pp[r, c] += float(h)
        Pm[r, c] -= float(h)
        Lp, sp = evaluate(Pp)
        Lm, sm = evaluate(Pm)
        if not (same(sp["pair_item"], sm["pair_item"]) and same(sp["pair_tile"], sm["pair_tile"])
                and same(sp["n_contrib"], sm["n_contrib"]) and np.array_equal(sp["rect"], sm["rect"])):
            continue
        flip = False
        for v in range(V):
            a_p, a_m = own_alpha(sp, v * n + c), own_alpha(sm, v * n + c)
            if a_p.size and (np.minimum(np.abs(255 * a_p - 1), np.abs(255 * a_m - 1)).min() < 1e-4
                             or np.any((a_p >= 1 / 255) != (a_m >= 1 / 255))):
                flip = True
                break
        if flip:
            continue
        two_h = float(Pp[r, c].item()) - float(Pm[r, c].item())
        d = sp["img"] - sm["img"]
        changed = int(torch.count_nonzero(d).item())
        kink = ((sp["img"] - w.targets) * (sm["img"] - w.targets) < 0)
        kink_bound = float((d.abs() * kink).sum().item()) * (1 - lam) * scale / two_h
        noise = np.sqrt(max(1, changed)) * 2 * 6e-8 * 3.0 * scale / two_h
        fd = (Lp - Lm) / two_h
        assert abs(fd - g[r, c]) <= 5e-2 * abs(g[r, c]) + 10 * noise + 2 * kink_bound, \
            (r, c, fd, g[r, c], noise, kink_bound)
        checked += 1
    assert checked == 64, (checked, tried)


def test_graph_and_host_steps_match_batched_steps(cuda_lib):
    """One fine-tuning step on the c0 workload through the batched calls, through the
    captured graph, and through the end-to-end graph (targets copied from pinned host
    memory on a side branch, loss read back to pinned host memory) gives the same loss
    and the same gradient up to the atomic order of the gradient sums; the host copy of
    the loss equals the device loss; the graphs replay."""
    from paper_2601_09417_gb300.finetune import FineTuner
    from paper_2601_09417_gb300.workloads import make_workload
    w = make_workload("c0")
    P0 = w.params.detach().clone()
    launch = dict(tile=(8, 8), ppt=1, group_lanes=16, persistent=True, extent=w.cfg["G"])
    runs = {}
    for mode in ("batched", "graph", "host"):
        ft = FineTuner(P0.clone(), w.cam_records, w.targets, fused_adam=False, **launch)
        host_t = torch.empty(w.targets.shape, dtype=torch.float32, pin_memory=True)
        host_t.copy_(w.targets)
        host_l = torch.zeros(1, dtype=torch.float64, pin_memory=True)
        step = {"batched": ft.step_batched, "graph": ft.step_graph,
                "host": lambda: ft.step_host(host_t, host_l)}[mode]
        step()
        torch.cuda.synchronize()
        runs[mode] = (float(ft.loss.item()), ft.grad.cpu().numpy())
        if mode == "host":
            assert host_l.item() == runs[mode][0] > 0
        step()                                   # a second replay / step
        torch.cuda.synchronize()
        ok, need, bad = ft.check()
        assert ok and bad == 0
        assert 0 < ft.loss.item() != runs[mode][0]        # the parameters moved, the loss too
    L0, g0 = runs["batched"]
    for mode in ("graph", "host"):
        L, g = runs[mode]
        assert abs(L - L0) <= 1e-12 * L0, (mode, L, L0)
        for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
            nrm, elt = rel_group_error(g[lo:hi], g0[lo:hi])
            assert nrm < 1e-5, (mode, lo, nrm)


@pytest.mark.parametrize("persistent", [False, True])
def test_fused_backward_adam_equals_separate_calls(cuda_lib, persistent):
    """vbm_raster_bwd_adam against vbm_raster_bwd (accumulate = 0, zeroed gradient) +
    vbm_adam on copies of the same state, at Adam step 6 with nonzero moments (the update
    is then smooth in the gradient): the columns of a second scene that no view renders
    take the zero-gradient step bit for bit, the rendered columns agree up to the atomic
    order of the splat-gradient sums, the step counters advance together, and a
    non-finite pixel gradient is counted alike."""
    vbm = cuda_lib
    W, H, V = 64, 48, 3
    P, cams, _ = scene(seed=11, n=1200, V=V, W=W, H=H)
    n1 = P.shape[1]
    extra, _, _ = scene(seed=12, n=300, V=1, W=W, H=H)
    P2 = np.concatenate([P, extra], axis=1)
    n = P2.shape[1]
    params, cams_dev = to_device(P2, cams)
    plan = vbm.Plan([0, n1, n], V, W, H, view_scene=[0] * V, tile_w=8, tile_h=8, pair_capacity=1 << 20,
                    flags=vbm.PLAN_PERSISTENT if persistent else 0, group_lanes=8)
    img = torch.zeros((V, 3, H, W), device="cuda")
    plan.forward(params, cams_dev, img)
    rng = np.random.default_rng(13)
    lrs = oadam.default_lrs(32.0)
    m0 = torch.from_numpy((0.01 * rng.standard_normal((14, n))).astype(np.float32)).cuda()
    v0 = torch.from_numpy((1e-3 * rng.random((14, n)) + 1e-6).astype(np.float32)).cuda()
    for bad_pixel in (False, True):
        dimg_h = rng.standard_normal((V, 3, H, W)).astype(np.float32)
        if bad_pixel:
            dimg_h[1, 0, H // 2, W // 2] = np.nan
        dimg = torch.from_numpy(dimg_h).cuda()
        out = {}
        for fused in (False, True):
            Pw, m, v = params.clone(), m0.clone(), v0.clone()
            step = torch.full((1,), 5, dtype=torch.int32, device="cuda")
            bad = torch.zeros(1, dtype=torch.int32, device="cuda")
            if fused:
                plan.backward_adam(Pw, cams_dev, dimg, m, v, n, step, lrs, nonfinite=bad)
            else:
                grad = torch.zeros_like(params)
                plan.backward(params, cams_dev, dimg, grad)
                vbm.adam(Pw, grad, m, v, n, step, lrs, nonfinite=bad)
            torch.cuda.synchronize()
            out[fused] = [t.cpu().numpy() for t in (Pw, m, v)] + [int(step.item()), int(bad.item())]
        (Pa, ma, va, sa, ba), (Pb, mb, vb, sb, bb) = out[False], out[True]
        assert sa == sb == 6
        assert ba == bb and (ba > 0) == bad_pixel
        for a, b in ((Pa, Pb), (ma, mb), (va, vb)):
            assert np.array_equal(a[:, n1:], b[:, n1:])          # unrendered scene: bit for bit
        if bad_pixel:
            continue
        P0 = P2.astype(np.float32)
        for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
            da, db = Pa[lo:hi, :n1] - P0[lo:hi, :n1], Pb[lo:hi, :n1] - P0[lo:hi, :n1]
            nrm, elt = rel_group_error(db, da)
            assert nrm < 1e-4, (lo, nrm, elt)
            nrm, _ = rel_group_error(mb[lo:hi, :n1], ma[lo:hi, :n1])
            assert nrm < 1e-5, (lo, nrm)
    plan.close()


def test_peak_probe(cuda_lib):
    """vbm_peak_probe reports its work exactly, and the rates it measures on one wave are
    positive and below the unit-count limits (FP32: 2 FLOP per lane per clock; ex2 a
    fraction of that)."""
    vbm = cuda_lib
    props = torch.cuda.get_device_properties(0)
    blocks = props.multi_processor_count * 8
    out = torch.zeros(blocks * 256, device="cuda")
    for kind, per_link in ((0, 2.0), (1, 4.0), (2, 1.0)):
        iters = 4096
        vbm.peak_probe(kind, blocks, iters, out)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        ops = vbm.peak_probe(kind, blocks, iters, out)
        e.record()
        e.synchronize()
        assert ops == blocks * 256 * iters * 8 * per_link
        rate = ops / (s.elapsed_time(e) * 1e-3)
        assert 0 < rate < props.multi_processor_count * 128 * 2 * 2.2e9 * 1.05
    assert torch.count_nonzero(out) == 0     # the chains never hit the guarded store
    with pytest.raises(vbm.VbmError) as err:
        vbm.peak_probe(3, blocks, 16, out)
    assert err.value.status == vbm.VBM_ERR_ARG
    with pytest.raises(vbm.VbmError):
        vbm.peak_probe(0, blocks, 10, out)         # not a multiple of 16
