"""GPU parity of the splatting forward/backward (Sec. 4.4) against the FP64 oracle.

Bars (from the method's accuracy targets):
  * tile keys, pair order and ranges bit-exact given the GPU's projected depths;
  * images within 1e-4 max-abs per channel, excluding pixels where an FP32 vs
    FP64 difference can flip a compositing cut-off (relative margin to
    alpha = 1/255 or T = 1e-4 below 1e-5); flagged pixels must stay rare;
  * gradients within 1e-3 relative (group norm) and
    |g - g_ref| <= 1e-3 (|g_ref| + rms(g_ref)) element-wise.
"""

import numpy as np
import pytest
import torch

from _helpers import gpu_binning_records, gpu_splats_as_oracle, plan_state, rel_group_error, scene, to_device
from oracle import raster as oraster
from oracle.raster import PJ

pytestmark = pytest.mark.gpu


def _forward(vbm, P, cams, W, H, tile=(16, 16), cap=1 << 22, scene_offset=None, view_scene=None, bg=(0, 0, 0),
             ppt=0, persistent=False, gl=0, seg=0, radix=False):
    params, cams_dev = to_device(P, cams)
    V = len(cams)
    so = [0, P.shape[1]] if scene_offset is None else scene_offset
    flags = (vbm.PLAN_PERSISTENT if persistent else 0) | (vbm.PLAN_RADIX_SORT if radix else 0)
    plan = vbm.Plan(so, V, W, H, view_scene=view_scene, tile_w=tile[0], tile_h=tile[1], pair_capacity=cap,
                    pixels_per_thread=ppt, flags=flags, group_lanes=gl, segment_len=seg)
    img = torch.zeros((V, 3, H, W), device="cuda")
    alpha = torch.zeros((V, H, W), device="cuda")
    plan.forward(params, cams_dev, img, alpha, bg=bg)
    torch.cuda.synchronize()
    return plan, params, cams_dev, img.cpu().numpy(), alpha.cpu().numpy()


def _tiles(W, H, tile):
    return (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]


def test_preprocess_matches_oracle(cuda_lib):
    P, cams, cams32 = scene(seed=1, n=3000, V=3, W=100, H=76)
    plan, *_ = _forward(cuda_lib, P, cams, 100, 76)
    st = plan_state(plan, 3)
    n = P.shape[1]
    P64 = P.astype(np.float64)
    flagged = 0
    for v in range(3):
        ref = oraster.project(P64, cams32[v], np.arange(n), 16, 16)
        sl = slice(v * n, (v + 1) * n)
        assert np.allclose(st["depth"][sl], ref[:, PJ["DEPTH"]], rtol=1e-6, atol=1e-5)
        assert np.allclose(st["col"][sl, 3], ref[:, PJ["OPAC"]], atol=2e-7)
        assert np.array_equal(st["col"][sl, :3], P[11:14].T)
        vis = ref[:, PJ["TOUCHED"]] > 0
        culled = ref[:, PJ["RADIUS"]] == 0
        safe = ((ref[:, PJ["M_RADIUS"]] > 1e-3) | culled) & (ref[:, PJ["M_RECT"]] > 1e-3) \
            & (ref[:, PJ["M_CULL"]] > 1e-3) & (ref[:, PJ["M_OPAC"]] > 1e-3)
        flagged += int((~safe).sum())
        g = st["geo"][sl]
        scale_uv = np.abs(ref[:, [PJ["U"], PJ["V"]]]) + 100.0
        assert (np.abs(g[vis, 0:2] - ref[vis][:, [PJ["U"], PJ["V"]]]) < 1e-6 * scale_uv[vis]).all()
        conic = np.stack([g[:, 2], g[:, 3], st["conic_c"][sl]], axis=1)
        cref = ref[:, [PJ["A"], PJ["B"], PJ["C"]]]
        cs = np.abs(cref[vis]).max(axis=1, keepdims=True)
        assert (np.abs(conic[vis] - cref[vis]) <= 2e-5 * cs).all()
        assert np.array_equal(st["radius"][sl][safe], ref[safe, PJ["RADIUS"]].astype(np.int32))
        rref = ref[:, [PJ["X0"], PJ["Y0"], PJ["X1"], PJ["Y1"]]].astype(np.int32)
        assert np.array_equal(st["rect"][sl][safe], rref[safe])
    assert flagged < 0.01 * 3 * n


@pytest.mark.parametrize("tile,radix", [((16, 16), False), ((8, 8), False), ((8, 4), False), ((16, 16), True),
                                        ((8, 8), True)])
def test_binning_bit_exact_given_gpu_depths(cuda_lib, tile, radix):
    """Pair lists, order and ranges equal, bit for bit, the oracle's (tile, depth, index)
    sort of the GPU's rectangles and depths, with the oracle's float32 tile test on the
    GPU's float32 splat records; the records' B/C and B/A are the float32 quotients of the
    GPU's own conic, and the test removes pairs (the lists are shorter than the
    rectangles)."""
    P, cams, cams32 = scene(seed=2, n=2500, V=3, W=100, H=76)
    plan, *_ = _forward(cuda_lib, P, cams, 100, 76, tile=tile, radix=radix, persistent=radix)
    st = plan_state(plan, 3)
    n = P.shape[1]
    TX, TY = _tiles(100, 76, tile)
    view_of = np.repeat(np.arange(3, dtype=np.int32), n)
    rec = gpu_binning_records(st)
    live = st["tau"] > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        assert np.array_equal(rec[live, 5], (rec[live, 3] / rec[live, 4]).astype(np.float32))
        assert np.array_equal(rec[live, 6], (rec[live, 3] / rec[live, 2]).astype(np.float32))
    tiles, items, ranges = oraster.bin_sort(view_of, st["rect"], st["depth"].astype(np.float64), TX, TY, 3,
                                            splat32=rec, tile=tile, image=(100, 76))
    area = int(((st["rect"][:, 2] - st["rect"][:, 0]) * (st["rect"][:, 3] - st["rect"][:, 1])).sum())
    assert tiles.size < area
    assert st["n_pairs"] == tiles.size > 0
    assert np.array_equal(st["pair_tile"].astype(np.int64), tiles)
    assert np.array_equal(st["pair_item"].astype(np.int64), items.astype(np.int64))
    assert np.array_equal(st["ranges"], ranges)
    # the placement records: listed-tile words as the oracle's lists give them, the depth
    # the splat record's bit for bit
    assert np.array_equal(st["listed"], _listed_words(tiles, items, st["rect"], st["n_items"], TX, TY))
    assert np.array_equal(st["place_depth"].view(np.uint32), st["depth"].view(np.uint32))


def _listed_words(tiles, items, rect, n_items, TX, TY):
    """Each item's listed-tile word from a pair list: for a rectangle of at most 8 tiles,
    bit k for its k-th tile (row-major) in the list; a larger rectangle with any listed
    tile: bit 31 alone; no listed tile: 0."""
    items = np.asarray(items, dtype=np.int64)
    local = np.asarray(tiles, dtype=np.int64) % (TX * TY)
    tx, ty = local % TX, local // TX
    x0, y0, x1, y1 = (rect[items, c].astype(np.int64) for c in range(4))
    cols = x1 - x0
    small = cols * (y1 - y0) <= 8
    words = np.zeros(n_items, dtype=np.uint32)
    k = (ty - y0) * cols + (tx - x0)
    np.bitwise_or.at(words, items[small], (np.uint32(1) << k[small].astype(np.uint32)))
    words[items[~small]] = np.uint32(1 << 31)
    return words


@pytest.mark.parametrize("radix", [False, True])
def test_binning_long_lists_bit_exact(cuda_lib, radix):
    """Crowded scene: one cluster of 10,000 small Gaussians (plus 500 exact copies, so
    equal depths must fall back to the index order) projects into a few tiles, whose
    lists exceed the 4096 keys one block sorts in shared memory; a wider cluster gives
    lists of every shorter length class (<= 32, <= 256, <= 4096).  The pair lists must
    equal the oracle's (tile, depth, index) sort bit for bit."""
    from vbm_inputs.gaussians import random_gaussians
    from vbm_inputs import orbit_cameras
    from vbm_inputs.cameras import cameras_as_float32
    G, W, H, tile = 32, 100, 76, (8, 8)
    core = random_gaussians(10000, 15.7, 16.3, seed=21, scale_range=(0.1, 0.4), opacity_logit_range=(-1.0, 2.0))
    wide = random_gaussians(3000, 8.0, 24.0, seed=22, scale_range=(0.2, 1.5), opacity_logit_range=(-2.0, 2.0))
    P = np.concatenate([core, core[:, :500], wide], axis=1).astype(np.float32)
    cams = orbit_cameras((G, G, G), 1, W, H)
    plan, *_ = _forward(cuda_lib, P, cams, W, H, tile=tile, radix=radix)
    st = plan_state(plan, 1)
    TX, TY = _tiles(W, H, tile)
    lengths = st["ranges"][:, 1] - st["ranges"][:, 0]
    assert lengths.max() > 2 * 4096
    for lo, hi in [(1, 32), (33, 256), (257, 4096)]:
        assert ((lengths >= lo) & (lengths <= hi)).any(), (lo, hi)
    rec = gpu_binning_records(st)
    tiles, items, ranges = oraster.bin_sort(np.zeros(st["n_items"], dtype=np.int32), st["rect"],
                                            st["depth"].astype(np.float64), TX, TY, 1, splat32=rec, tile=tile,
                                            image=(W, H))
    assert st["n_pairs"] == tiles.size
    assert np.array_equal(st["pair_tile"].astype(np.int64), tiles)
    assert np.array_equal(st["pair_item"].astype(np.int64), items.astype(np.int64))
    assert np.array_equal(st["ranges"], ranges)
    plan.close()


@pytest.mark.parametrize("tile,ppt,persistent,gl", [((16, 16), 1, False, 32), ((16, 16), 2, False, 32),
                                                    ((16, 16), 4, False, 32), ((8, 8), 2, False, 32),
                                                    ((16, 8), 1, False, 32), ((16, 8), 4, False, 32),
                                                    ((16, 16), 1, True, 32), ((8, 8), 1, True, 32),
                                                    ((8, 8), 1, True, 8), ((8, 8), 1, False, 16),
                                                    ((16, 16), 1, False, 8), ((16, 16), 2, True, 16),
                                                    ((8, 8), 2, True, 4), ((16, 16), 1, False, 4), ((16, 8), 4, True, 4),
                                                    ((16, 8), 4, False, 8), ((8, 8), 2, False, 8),
                                                    ((8, 4), 1, True, 16), ((8, 4), 1, False, 32),
                                                    ((16, 4), 1, True, 8), ((8, 8), 1, "radix", 16)])
def test_composite_matches_oracle_on_gpu_splats(cuda_lib, tile, ppt, persistent, gl):
    """persistent = "radix": a persistent plan ordering its pairs by device radix sorts."""
    W, H = 100, 76
    P, cams, cams32 = scene(seed=3, n=2500, V=2, W=W, H=H)
    bg = (0.1, 0.2, 0.05)
    plan, _, _, img, alpha = _forward(cuda_lib, P, cams, W, H, tile=tile, bg=bg, ppt=ppt, persistent=bool(persistent),
                                      gl=gl, radix=persistent == "radix")
    st = plan_state(plan, 2)
    splat, color = gpu_splats_as_oracle(st)
    ref = oraster.render(2, W, H, tile[0], tile[1], st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                         np.array(bg))
    good = ref["margin"] > 1e-5
    assert good.mean() > 0.99, good.mean()
    err = np.abs(img - ref["img"]).transpose(1, 0, 2, 3)[:, good]
    assert err.max() <= 1e-4, err.max()
    assert np.abs(alpha - (1 - ref["T_final"]))[good].max() <= 1e-4
    assert np.array_equal(st["n_contrib"][good], ref["n_contrib"][good])
    assert np.abs(st["T_final"] - ref["T_final"])[good].max() <= 1e-4
    assert img.max() > 0.05      # the scene is not empty


@pytest.mark.parametrize("ppt,persistent,recompute", [(1, False, False), (2, True, False), (2, True, True),
                                                     (1, True, True)])
def test_profiling_counts_match_oracle(cuda_lib, ppt, persistent, recompute):
    """The plan's profiling hooks: per pixel the number of list entries evaluated (up to and
    including the one that ended compositing) and, for recompute plans, the contributor
    count equal the oracle's on the GPU's own splats and lists; the image of a forward with
    the hooks set (a separately compiled kernel variant) is bit-identical to one without."""
    vbm = cuda_lib
    W, H, V = 100, 76, 2
    P, cams, cams32 = scene(seed=8, n=2500, V=V, W=W, H=H)
    params, cams_dev = to_device(P, cams)
    flags = (vbm.PLAN_PERSISTENT if persistent else 0) | (vbm.PLAN_RECOMPUTE if recompute else 0)
    plan = vbm.Plan([0, P.shape[1]], V, W, H, pair_capacity=1 << 22, pixels_per_thread=ppt, flags=flags,
                    group_lanes=8)
    img0 = torch.zeros((V, 3, H, W), device="cuda")
    plan.forward(params, cams_dev, img0)
    n_eval = torch.full((V, H, W), -1, dtype=torch.int32, device="cuda")
    n_contrib = torch.full((V, H, W), -1, dtype=torch.int32, device="cuda") if recompute else None
    plan.set_profile(None, n_eval, n_contrib)
    img1 = torch.zeros_like(img0)
    plan.forward(params, cams_dev, img1)
    plan.set_profile()
    torch.cuda.synchronize()
    assert torch.equal(img0, img1)
    st = plan_state(plan, V)
    splat, color = gpu_splats_as_oracle(st)
    ref = oraster.render(V, W, H, 16, 16, st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                         np.zeros(3))
    good = ref["margin"] > 1e-5
    assert good.mean() > 0.99
    assert np.array_equal(n_eval.cpu().numpy()[good], ref["n_eval"][good])
    nc = n_contrib.cpu().numpy() if recompute else st["n_contrib"]
    assert np.array_equal(nc[good], ref["n_contrib"][good])
    assert (ref["n_eval"] > 1).any()
    plan.close()


def _flag_pixels_of_unsafe_items(ref_fwd, gpu_rect, n_views, W, H, tile, n):
    """Pixels of tiles whose lists differ between the FP32 and FP64 projections: the tiles in
    the symmetric difference of an item's two rectangles (a radius, rectangle or culling
    decision that FP32 rounding flipped)."""
    pj = ref_fwd["proj"]
    rref = pj[:, [PJ["X0"], PJ["Y0"], PJ["X1"], PJ["Y1"]]].astype(np.int32)
    TX, TY = (W + tile[0] - 1) // tile[0], (H + tile[1] - 1) // tile[1]
    tiles = np.zeros((n_views, TY, TX), dtype=bool)
    for it in np.nonzero(np.any(rref != gpu_rect, axis=1))[0]:
        a = np.zeros((TY, TX), dtype=bool)
        b = np.zeros((TY, TX), dtype=bool)
        a[rref[it, 1]:rref[it, 3], rref[it, 0]:rref[it, 2]] = True
        b[gpu_rect[it, 1]:gpu_rect[it, 3], gpu_rect[it, 0]:gpu_rect[it, 2]] = True
        tiles[it // n] |= a ^ b
    mask = np.repeat(np.repeat(tiles, tile[1], axis=1), tile[0], axis=2)[:, :H, :W]
    return mask


def test_end_to_end_image_matches_fp64_oracle(cuda_lib):
    W, H = 128, 128
    P, cams, cams32 = scene(seed=4, n=4000, V=1, W=W, H=H)
    plan, _, _, img, _ = _forward(cuda_lib, P, cams, W, H)
    st = plan_state(plan, 1)
    ref = oraster.splat_forward(P.astype(np.float64), cams32, 16, 16)
    # excluded: pixels within 1e-5 (relative) of a compositing cut-off in FP64, and the
    # pixels of tiles whose listing an FP32 rounding of a rectangle changed; the share
    # must stay under 1% and is reported
    bad = _flag_pixels_of_unsafe_items(ref, st["rect"], 1, W, H, (16, 16), P.shape[1]) | (ref["margin"] < 1e-5)
    print("excluded pixels: %d of %d" % (bad.sum(), bad.size))
    assert bad.mean() < 0.01, bad.mean()
    err = np.abs(img - ref["img"]).transpose(1, 0, 2, 3)[:, ~bad]
    assert err.max() <= 1e-4, err.max()


@pytest.mark.parametrize("ppt,persistent,gl,seg", [(1, False, 32, 0), (2, False, 32, 0), (4, False, 32, 0),
                                                   (1, True, 32, 0), (1, False, 8, 0), (1, True, 16, 0),
                                                   (2, False, 8, 0), (4, True, 16, 0), (1, True, 16, 32),
                                                   (2, True, 8, 64), (4, True, 32, 32), (1, True, 32, -1),
                                                   (2, True, 4, 64), (1, False, 4, 0), (4, True, 4, 32)])
def test_backward_matches_oracle(cuda_lib, ppt, persistent, gl, seg):
    """seg > 0: tile lists longer than seg entries are walked by the backward as
    segments starting from the forward's checkpoints; -1: never split."""
    W, H, V = 100, 76, 2
    P, cams, cams32 = scene(seed=5, n=2000, V=V, W=W, H=H)
    n = P.shape[1]
    bg = (0.05, 0.1, 0.2)
    plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H, bg=bg, ppt=ppt, persistent=persistent,
                                              gl=gl, seg=seg)
    if seg > 0:   # the split is exercised: pixels still composite past a segment boundary
        st0 = plan_state(plan, V)
        assert (st0["n_contrib"] > seg).any()
    st = plan_state(plan, V)
    splat, color = gpu_splats_as_oracle(st)
    ref = oraster.render(V, W, H, 16, 16, st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                         np.array(bg))
    rng = np.random.default_rng(0)
    w = rng.standard_normal((V, 3, H, W)).astype(np.float32)
    wa = rng.standard_normal((V, H, W)).astype(np.float32)
    keep = ref["margin"] > 1e-5            # no gradient through pixels near a cut-off
    w *= keep[:, None]
    wa *= keep
    grad = torch.zeros_like(params)
    plan.backward(params, cams_dev, torch.from_numpy(w).cuda(), grad, dalpha=torch.from_numpy(wa).cuda(), bg=bg)
    torch.cuda.synchronize()
    st = plan_state(plan, V)
    g_ref, c_ref = oraster.render_bwd(V, W, H, 16, 16, st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                                      np.array(bg), w.astype(np.float64), wa.astype(np.float64))
    gs = st["g_splat"]
    for k in range(6):
        nrm, elt = rel_group_error(gs[k], g_ref[:, k])
        assert nrm < 1e-3 and elt < 1e-3, (k, nrm, elt)
    for k in range(3):
        nrm, elt = rel_group_error(gs[6 + k], c_ref[:, k])
        assert nrm < 1e-3 and elt < 1e-3, (k, nrm, elt)
    # chain rule to the parameters, checked on the GPU's own per-item gradients
    P64 = P.astype(np.float64)
    gfull = np.zeros((14, n))
    for v in range(V):
        sl = slice(v * n, (v + 1) * n)
        gp = oraster.project_bwd(P64, cams32[v], np.arange(n), gs[:6, sl].T.astype(np.float64))
        gfull += gp.T
        gfull[11:14] += gs[6:9, sl].astype(np.float64)
    g_gpu = grad.cpu().numpy()
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
        nrm, elt = rel_group_error(g_gpu[lo:hi], gfull[lo:hi])
        assert nrm < 1e-3 and elt < 1e-3, (lo, nrm, elt)


def test_backward_end_to_end_fp64(cuda_lib):
    """Whole backward (splats from FP32 parameters) against the FP64 oracle's gradient."""
    W, H, V = 96, 96, 2
    P, cams, cams32 = scene(seed=6, n=1500, V=V, W=W, H=H)
    plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H)
    st = plan_state(plan, V)
    ref = oraster.splat_forward(P.astype(np.float64), cams32, 16, 16)
    bad = _flag_pixels_of_unsafe_items(ref, st["rect"], V, W, H, (16, 16), P.shape[1]) | (ref["margin"] < 1e-3)
    w = np.random.default_rng(1).standard_normal((V, 3, H, W))
    w *= ~bad[:, None]
    grad = torch.zeros_like(params)
    plan.backward(params, cams_dev, torch.from_numpy(w.astype(np.float32)).cuda(), grad)
    torch.cuda.synchronize()
    gref, _, _ = oraster.splat_backward(ref, P.astype(np.float64), cams32, w)
    g = grad.cpu().numpy()
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
        nrm, elt = rel_group_error(g[lo:hi], gref[lo:hi])
        assert nrm < 1e-3 and elt < 1e-3, (lo, nrm, elt)


@pytest.mark.parametrize("persistent,seg", [(False, 0), (True, 64), (True, -1)])
def test_second_backward_of_one_forward(cuda_lib, persistent, seg):
    """Two backward calls after one forward give the same gradient (up to the atomic order
    of the splat-gradient sums): the second finds its splat-gradient records and, in
    persistent plans, its work-queue counter cleared again."""
    W, H, V = 96, 72, 2
    P, cams, _ = scene(seed=14, n=4000, V=V, W=W, H=H)
    plan, params, cams_dev, _, _ = _forward(cuda_lib, P, cams, W, H, tile=(8, 8), persistent=persistent,
                                            seg=seg, gl=8)
    if seg > 0:
        assert plan_state(plan, V)["seg_count"][0] > 0          # some lists are walked as segments
    w = torch.from_numpy(np.random.default_rng(15).standard_normal((V, 3, H, W)).astype(np.float32)).cuda()
    grads = []
    for _ in range(2):
        g = torch.zeros_like(params)
        plan.backward(params, cams_dev, w, g)
        torch.cuda.synchronize()
        grads.append(g.cpu().numpy())
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
        nrm, _ = rel_group_error(grads[1][lo:hi], grads[0][lo:hi])
        assert nrm < 1e-5, (lo, nrm)
    assert np.abs(grads[0]).max() > 0
    plan.close()


def test_per_view_calls_equal_batched_call(cuda_lib):
    W, H, V = 64, 48, 4
    P, cams, cams32 = scene(seed=7, n=1500, V=V, W=W, H=H)
    plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H)
    w = torch.from_numpy(np.random.default_rng(2).standard_normal((V, 3, H, W)).astype(np.float32)).cuda()
    g_batch = torch.zeros_like(params)
    plan.backward(params, cams_dev, w, g_batch)
    img_views = torch.zeros((V, 3, H, W), device="cuda")
    g_views = torch.zeros_like(params)
    for v in range(V):
        plan.forward(params, cams_dev, img_views, view_begin=v, view_count=1)
        plan.backward(params, cams_dev, w, g_views, view_begin=v, view_count=1, accumulate=v > 0)
    torch.cuda.synchronize()
    assert np.array_equal(img_views.cpu().numpy(), img)
    nrm, elt = rel_group_error(g_views.cpu().numpy(), g_batch.cpu().numpy())
    assert nrm < 1e-5 and elt < 1e-4


def test_uneven_multi_scene_batch(cuda_lib):
    W, H = 80, 64
    sizes = [500, 1500, 37]
    Ps = [scene(seed=10 + i, n=s, V=1, W=W, H=H)[0] for i, s in enumerate(sizes)]
    P = np.concatenate(Ps, axis=1)
    so = np.concatenate([[0], np.cumsum(sizes)])
    view_scene = [0, 1, 1, 2, 0]
    _, cams, cams32 = scene(seed=0, n=1, V=5, W=W, H=H)
    plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H, scene_offset=so, view_scene=view_scene,
                                              persistent=True, gl=8)
    ref = oraster.splat_forward(P.astype(np.float64), cams32, 16, 16, scene_offset=so, view_scene=view_scene)
    st = plan_state(plan, 5)
    assert st["n_items"] == sum(sizes[s] for s in view_scene)
    splat, color = gpu_splats_as_oracle(st)
    ref_g = oraster.render(5, W, H, 16, 16, st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                           np.zeros(3))
    good = ref_g["margin"] > 1e-5
    assert np.abs(img - ref_g["img"]).transpose(1, 0, 2, 3)[:, good].max() <= 1e-4
    # each view shows only its own scene
    for v, s in enumerate(view_scene):
        single = oraster.splat_forward(Ps[s].astype(np.float64), [cams32[v]], 16, 16)
        gd = good[v] & (single["margin"][0] > 1e-3) & (ref["margin"][v] > 1e-3)
        assert np.abs(img[v] - single["img"][0])[:, gd].max() <= 1e-3


@pytest.mark.parametrize("persistent,radix", [(False, False), (True, False), (True, True), (False, True)])
def test_capacity_overflow_is_reported(cuda_lib, persistent, radix):
    W, H = 64, 48
    P, cams, _ = scene(seed=8, n=800, V=1, W=W, H=H)
    plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H, cap=16, bg=(0.3, 0.2, 0.1),
                                              persistent=persistent, radix=radix)
    ok, need = plan.check()
    assert not ok and need > 16
    assert np.allclose(img[0, 0], 0.3) and np.allclose(img[0, 2], 0.1)
    # the backward of a call that overflowed leaves the gradient at zero
    grad = torch.zeros_like(params)
    plan.backward(params, cams_dev, torch.ones((1, 3, H, W), device="cuda"), grad)
    torch.cuda.synchronize()
    assert not grad.any()
    ok, _ = plan.check()         # the status word is cleared by the check
    assert ok


@pytest.mark.parametrize("persistent,radix", [(False, False), (True, True)])
def test_empty_and_culled_scenes(cuda_lib, persistent, radix):
    W, H = 40, 24
    bg = (0.25, 0.5, 0.75)
    P = np.zeros((14, 0), dtype=np.float32)
    _, cams, _ = scene(seed=0, n=1, V=2, W=W, H=H)
    plan, _, _, img, alpha = _forward(cuda_lib, P, cams, W, H, bg=bg, persistent=persistent, radix=radix)
    assert np.array_equal(img[:, 0], np.full((2, H, W), 0.25, dtype=np.float32)) and alpha.max() == 0
    # every Gaussian behind the camera (camera-space z = -5)
    P, cams, _ = scene(seed=9, n=50, V=1, W=W, H=H)
    R, t = np.asarray(cams[0]["R"]), np.asarray(cams[0]["t"])
    P[0:3] = (R.T @ (np.array([0.0, 0.0, -5.0]) - t))[:, None]
    plan, _, _, img, alpha = _forward(cuda_lib, P, cams, W, H, bg=bg, persistent=persistent, radix=radix)
    assert alpha.max() == 0 and np.allclose(img[0, 2], 0.75)


@pytest.mark.parametrize("persistent,gl,seg", [(False, 32, 0), (True, 32, 0), (True, 8, 0), (True, 16, 32),
                                              (True, 32, 64), (True, 16, "radix")])
def test_recompute_mode_matches_stored_state(cuda_lib, persistent, gl, seg):
    """VBM_PLAN_RECOMPUTE keeps no per-pixel state; the backward replays the forward's
    decisions (for lists split into segments of seg entries, it reads the final state the
    forward kept for those tiles only), so images are bit-identical and gradients equal
    up to atomic order and FP32 rounding."""
    vbm = cuda_lib
    W, H, V = 96, 80, 3
    P, cams, cams32 = scene(seed=12, n=2000, V=V, W=W, H=H)
    params, cams_dev = to_device(P, cams)
    w = torch.from_numpy(np.random.default_rng(3).standard_normal((V, 3, H, W)).astype(np.float32)).cuda()
    out = []
    radix = seg == "radix"        # radix-sort ordering, default segments
    seg = 0 if radix else seg
    for flags in (0, vbm.PLAN_RECOMPUTE):
        fl = flags | (vbm.PLAN_PERSISTENT if persistent else 0) | (vbm.PLAN_RADIX_SORT if radix else 0)
        plan = vbm.Plan([0, P.shape[1]], V, W, H, pair_capacity=1 << 22, flags=fl, tile_w=8, tile_h=8,
                        pixels_per_thread=1, group_lanes=gl, segment_len=seg)
        img = torch.zeros((V, 3, H, W), device="cuda")
        plan.forward(params, cams_dev, img)
        if seg > 0 and not flags:   # the split is exercised
            st = plan_state(plan, V)
            assert (st["n_contrib"] > seg).any()
        grad = torch.zeros_like(params)
        plan.backward(params, cams_dev, w, grad)
        torch.cuda.synchronize()
        out.append((img.cpu().numpy(), grad.cpu().numpy()))
        if flags:
            assert plan.buffers().T_final is None
    assert np.array_equal(out[0][0], out[1][0])
    nrm, elt = rel_group_error(out[1][1], out[0][1])
    assert nrm < 1e-5 and elt < 1e-4, (nrm, elt)


@pytest.mark.parametrize("tile,ppt,gl", [((8, 8), 1, 16), ((8, 8), 2, 8), ((8, 8), 1, 32), ((8, 4), 1, 16)])
def test_segmented_backward_equals_whole_walk(cuda_lib, tile, ppt, gl):
    """A cluster of faint splats gives tiles lists of several hundred entries along
    which the pixels keep compositing.  Walking such lists as segments of 32 or 64
    entries, each started from the forward's checkpoint (transmittance, colour still to
    come), must leave the image unchanged bit for bit and give the gradients of the whole
    walk up to FP32 rounding, and the oracle's (on the GPU's splats) within the bars."""
    from vbm_inputs.gaussians import random_gaussians
    from vbm_inputs import orbit_cameras
    from vbm_inputs.cameras import cameras_as_float32
    G, W, H, V = 32, 96, 72, 2
    P = random_gaussians(3000, 12.0, 20.0, seed=31, scale_range=(0.3, 1.2),
                         opacity_logit_range=(-4.5, -2.5)).astype(np.float32)
    cams = orbit_cameras((G, G, G), V, W, H)
    bg = (0.1, 0.05, 0.2)
    rng = np.random.default_rng(4)
    w = torch.from_numpy(rng.standard_normal((V, 3, H, W)).astype(np.float32)).cuda()
    wa = torch.from_numpy(rng.standard_normal((V, H, W)).astype(np.float32)).cuda()
    out = {}
    for seg in (-1, 32, 64):
        plan, params, cams_dev, img, alpha = _forward(cuda_lib, P, cams, W, H, tile=tile, bg=bg, ppt=ppt,
                                                      persistent=True, gl=gl, seg=seg)
        grad = torch.zeros_like(params)
        plan.backward(params, cams_dev, w, grad, dalpha=wa, bg=bg)
        torch.cuda.synchronize()
        out[seg] = (img, alpha, grad.cpu().numpy(), plan_state(plan, V))
    st = out[32][3]
    lengths = st["ranges"][:, 1] - st["ranges"][:, 0]
    assert lengths.max() > 8 * 32, lengths.max()
    assert (st["n_contrib"] > 4 * 32).any()         # pixels composite across several boundaries
    # every list longer than 32 entries is split while the checkpoint pool (about two pairs
    # per item) lasts; with 8x4 tiles it runs out and the remaining long tiles are walked
    # whole: both kinds must agree with the whole walk
    units, seg_tiles, slots_asked, _ = st["seg_count"]
    n_long = int((lengths > 32).sum())
    assert seg_tiles > 0 and units >= 2 * seg_tiles
    if slots_asked > st["checkpoint_slots"]:
        assert seg_tiles < n_long, (seg_tiles, n_long)
    else:
        assert seg_tiles == n_long, (seg_tiles, n_long)
    if tile == (8, 4):
        assert slots_asked > st["checkpoint_slots"], (slots_asked, st["checkpoint_slots"])
    assert out[-1][3]["seg_count"] is None and out[-1][3]["checkpoint_slots"] == 0
    for seg in (32, 64):
        assert np.array_equal(out[seg][0], out[-1][0]) and np.array_equal(out[seg][1], out[-1][1])
        for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14)]:
            nrm, elt = rel_group_error(out[seg][2][lo:hi], out[-1][2][lo:hi])
            assert nrm < 1e-4 and elt < 1e-4, (seg, lo, nrm, elt)
    # segmented walk against the FP64 oracle on the GPU's own splats
    splat, color = gpu_splats_as_oracle(st)
    ref = oraster.render(V, W, H, tile[0], tile[1], st["ranges"], st["pair_item"].astype(np.int32), splat, color,
                         np.array(bg))
    keep = ref["margin"] > 1e-5
    wk = w.cpu().numpy().astype(np.float64) * keep[:, None]
    wak = wa.cpu().numpy().astype(np.float64) * keep
    plan, params, cams_dev, _, _ = _forward(cuda_lib, P, cams, W, H, tile=tile, bg=bg, ppt=ppt, persistent=True,
                                            gl=gl, seg=32)
    grad = torch.zeros_like(params)
    plan.backward(params, cams_dev, torch.from_numpy(wk.astype(np.float32)).cuda(), grad,
                  dalpha=torch.from_numpy(wak.astype(np.float32)).cuda(), bg=bg)
    torch.cuda.synchronize()
    st = plan_state(plan, V)
    g_ref, c_ref = oraster.render_bwd(V, W, H, tile[0], tile[1], st["ranges"], st["pair_item"].astype(np.int32),
                                      splat, color, np.array(bg), wk, wak)
    gs = st["g_splat"]
    for k in range(6):
        nrm, elt = rel_group_error(gs[k], g_ref[:, k])
        assert nrm < 1e-3 and elt < 1e-3, (k, nrm, elt)
    for k in range(3):
        nrm, elt = rel_group_error(gs[6 + k], c_ref[:, k])
        assert nrm < 1e-3 and elt < 1e-3, (k, nrm, elt)


@pytest.mark.parametrize("tile,persistent", [((8, 8), True), ((16, 16), False)])
def test_radix_ordering_equals_bucketed_ordering(cuda_lib, tile, persistent):
    """The device radix sorts (items by depth, pairs stably by tile) and the bucketed
    per-tile sort give the same lists, ranges, images and (up to atomic order) gradients,
    on uneven scenes of a batch."""
    vbm = cuda_lib
    W, H = 96, 72
    P1, cams, _ = scene(seed=41, n=1800, V=3, W=W, H=H)
    P2, _, _ = scene(seed=42, n=700, V=3, W=W, H=H)
    P = np.concatenate([P1, P2], axis=1)
    so, vs = [0, P1.shape[1], P.shape[1]], [0, 1, 1]
    w = torch.from_numpy(np.random.default_rng(5).standard_normal((3, 3, H, W)).astype(np.float32)).cuda()
    out = []
    for radix in (False, True):
        plan, params, cams_dev, img, _ = _forward(cuda_lib, P, cams, W, H, tile=tile, scene_offset=so, view_scene=vs,
                                                  persistent=persistent, radix=radix)
        grad = torch.zeros_like(params)
        plan.backward(params, cams_dev, w, grad)
        torch.cuda.synchronize()
        out.append((plan_state(plan, 3), img, grad.cpu().numpy()))
        ok, need = plan.check()
        assert ok, need
    (a, ia, ga), (b, ib, gb) = out
    assert a["n_pairs"] == b["n_pairs"] > 0
    for k in ("pair_tile", "pair_item", "ranges"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(ia, ib)
    nrm, elt = rel_group_error(gb, ga)
    assert nrm < 1e-5 and elt < 1e-4, (nrm, elt)


@pytest.mark.parametrize("recompute", [False, True])
def test_backward_launch_configuration_is_its_own(cuda_lib, recompute):
    """The backward compositing kernel may run its own pixels per thread and lane groups
    (its warp regions do not depend on the forward's): gradients equal, up to atomic order
    and FP32 rounding, those of the backward in the forward's configuration."""
    vbm = cuda_lib
    W, H, V = 96, 80, 2
    P, cams, _ = scene(seed=15, n=2000, V=V, W=W, H=H)
    params, cams_dev = to_device(P, cams)
    w = torch.from_numpy(np.random.default_rng(6).standard_normal((V, 3, H, W)).astype(np.float32)).cuda()
    flags = vbm.PLAN_PERSISTENT | (vbm.PLAN_RECOMPUTE if recompute else 0)
    out = []
    for bppt, bgl in ((0, 0), (2, 8), (1, 32)):
        plan = vbm.Plan([0, P.shape[1]], V, W, H, pair_capacity=1 << 22, flags=flags, tile_w=8, tile_h=8,
                        pixels_per_thread=1, group_lanes=16, segment_len=64, bwd_pixels_per_thread=bppt,
                        bwd_group_lanes=bgl)
        img = torch.zeros((V, 3, H, W), device="cuda")
        plan.forward(params, cams_dev, img)
        grad = torch.zeros_like(params)
        plan.backward(params, cams_dev, w, grad)
        torch.cuda.synchronize()
        out.append((img.cpu().numpy(), grad.cpu().numpy()))
    for img, g in out[1:]:
        assert np.array_equal(img, out[0][0])
        nrm, elt = rel_group_error(g, out[0][1])
        assert nrm < 1e-5 and elt < 1e-4, (nrm, elt)
