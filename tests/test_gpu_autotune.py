"""The autotuner of the splatting launch configuration (tile shape, pixels per thread, lanes
per group, persistence, and for a persistent winner the per-warp list length) on a small
scene: the choice is one of the candidates, every timing is finite, and the chosen
configuration renders the same image as any other."""

import numpy as np
import pytest
import torch

from _helpers import scene, to_device

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_a_segment_length(cuda_lib):
    from paper_2601_09417_gb300 import autotune
    vbm = cuda_lib
    W, H, V = 96, 80, 2
    P, cams, _ = scene(seed=14, n=2000, V=V, W=W, H=H)
    params, cams_dev = to_device(P, cams)
    from vbm_inputs.cameras import camera_array
    recs = camera_array(cams)
    cands = [((8, 8), 1, 16, True), ((16, 16), 1, 32, False)]
    (tile, ppt, gl, pers, seg, bppt, bgl), table = autotune.autotune(params, recs, V, W, H, candidates=cands,
                                                                     use_cache=False)
    assert (tile, ppt, gl, pers) in cands
    main = [r for r in table if r.get("stage") is None]
    assert all(np.isfinite(r["ms_fwd"]) and np.isfinite(r["ms_bwd"]) for r in main)
    pairs = [r for r in table if r.get("stage") == "combination"]
    assert pairs and all(np.isfinite(r["ms_final"]) for r in pairs)
    assert (list(tile), ppt, gl, pers, bppt, bgl) in [(r["tile"], r["ppt"], r["group_lanes"], r["persistent"],
                                                       r["bwd_ppt"], r["bwd_group_lanes"]) for r in pairs]
    assert len(main) == len(cands) and all(np.isfinite(r["ms"]) and r["ms"] > 0 for r in main)
    segs = [r for r in table if r.get("stage") == "segment"]
    if pers:
        assert [r["segment_len"] for r in segs] == list(autotune.SEGMENT_LENGTHS)
        assert seg in autotune.SEGMENT_LENGTHS and all(np.isfinite(r["ms"]) for r in segs)
    else:
        assert seg == 0 and not segs
    # the tuned plan renders the image of an untuned one bit for bit
    imgs = []
    for t, p_, g_, per, s_, bp, bg in ((tile, ppt, gl, pers, seg, bppt, bgl), ((16, 16), 1, 32, False, 0, 0, 0)):
        plan = vbm.Plan([0, P.shape[1]], V, W, H, tile_w=t[0], tile_h=t[1], pair_capacity=1 << 22,
                        pixels_per_thread=p_, group_lanes=g_, flags=vbm.PLAN_PERSISTENT if per else 0,
                        segment_len=s_, bwd_pixels_per_thread=bp, bwd_group_lanes=bg)
        img = torch.zeros((V, 3, H, W), device="cuda")
        plan.forward(params, cams_dev, img)
        torch.cuda.synchronize()
        imgs.append(img.cpu().numpy())
        plan.close()
    assert np.abs(imgs[0] - imgs[1]).max() <= 1e-5
