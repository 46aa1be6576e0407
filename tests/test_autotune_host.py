"""Host logic without a GPU: the autotuner's candidate list and the configuration tuples
handed to its timing trials (segment length last, pair capacity in its place), and the
fine-tuner's choice to recompute per-pixel state when storing it would crowd memory."""

import pytest

pytest.importorskip("torch")

from paper_2601_09417_gb300 import autotune as at


def test_candidates_respect_region_rows():
    assert len(at.CANDIDATES) == len(set(at.CANDIDATES))
    for tile, ppt, gl, pers in at.CANDIDATES:
        assert tile[1] % (4 * ppt) == 0 and gl in (4, 8, 16, 32)
    assert {gl for _, _, gl, _ in at.CANDIDATES} == {4, 8, 16, 32}
    assert -1 in at.SEGMENT_LENGTHS and all(s == -1 or s % 32 == 0 for s in at.SEGMENT_LENGTHS)


def test_retime_passes_segment_length_and_capacity(monkeypatch):
    made = []

    class Trial:
        def __init__(self, params, cams, n_views, W, H, so, vs, tile, ppt, gl, persistent, cap, segment_len=0,
                     bwd_ppt=0, bwd_gl=0, recompute=False):
            made.append((tile, ppt, gl, persistent, cap, segment_len, bwd_ppt, bwd_gl, recompute))

        def run(self, iters):
            return [1.0 + len(made)] * iters

        def close(self):
            return True, 0

    monkeypatch.setattr(at, "_Trial", Trial)
    out = at.retime(None, None, 2, 8, 8, [0, 1], None,
                    [((8, 8), 1, 16, True), ((16, 8), 2, 8, True, 128), ((8, 8), 1, 16, True, 64, 2, 8)], 12345,
                    rounds=2, iters=1, recompute=True)
    assert made == [((8, 8), 1, 16, True, 12345, 0, 0, 0, True), ((16, 8), 2, 8, True, 12345, 128, 0, 0, True),
                    ((8, 8), 1, 16, True, 12345, 64, 2, 8, True)]
    assert len(out) == 3


def test_recompute_is_chosen_when_state_would_crowd_memory():
    from paper_2601_09417_gb300.finetune import STATE_MEMORY_SHARE, choose_recompute
    px = 8 * 1024 * 1024                       # 8 views of 1024^2: 64 MiB of state
    assert not choose_recompute(px, 200 << 30)  # a mostly free GB300
    assert choose_recompute(px, 1 << 30)        # 1 GiB free: 64 MiB is above the share
    edge = 8 * px / STATE_MEMORY_SHARE
    assert not choose_recompute(px, edge) and choose_recompute(px, edge - 1)
