"""Shared helpers of the parity tests: seeded scenes, device-buffer readers and the
oracle's transition banks (cached: the five-level bior4.4 bank takes ~25 s)."""

import functools

import numpy as np

from vbm_inputs import gaussians_in_view, orbit_cameras
from vbm_inputs.cameras import camera_array, cameras_as_float32

@functools.lru_cache(maxsize=None)
def _oracle_bank_cached(levels, wavelet):
    from oracle import bank as obank
    return tuple(obank.build_bank(levels, "bior4.4" if wavelet == 0 else "haar"))


def oracle_bank(levels, wavelet=0, ablation=0):
    """The oracle's FP64 bank for `levels` (wavelet 0 bior4.4, 1 Haar); ablation flags
    1 (isotropic covariance) and 2 (unit weight) as in vbm_bank_ablate."""
    from oracle import bank as obank
    entries = [dict(e) for e in _oracle_bank_cached(levels, wavelet)]
    if ablation:
        entries = obank.ablate(entries, isotropic=bool(ablation & 1), unit_weight=bool(ablation & 2))
    return entries


def read_device(ptr, shape, dtype):
    """Copy device memory at a raw pointer into a numpy array."""
    from paper_2601_09417_gb300 import vbm
    if int(np.prod(shape)) == 0:
        return np.zeros(shape, dtype=dtype)
    return vbm.device_tensor(ptr, shape, dtype).cpu().numpy().copy()


def scene(seed=0, n=2000, G=32, V=2, W=100, H=76, **kw):
    """Random Gaussians (float32) inside a G^3 box and an orbit of V cameras."""
    P = gaussians_in_view(n, G, seed=seed, **kw).astype(np.float32)
    cams = orbit_cameras((G, G, G), V, W, H)
    return P, cams, cameras_as_float32(cams)


def to_device(P, cams, device="cuda"):
    import torch
    from paper_2601_09417_gb300 import vbm
    return torch.from_numpy(np.ascontiguousarray(P)).to(device), vbm.cameras_to_device(camera_array(cams), device)


def split_records(rec):
    """The fields of a plan's per-item splat records ([n][16] float32, one 64-byte line
    each: u v A B | r g b opacity | half-widths, B/C, B/A | C, tau, depth, radius (int32 bits))."""
    return dict(geo=np.ascontiguousarray(rec[:, 0:4]), col=np.ascontiguousarray(rec[:, 4:8]),
                cull=np.ascontiguousarray(rec[:, 8:12]), conic_c=np.ascontiguousarray(rec[:, 12]),
                tau=np.ascontiguousarray(rec[:, 13]), depth=np.ascontiguousarray(rec[:, 14]),
                radius=np.ascontiguousarray(rec[:, 15]).view(np.int32))


def split_place(place):
    """A plan's per-item placement records ([n][4] uint32: x0 | x1 << 16, y0 | y1 << 16,
    listed-tile word, depth bits) as the tile rectangle [n][4] = x0 y0 x1 y1 (int32), the
    listed-tile words and the depths."""
    place = np.asarray(place, dtype=np.uint32)
    rect = np.stack([place[:, 0] & 0xFFFF, place[:, 1] & 0xFFFF, place[:, 0] >> 16, place[:, 1] >> 16],
                    axis=1).astype(np.int32)
    return dict(rect=rect, listed=np.ascontiguousarray(place[:, 2]),
                place_depth=np.ascontiguousarray(place[:, 3]).view(np.float32))


def plan_state(plan, n_views):
    """Numpy copies of a plan's buffers after a forward (and backward) call."""
    b = plan.buffers()
    n = b.n_items
    st = dict(n_items=n)
    rec = read_device(b.rec, (n, 16), np.float32)
    st.update(split_records(rec))
    st.update(split_place(read_device(b.place, (n, 4), np.uint32)))
    n_pairs = int(read_device(b.n_pairs, (1,), np.int64)[0])
    st["n_pairs"] = n_pairs
    st["pair_tile"] = read_device(b.pair_tile, (n_pairs,), np.uint32)
    st["pair_item"] = read_device(b.pair_item, (n_pairs,), np.uint32)
    TX = (plan.width + plan.tile_w - 1) // plan.tile_w
    TY = (plan.height + plan.tile_h - 1) // plan.tile_h
    st["ranges"] = read_device(b.ranges, (n_views * TX * TY, 2), np.int32)
    if b.T_final:
        st["T_final"] = read_device(b.T_final, (plan.n_views, plan.height, plan.width), np.float32)
        st["n_contrib"] = read_device(b.n_contrib, (plan.n_views, plan.height, plan.width), np.int32)
    st["g_splat"] = np.ascontiguousarray(read_device(b.g_splat, (n, 12), np.float32)[:, :9].T)
    st["seg_count"] = read_device(b.seg_count, (4,), np.int32) if b.seg_count else None
    st["checkpoint_slots"] = int(b.checkpoint_slots)
    return st


def gpu_binning_records(st, items=None):
    """The GPU's float32 binning records [n][8] = u v A B C B/C B/A tau of a plan state."""
    sel = slice(None) if items is None else items
    return np.stack([st["geo"][sel, 0], st["geo"][sel, 1], st["geo"][sel, 2], st["geo"][sel, 3],
                     st["conic_c"][sel], st["cull"][sel, 2], st["cull"][sel, 3], st["tau"][sel]],
                    axis=1).astype(np.float32)


def gpu_splats_as_oracle(st):
    """GPU per-item splat records as the oracle's (n, 6) u v A B C opacity and (n, 3) colour."""
    g = st["geo"].astype(np.float64)
    splat = np.stack([g[:, 0], g[:, 1], g[:, 2], g[:, 3], st["conic_c"].astype(np.float64),
                      st["col"][:, 3].astype(np.float64)], axis=1)
    return splat, st["col"][:, :3].astype(np.float64)


def rel_group_error(g, ref):
    """(norm-wise relative error, worst element error / (|ref| + rms(ref)))."""
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    nrm = np.linalg.norm(ref)
    if nrm == 0:
        return float(np.linalg.norm(g)), float(np.abs(g).max(initial=0.0))
    rms = np.sqrt(np.mean(ref * ref))
    return float(np.linalg.norm(g - ref) / nrm), float((np.abs(g - ref) / (np.abs(ref) + rms)).max())
