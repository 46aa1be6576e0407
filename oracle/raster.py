"""ctypes wrapper around oracle/raster_ref.c (FP64 splatting oracle; test infrastructure only).

The C file is compiled with gcc into oracle/_build/ on first use (or by
__graft_entry__.build()).  Floating-point contraction is disabled so the
oracle gives the same bits on x86-64 and aarch64.

Items: the unit of projection is one (view, Gaussian) pair.  For a single
scene every view sees all N Gaussians and item = view * N + g.  For several
scenes (uneven batches) view v sees the Gaussians [off[s], off[s+1]) of its
scene s = view_scene[v], and items are numbered view by view.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raster_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc_raster.so")

NPROJ = 18
PJ = dict(U=0, V=1, A=2, B=3, C=4, OPAC=5, DEPTH=6, RADIUS=7, X0=8, Y0=9, X1=10, Y1=11,
          TOUCHED=12, M_RADIUS=13, M_RECT=14, M_CULL=15, M_CLAMP=16, M_OPAC=17)

_lib = None


def build_library(force=False):
    """Compile raster_ref.c into a shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        P = ctypes.c_void_p
        I64, I32 = ctypes.c_int64, ctypes.c_int
        lib.orc_project.argtypes = [I64, P, P, I64, P, I32, I32, P]
        lib.orc_bin_sort.argtypes = [I64, P, P, P, I32, I32, I32, I64, P, P, P, P, P, I32, I32, I32, I32]
        lib.orc_tile_min_q.argtypes = [ctypes.c_double] * 9
        lib.orc_tile_min_q.restype = ctypes.c_double
        lib.orc_tile_min_q_f32.argtypes = [ctypes.c_float] * 11
        lib.orc_tile_min_q_f32.restype = ctypes.c_float
        lib.orc_bin_sort.restype = I64
        lib.orc_render.argtypes = [I32, I32, I32, I32, I32, P, P, P, P, P, P, P, P, P, P, P]
        lib.orc_render_bwd.argtypes = [I32, I32, I32, I32, I32, P, P, P, P, P, P, P, P, P, I64]
        lib.orc_render_brute.argtypes = [I32, I32, I32, I32, I32, I64, P, P, P, P, P, P, P, P]
        lib.orc_project_bwd_items.argtypes = [I64, P, P, I64, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera_record(cam):
    """19-double camera record: R[9] t[3] fx fy cx cy znear width height."""
    rec = np.zeros(19)
    rec[0:9] = np.asarray(cam["R"], dtype=np.float64).reshape(9)
    rec[9:12] = np.asarray(cam["t"], dtype=np.float64)
    rec[12:19] = [cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["znear"], cam["width"], cam["height"]]
    return rec


def project(P, cam, gidx, tile_w, tile_h):
    """Per-item projection records (n_items, NPROJ) for Gaussians gidx seen by cam."""
    lib = _load()
    P = _c64(P)
    gidx = np.ascontiguousarray(gidx, dtype=np.int64)
    out = np.zeros((gidx.size, NPROJ))
    lib.orc_project(gidx.size, _p(gidx), _p(P), P.shape[1], _p(camera_record(cam)),
                    tile_w, tile_h, _p(out))
    return out


def splat_records(splat, dtype=np.float64):
    """Binning records [n][8] = u v A B C B/C B/A tau from splats (n, 6) = u v A B C opacity,
    tau = 2 (ln(255 o) + 1e-3), in the given precision (float32: each value rounded as a
    float32 implementation holds it, B/C and B/A divided in float32)."""
    sp = np.asarray(splat, dtype=np.float64)
    if dtype == np.float32:
        f = sp.astype(np.float32)
        out = np.zeros((sp.shape[0], 8), dtype=np.float32)
        out[:, 0:5] = f[:, 0:5]
        with np.errstate(divide="ignore", invalid="ignore"):
            out[:, 5] = np.where(f[:, 4] != 0, f[:, 3] / f[:, 4], np.float32(0))
            out[:, 6] = np.where(f[:, 2] != 0, f[:, 3] / f[:, 2], np.float32(0))
        return out
    out = np.zeros((sp.shape[0], 8))
    out[:, 0:5] = sp[:, 0:5]
    with np.errstate(divide="ignore", invalid="ignore"):
        out[:, 5] = np.where(sp[:, 4] != 0, sp[:, 3] / sp[:, 4], 0.0)
        out[:, 6] = np.where(sp[:, 2] != 0, sp[:, 3] / sp[:, 2], 0.0)
        out[:, 7] = np.where(sp[:, 5] > 0, 2.0 * (np.log(255.0 * np.maximum(sp[:, 5], 1e-300)) + 1e-3), -1.0)
    return out


def tile_min_q(u, v, A, B, C, x0, x1, y0, y1):
    """Smallest A dx^2 + 2 B dx dy + C dy^2 over the rectangle [x0, x1] x [y0, y1] (FP64)."""
    return _load().orc_tile_min_q(u, v, A, B, C, x0, x1, y0, y1)


def tile_min_q_f32(u, v, A, B, C, bc, ba, x0, x1, y0, y1):
    """The float32 copy of tile_min_q (the edges facing the centre only), every argument
    rounded to float32 first; bc = B / C and ba = B / A as the caller rounded them."""
    return float(np.float32(_load().orc_tile_min_q_f32(*[float(np.float32(a)) for a in
                                                          (u, v, A, B, C, bc, ba, x0, x1, y0, y1)])))


def bin_sort(view_of, rect, depth, TX, TY, n_views, capacity=None, splat64=None, splat32=None, tile=(16, 16),
             image=None):
    """Sorted (tiles, items) pair lists and per-tile ranges (n_tiles, 2).  With splat64 or
    splat32 (binning records from splat_records) only the tiles passing the exact tile
    test are listed; image = (W, H) is then required."""
    lib = _load()
    view_of = np.ascontiguousarray(view_of, dtype=np.int32)
    rect = np.ascontiguousarray(rect, dtype=np.int32).reshape(-1, 4)
    depth = _c64(depth)
    total = int(((rect[:, 2] - rect[:, 0]).astype(np.int64) * (rect[:, 3] - rect[:, 1])).sum())
    cap = total if capacity is None else capacity
    tiles = np.zeros(max(total, 1), dtype=np.int64)
    items = np.zeros(max(total, 1), dtype=np.int32)
    ranges = np.zeros((n_views * TY * TX, 2), dtype=np.int32)
    sp64 = None if splat64 is None else np.ascontiguousarray(splat64, dtype=np.float64)
    sp32 = None if splat32 is None else np.ascontiguousarray(splat32, dtype=np.float32)
    W, H = image if image is not None else (0, 0)
    if (sp64 is not None or sp32 is not None) and image is None:
        raise ValueError("image size needed for the tile test")
    n = lib.orc_bin_sort(view_of.size, _p(view_of), _p(rect), _p(depth), TX, TY, n_views, cap,
                         _p(tiles), _p(items), _p(ranges), None if sp64 is None else _p(sp64),
                         None if sp32 is None else _p(sp32), tile[0], tile[1], W, H)
    if n < 0:
        raise OverflowError("pair capacity exceeded")
    return tiles[:n], items[:n], ranges


def render(n_views, W, H, tile_w, tile_h, ranges, items, splat, color, bg):
    lib = _load()
    ranges = np.ascontiguousarray(ranges, dtype=np.int32)
    items = np.ascontiguousarray(items, dtype=np.int32)
    splat, color, bg = _c64(splat), _c64(color), _c64(bg)
    img = np.zeros((n_views, 3, H, W))
    T = np.zeros((n_views, H, W))
    nc = np.zeros((n_views, H, W), dtype=np.int32)
    ne = np.zeros((n_views, H, W), dtype=np.int32)
    margin = np.zeros((n_views, H, W))
    nb = np.zeros((n_views, H, W), dtype=np.int32)
    lib.orc_render(n_views, W, H, tile_w, tile_h, _p(ranges), _p(items), _p(splat), _p(color), _p(bg),
                   _p(img), _p(T), _p(nc), _p(ne), _p(margin), _p(nb))
    return dict(img=img, T_final=T, n_contrib=nc, n_eval=ne, margin=margin, n_blend=nb)


def render_bwd(n_views, W, H, tile_w, tile_h, ranges, items, splat, color, bg, dL_dimg, dL_dalpha=None):
    lib = _load()
    ranges = np.ascontiguousarray(ranges, dtype=np.int32)
    items = np.ascontiguousarray(items, dtype=np.int32)
    splat, color, bg, dL_dimg = _c64(splat), _c64(color), _c64(bg), _c64(dL_dimg)
    n_items = splat.shape[0]
    g_splat = np.zeros((n_items, 6))
    g_color = np.zeros((n_items, 3))
    max_list = int((ranges[:, 1] - ranges[:, 0]).max()) if ranges.size else 0
    da = None if dL_dalpha is None else _c64(dL_dalpha)
    lib.orc_render_bwd(n_views, W, H, tile_w, tile_h, _p(ranges), _p(items), _p(splat), _p(color), _p(bg),
                       _p(dL_dimg), None if da is None else _p(da), _p(g_splat), _p(g_color), max_list)
    return g_splat, g_color


def render_brute(n_views, W, H, tile_w, tile_h, view_of, rect, depth, splat, color, bg):
    lib = _load()
    view_of = np.ascontiguousarray(view_of, dtype=np.int32)
    rect = np.ascontiguousarray(rect, dtype=np.int32).reshape(-1, 4)
    depth, splat, color, bg = _c64(depth), _c64(splat), _c64(color), _c64(bg)
    img = np.zeros((n_views, 3, H, W))
    T = np.zeros((n_views, H, W))
    lib.orc_render_brute(n_views, W, H, tile_w, tile_h, view_of.size, _p(view_of), _p(rect), _p(depth),
                         _p(splat), _p(color), _p(bg), _p(img), _p(T))
    return img, T


def project_bwd(P, cam, gidx, g_splat):
    """Per-item parameter gradients (n_items, 14) from per-item splat gradients."""
    lib = _load()
    P = _c64(P)
    gidx = np.ascontiguousarray(gidx, dtype=np.int64)
    g_splat = _c64(g_splat)
    out = np.zeros((gidx.size, 14))
    lib.orc_project_bwd_items(gidx.size, _p(gidx), _p(P), P.shape[1], _p(camera_record(cam)),
                              _p(g_splat), _p(out))
    return out


# ------------------------------------------------------------------ scenes

def items_of(n_gauss, n_views, scene_offset=None, view_scene=None):
    """(view_of_item, gaussian_of_item) for a batch (see module docstring)."""
    if scene_offset is None:
        view_of = np.repeat(np.arange(n_views, dtype=np.int32), n_gauss)
        g_of = np.tile(np.arange(n_gauss, dtype=np.int64), n_views)
        return view_of, g_of
    vs, gs = [], []
    for v in range(n_views):
        s = view_scene[v]
        lo, hi = scene_offset[s], scene_offset[s + 1]
        vs.append(np.full(hi - lo, v, dtype=np.int32))
        gs.append(np.arange(lo, hi, dtype=np.int64))
    return np.concatenate(vs), np.concatenate(gs)


def splat_forward(P, cams, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0), scene_offset=None, view_scene=None,
                  timings=None):
    """Full FP64 forward for a batch of views: projection, binning, compositing.  With a
    dict `timings`, the wall time of each phase (project, bin_sort, render) is added to it."""
    P = _c64(P)
    n = P.shape[1]
    V = len(cams)
    W, H = cams[0]["width"], cams[0]["height"]
    TX, TY = (W + tile_w - 1) // tile_w, (H + tile_h - 1) // tile_h
    clock = _PhaseClock(timings)
    view_of, g_of = items_of(n, V, scene_offset, view_scene)
    proj = np.zeros((view_of.size, NPROJ))
    for v in range(V):
        sel = view_of == v
        proj[sel] = project(P, cams[v], g_of[sel], tile_w, tile_h)
    rect = proj[:, [PJ["X0"], PJ["Y0"], PJ["X1"], PJ["Y1"]]].astype(np.int32)
    splat = proj[:, [PJ["U"], PJ["V"], PJ["A"], PJ["B"], PJ["C"], PJ["OPAC"]]]
    clock.lap("project")
    tiles, items, ranges = bin_sort(view_of, rect, proj[:, PJ["DEPTH"]], TX, TY, V,
                                    splat64=splat_records(splat), tile=(tile_w, tile_h), image=(W, H))
    clock.lap("bin_sort")
    color = P[11:14, g_of].T
    bg = np.asarray(bg, dtype=np.float64)
    out = render(V, W, H, tile_w, tile_h, ranges, items, splat, color, bg)
    clock.lap("render")
    out.update(proj=proj, rect=rect, tiles=tiles, items=items, ranges=ranges, splat=splat, color=color,
               view_of=view_of, g_of=g_of, W=W, H=H, tile_w=tile_w, tile_h=tile_h, bg=bg)
    return out


def splat_backward(fwd, P, cams, dL_dimg, dL_dalpha=None, timings=None):
    """FP64 gradient P[14][N] of a loss with image gradient dL_dimg (V, 3, H, W).  With a
    dict `timings`, the wall time of each phase (render_bwd, project_bwd) is added to it."""
    P = _c64(P)
    n = P.shape[1]
    clock = _PhaseClock(timings)
    g_splat, g_color = render_bwd(len(cams), fwd["W"], fwd["H"], fwd["tile_w"], fwd["tile_h"],
                                  fwd["ranges"], fwd["items"], fwd["splat"], fwd["color"], fwd["bg"],
                                  dL_dimg, dL_dalpha)
    clock.lap("render_bwd")
    grad = np.zeros((14, n))
    view_of, g_of = fwd["view_of"], fwd["g_of"]
    for v in range(len(cams)):
        sel = np.nonzero(view_of == v)[0]
        gp = project_bwd(P, cams[v], g_of[sel], g_splat[sel])
        np.add.at(grad.T, g_of[sel], gp)
    np.add.at(grad[11:14].T, g_of, g_color)
    clock.lap("project_bwd")
    return grad, g_splat, g_color


class _PhaseClock:
    """Adds the wall time since the previous lap to timings[name] (no-op without a dict)."""

    def __init__(self, timings):
        import time
        self._now = time.perf_counter
        self.timings = timings
        self.t = self._now()

    def lap(self, name):
        if self.timings is None:
            return
        t = self._now()
        self.timings[name] = self.timings.get(name, 0.0) + (t - self.t)
        self.t = t
