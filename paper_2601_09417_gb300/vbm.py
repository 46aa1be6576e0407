"""ctypes binding of libvbm (include/vbm.h): argument marshalling only.

Every function here forwards torch tensors (device pointers) and the current
CUDA stream to the C ABI; all arithmetic happens in the library's kernels.
If the library is missing the binding raises: there is no fallback path.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvbm.so")

VBM_OK, VBM_ERR_ARG, VBM_ERR_CAPACITY, VBM_ERR_CUDA, VBM_ERR_TIMEOUT, VBM_ERR_NOMEM, VBM_ERR_NUMERIC = range(7)
PLAN_RECOMPUTE = 1
PLAN_PERSISTENT = 2
PLAN_RADIX_SORT = 4

EXPORTED = ["vbm_last_error", "vbm_version", "vbm_bank_build", "vbm_tf_apply", "vbm_dwt3d",
            "vbm_build_workspace_size", "vbm_build", "vbm_render_dvr", "vbm_plan_create",
            "vbm_plan_destroy", "vbm_plan_check", "vbm_raster_fwd", "vbm_raster_bwd",
            "vbm_plan_get_buffers", "vbm_loss_workspace_size", "vbm_loss", "vbm_adam",
            "vbm_kernel_launches", "vbm_plan_set_profile", "vbm_loss_static", "vbm_bank_ablate",
            "vbm_peak_probe", "vbm_raster_bwd_adam"]


class VbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("vbm error %d: %s" % (status, msg))
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class TF(ctypes.Structure):
    _fields_ = [("n_knots", ctypes.c_int32), ("x", ctypes.c_float * 16), ("rgba", (ctypes.c_float * 4) * 16)]


class BankEntry(ctypes.Structure):
    _fields_ = [("j", ctypes.c_int32), ("o", ctypes.c_int32 * 3), ("u", ctypes.c_double * 3),
                ("cov", ctypes.c_double * 6), ("w", ctypes.c_double), ("log_scale", ctypes.c_float * 3),
                ("quat", ctypes.c_float * 4)]


class Bank(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("wavelet", ctypes.c_int32), ("n_sub", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("tau", ctypes.c_double), ("ridge_rel", ctypes.c_double),
                ("sub", BankEntry * 64)]


class Select(ctypes.Structure):
    _fields_ = [("alpha_E", ctypes.c_double), ("beta_N", ctypes.c_double), ("lambda_mad", ctypes.c_double),
                ("K_tot", ctypes.c_int64), ("min_per_band", ctypes.c_int32), ("energy_comp", ctypes.c_int32)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("n_scenes", ctypes.c_int32), ("n_views", ctypes.c_int32),
                ("scene_offset", ctypes.POINTER(ctypes.c_int64)), ("view_scene", ctypes.POINTER(ctypes.c_int32)),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("pair_capacity", ctypes.c_int64), ("flags", ctypes.c_int32),
                ("pixels_per_thread", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("segment_len", ctypes.c_int32), ("bwd_pixels_per_thread", ctypes.c_int32),
                ("bwd_group_lanes", ctypes.c_int32)]


class PlanBuffers(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int64)] + [(name, ctypes.c_void_p) for name in
                                                ("rec", "place", "pair_tile", "pair_item", "ranges",
                                                 "n_pairs", "T_final", "n_contrib", "g_splat", "seg_count")] + \
        [("checkpoint_slots", ctypes.c_int64)]


_lib = None


def load():
    """Load libvbm.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libvbm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    V, I32, I64, F32, F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
    S = ctypes.c_size_t
    sig = {
        "vbm_last_error": (ctypes.c_char_p, []),
        "vbm_version": (ctypes.c_int, []),
        "vbm_bank_build": (I32, [I32, I32, F64, F64, ctypes.POINTER(Bank)]),
        "vbm_bank_ablate": (I32, [ctypes.POINTER(Bank), I32]),
        "vbm_tf_apply": (I32, [V, I64, ctypes.POINTER(TF), V, V]),
        "vbm_dwt3d": (I32, [V, I32, ctypes.POINTER(ctypes.c_int * 3), I32, I32, V, V]),
        "vbm_build_workspace_size": (I32, [ctypes.POINTER(ctypes.c_int * 3), I32, ctypes.POINTER(S)]),
        "vbm_build": (I32, [V, ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(TF), ctypes.POINTER(Bank),
                            ctypes.POINTER(Select), V, I64, ctypes.POINTER(I64), V, V, V, S, V]),
        "vbm_render_dvr": (I32, [V, ctypes.POINTER(ctypes.c_int * 3), ctypes.POINTER(TF), V, I32, I32, I32, F32,
                                 V, V]),
        "vbm_plan_create": (I32, [ctypes.POINTER(PlanDesc), ctypes.POINTER(V)]),
        "vbm_plan_destroy": (I32, [V]),
        "vbm_plan_check": (I32, [V, V, ctypes.POINTER(I64)]),
        "vbm_raster_fwd": (I32, [V, V, I64, V, I32, I32, ctypes.POINTER(F32 * 3), V, V, V]),
        "vbm_raster_bwd": (I32, [V, V, I64, V, I32, I32, ctypes.POINTER(F32 * 3), V, V, V, I32, V]),
        "vbm_plan_get_buffers": (I32, [V, ctypes.POINTER(PlanBuffers)]),
        "vbm_loss_workspace_size": (I32, [I32, I32, I32, ctypes.POINTER(S)]),
        "vbm_loss": (I32, [V, V, I32, I32, I32, F32, F64, V, I32, V, V, S, V]),
        "vbm_adam": (I32, [V, V, V, V, I64, I64, V, ctypes.POINTER(F32 * 5), F32, F32, F32, V, V]),
        "vbm_raster_bwd_adam": (I32, [V, V, I64, V, I32, I32, ctypes.POINTER(F32 * 3), V, V, V, V, I64, V,
                                      ctypes.POINTER(F32 * 5), F32, F32, F32, V, V]),
        "vbm_kernel_launches": (I64, []),
        "vbm_loss_static": (I32, [V, V, I32, I32, I32, F32, F64, V, I32, V, V]),
        "vbm_plan_set_profile": (I32, [V, I32, ctypes.POINTER(V), V, V]),
        "vbm_peak_probe": (I32, [I32, I32, I32, V, ctypes.POINTER(F64), V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != VBM_OK:
        raise VbmError(status, load().vbm_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dims(dims):
    return (ctypes.c_int * 3)(*[int(d) for d in dims])


# ----------------------------------------------------------------- structs

def make_tf(knots_x, knots_rgba):
    tf = TF()
    n = len(knots_x)
    if not 2 <= n <= 16:
        raise ValueError("2..16 knots")
    tf.n_knots = n
    for i in range(n):
        tf.x[i] = float(knots_x[i])
        for c in range(4):
            tf.rgba[i][c] = float(knots_rgba[i][c])
    return tf


def make_select(K_tot, alpha_E=0.5, beta_N=0.5, lambda_mad=3.0, min_per_band=10, energy_comp=True):
    return Select(alpha_E, beta_N, lambda_mad, int(K_tot), int(min_per_band), int(bool(energy_comp)))


def cameras_to_device(cam_records, device="cuda"):
    """Copy packed 80-byte camera records (numpy structured array) to the device."""
    import torch
    raw = np.ascontiguousarray(cam_records).view(np.uint8).reshape(-1)
    return torch.from_numpy(raw.copy()).to(device)


_TYPESTR = {np.dtype(np.float32): "<f4", np.dtype(np.int32): "<i4", np.dtype(np.uint32): "<u4",
            np.dtype(np.int64): "<i8", np.dtype(np.float64): "<f8", np.dtype(np.uint8): "|u1"}


class _DeviceArray:
    def __init__(self, ptr, shape, dtype):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape),
                                         "typestr": _TYPESTR[np.dtype(dtype)], "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_tensor(ptr, shape, dtype):
    """A torch tensor aliasing library-owned device memory (e.g. plan buffers); no copy."""
    import torch
    return torch.as_tensor(_DeviceArray(ptr, shape, dtype), device="cuda")


# -------------------------------------------------------------------- API

def version():
    return load().vbm_version()


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load().vbm_kernel_launches())


def bank_build(levels, wavelet=0, tau=0.1, ridge_rel=1e-6):
    bank = Bank()
    _check(load().vbm_bank_build(levels, wavelet, tau, ridge_rel, ctypes.byref(bank)))
    return bank


BANK_ISOTROPIC = 1
BANK_UNIT_WEIGHT = 2


def bank_ablate(bank, flags):
    """Apply ablation flags (BANK_ISOTROPIC, BANK_UNIT_WEIGHT) to a bank in place."""
    _check(load().vbm_bank_ablate(ctypes.byref(bank), int(flags)))
    return bank


def bank_to_dicts(bank):
    out = []
    for i in range(bank.n_sub):
        e = bank.sub[i]
        c = list(e.cov)
        cov = np.array([[c[0], c[3], c[4]], [c[3], c[1], c[5]], [c[4], c[5], c[2]]])
        out.append(dict(j=e.j, o=tuple(e.o), u=np.array(e.u[:]), cov=cov, w=e.w,
                        log_scale=np.array(e.log_scale[:]), quat=np.array(e.quat[:])))
    return out


def tf_apply(volume, tf, out):
    _check(load().vbm_tf_apply(_ptr(volume), volume.numel(), ctypes.byref(tf), _ptr(out), _stream()))


def dwt3d(data, n_channels, dims, levels, wavelet, tmp):
    _check(load().vbm_dwt3d(_ptr(data), n_channels, _dims(dims), levels, wavelet, _ptr(tmp), _stream()))


def build(volume, dims, tf, bank, sel, capacity, coef=None, keep=None):
    """Volume -> Gaussians.  Returns (params[14][capacity] tensor, n)."""
    import torch
    lib = load()
    size = ctypes.c_size_t()
    _check(lib.vbm_build_workspace_size(_dims(dims), bank.levels, ctypes.byref(size)))
    ws = torch.empty(size.value, dtype=torch.uint8, device=volume.device)
    params = torch.zeros((14, max(int(capacity), 1)), dtype=torch.float32, device=volume.device)
    n = ctypes.c_int64()
    st = lib.vbm_build(_ptr(volume), _dims(dims), ctypes.byref(tf), ctypes.byref(bank), ctypes.byref(sel),
                       _ptr(params), int(capacity), ctypes.byref(n), _ptr(coef), _ptr(keep), _ptr(ws),
                       size.value, _stream())
    if st == VBM_ERR_CAPACITY:
        raise VbmError(st, "capacity %d < %d" % (capacity, n.value))
    _check(st)
    return params, n.value


def render_dvr(volume, dims, tf, cams_dev, n_views, width, height, step, out):
    _check(load().vbm_render_dvr(_ptr(volume), _dims(dims), ctypes.byref(tf), _ptr(cams_dev), n_views, width,
                                 height, float(step), _ptr(out), _stream()))


MAX_PAIR_CAPACITY = (1 << 31) - 1


def default_pair_capacity(n_items):
    """Pair capacity for a batch of n_items (view, Gaussian) items: 24 pairs per item
    (about 1.3 are used on the benchmark workloads), at least 2^20, at most the ABI's
    limit.  A call that needs more renders background and vbm_plan_check reports it."""
    return int(min(MAX_PAIR_CAPACITY, max(1 << 20, 24 * int(n_items))))


def batch_items(scene_offset, n_views, view_scene=None):
    """(view, Gaussian) items of a batch: the sizes of the scenes its views render."""
    so = np.asarray(scene_offset, dtype=np.int64)
    if view_scene is None:
        return int(n_views * (so[-1] - so[0]))
    vs = np.asarray(view_scene, dtype=np.int64)
    return int((so[vs + 1] - so[vs]).sum())


class Plan:
    """Owner of a vbm_plan (device buffers of the splatting forward/backward)."""

    def __init__(self, scene_offset, n_views, width, height, view_scene=None, tile_w=16, tile_h=16,
                 pair_capacity=1 << 20, flags=0, pixels_per_thread=0, group_lanes=0, segment_len=0,
                 bwd_pixels_per_thread=0, bwd_group_lanes=0):
        lib = load()
        self._lib = lib
        so = np.ascontiguousarray(scene_offset, dtype=np.int64)
        self.scene_offset = so
        self.n_views = int(n_views)
        self.width, self.height = int(width), int(height)
        self.tile_w, self.tile_h = int(tile_w), int(tile_h)
        self.pair_capacity = int(pair_capacity)
        vs = None if view_scene is None else np.ascontiguousarray(view_scene, dtype=np.int32)
        self.view_scene = vs
        d = PlanDesc()
        d.n_scenes = so.size - 1
        d.n_views = self.n_views
        d.scene_offset = so.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.view_scene = None if vs is None else vs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.width, d.height, d.tile_w, d.tile_h = self.width, self.height, self.tile_w, self.tile_h
        d.pair_capacity = self.pair_capacity
        d.flags = int(flags)
        d.pixels_per_thread = int(pixels_per_thread)
        self.pixels_per_thread = int(pixels_per_thread)
        d.group_lanes = int(group_lanes)
        self.group_lanes = int(group_lanes)
        d.segment_len = int(segment_len)
        self.segment_len = int(segment_len)
        d.bwd_pixels_per_thread = int(bwd_pixels_per_thread)
        d.bwd_group_lanes = int(bwd_group_lanes)
        h = ctypes.c_void_p()
        _check(lib.vbm_plan_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.vbm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        """(ok, pairs_needed): synchronises the current stream."""
        need = ctypes.c_int64()
        st = self._lib.vbm_plan_check(self.handle, _stream(), ctypes.byref(need))
        if st == VBM_ERR_CAPACITY:
            return False, need.value
        _check(st)
        return True, need.value

    def forward(self, params, cams_dev, img, alpha=None, view_begin=0, view_count=None, bg=(0.0, 0.0, 0.0)):
        vc = self.n_views - view_begin if view_count is None else view_count
        bgc = (ctypes.c_float * 3)(*bg)
        _check(self._lib.vbm_raster_fwd(self.handle, _ptr(params), params.shape[1], _ptr(cams_dev), view_begin,
                                        vc, ctypes.byref(bgc), _ptr(img), _ptr(alpha), _stream()))

    def backward(self, params, cams_dev, dimg, grad, dalpha=None, view_begin=0, view_count=None,
                 bg=(0.0, 0.0, 0.0), accumulate=False):
        vc = self.n_views - view_begin if view_count is None else view_count
        bgc = (ctypes.c_float * 3)(*bg)
        _check(self._lib.vbm_raster_bwd(self.handle, _ptr(params), params.shape[1], _ptr(cams_dev), view_begin,
                                        vc, ctypes.byref(bgc), _ptr(dimg), _ptr(dalpha), _ptr(grad),
                                        int(bool(accumulate)), _stream()))

    def backward_adam(self, params, cams_dev, dimg, m, v, n, step, lrs, dalpha=None, view_begin=0, view_count=None,
                      bg=(0.0, 0.0, 0.0), beta1=0.9, beta2=0.999, eps=1e-15, nonfinite=None):
        """The backward of the last forward fused with the Adam step (vbm_raster_bwd_adam):
        params, m and v are updated in place; no gradient array is written."""
        vc = self.n_views - view_begin if view_count is None else view_count
        bgc = (ctypes.c_float * 3)(*bg)
        lr = (ctypes.c_float * 5)(*[float(x) for x in lrs])
        _check(self._lib.vbm_raster_bwd_adam(self.handle, _ptr(params), params.shape[1], _ptr(cams_dev), view_begin,
                                             vc, ctypes.byref(bgc), _ptr(dimg), _ptr(dalpha), _ptr(m), _ptr(v),
                                             int(n), _ptr(step), ctypes.byref(lr), float(beta1), float(beta2),
                                             float(eps), _ptr(nonfinite), _stream()))

    def set_profile(self, events=None, n_eval=None, n_contrib=None):
        """Record cudaEvents (4 or 7 torch.cuda.Event, see vbm_plan_set_profile) around the
        compositing kernels and the projection, and/or per-pixel evaluated counts (and, for
        recompute-mode plans, per-pixel contributor counts)."""
        n_ev = 0 if events is None else len(events)
        arr = (ctypes.c_void_p * max(1, n_ev))(*[ctypes.c_void_p(e.cuda_event) for e in (events or [])])
        _check(self._lib.vbm_plan_set_profile(self.handle, n_ev, ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)),
                                              _ptr(n_eval), _ptr(n_contrib)))
        self._profile_keepalive = (events, n_eval, n_contrib)

    def buffers(self):
        b = PlanBuffers()
        _check(self._lib.vbm_plan_get_buffers(self.handle, ctypes.byref(b)))
        return b


def loss_workspace(n_images, height, width, device="cuda"):
    import torch
    size = ctypes.c_size_t()
    _check(load().vbm_loss_workspace_size(n_images, height, width, ctypes.byref(size)))
    return torch.empty(size.value, dtype=torch.uint8, device=device)


def loss(img, target, n_images, height, width, lam, scale, loss_out, dimg, ws, accumulate=False):
    _check(load().vbm_loss(_ptr(img), _ptr(target), n_images, height, width, float(lam), float(scale),
                           _ptr(loss_out), int(bool(accumulate)), _ptr(dimg), _ptr(ws), ws.numel(), _stream()))


def loss_static(img, target, n_images, height, width, lam, scale, loss_out, dimg, accumulate=False):
    """vbm_loss without a workspace: scratch lives in the library's static device array."""
    _check(load().vbm_loss_static(_ptr(img), _ptr(target), n_images, height, width, float(lam), float(scale),
                                  _ptr(loss_out), int(bool(accumulate)), _ptr(dimg), _stream()))


def peak_probe(kind, blocks, iters, out):
    """Launch one throughput probe (0 FP32 FMA, 1 FP32x2 FMA, 2 ex2) on the current stream;
    returns its work (FLOP, or ex2 evaluations) for the caller's timing."""
    ops = ctypes.c_double()
    _check(load().vbm_peak_probe(int(kind), int(blocks), int(iters), _ptr(out), ctypes.byref(ops), _stream()))
    return ops.value


def adam(params, grad, m, v, n, step, lrs, beta1=0.9, beta2=0.999, eps=1e-15, nonfinite=None):
    lr = (ctypes.c_float * 5)(*[float(x) for x in lrs])
    _check(load().vbm_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(n), params.shape[1], _ptr(step),
                           ctypes.byref(lr), float(beta1), float(beta2), float(eps), _ptr(nonfinite), _stream()))
