"""Python binding of libfhgs.so (include/fhgs.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory, streams and autograd wiring.
If the library is missing the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np
import torch

from . import _build

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_ALIGNMENT, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NUMERIC, \
    ERR_NO_DEVICE = range(9)
PATH_AUTO, PATH_FP32, PATH_TC = 0, 1, 2
GEOM_EWA, GEOM_SURFEL = 0, 1
F32, BF16 = 0, 1
FUSE_ACCUMULATE, FUSE_FINALIZE, FUSE_NORMALIZE = 1, 2, 4
MAX_CAMS = 32
NOALLOC_MAX_ENTRIES = 262144  # FHGS_NOALLOC_MAX_ENTRIES of include/fhgs.h

EXPORTS = ["fhgs_create", "fhgs_destroy", "fhgs_last_error", "fhgs_status_string", "fhgs_abi_version",
           "fhgs_default_params", "fhgs_proj_bytes", "fhgs_total_tiles", "fhgs_reserve", "fhgs_sync_status",
           "fhgs_project", "fhgs_bin_sort", "fhgs_render_fwd", "fhgs_render_bwd", "fhgs_fuse_features",
           "fhgs_profile_enable", "fhgs_profile_read", "fhgs_launch_count", "fhgs_render_bwd_noalloc",
           "fhgs_ndfd_fwd", "fhgs_ndfd_bwd", "fhgs_point_features", "fhgs_l1_loss", "fhgs_adam_state_floats",
           "fhgs_adam_gaussians", "fhgs_noalloc_sync_status", "fhgs_debug_wait_probe", "fhgs_ffma_probe",
           "fhgs_activate_gaussians", "fhgs_sum"]
MAX_POINT_VIEWS = 4096  # FHGS_MAX_POINT_VIEWS of include/fhgs.h
NDFD_K, NDFD_LAMBDA = 20.0, 0.5  # the activation's slope and threshold (Sec. 4)


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12)]


class Params(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("path", ctypes.c_int32), ("batch", ctypes.c_int32), ("d_split", ctypes.c_int32),
                ("znear", ctypes.c_float), ("dilation", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("t_eps", ctypes.c_float), ("cutoff_sq", ctypes.c_float),
                ("fov_clamp", ctypes.c_float), ("bg", ctypes.c_float * 3), ("geometry", ctypes.c_int32),
                ("list_cut", ctypes.c_int32)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 5), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacities", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("n", ctypes.c_int64)]


class Bins(ctypes.Structure):
    _fields_ = [("gids", ctypes.c_void_p), ("keys", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("n_instances", ctypes.c_void_p), ("capacity", ctypes.c_int64)]


class NdfdState(ctypes.Structure):
    """fhgs_ndfd_state: the NDFD forward's end state (F_N, T, last contributor) for its backward."""
    _fields_ = [("F", ctypes.c_void_p), ("T", ctypes.c_void_p), ("last", ctypes.c_void_p)]


class FhgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fhgs status {status}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libfhgs.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libfhgs.so is not built ({_build.LIB}); run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i32, i64, f32p = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        L.fhgs_create.argtypes = [ctypes.POINTER(vp), i32]
        L.fhgs_destroy.argtypes = [vp]
        L.fhgs_destroy.restype = None
        L.fhgs_last_error.argtypes = [vp]
        L.fhgs_last_error.restype = ctypes.c_char_p
        L.fhgs_status_string.argtypes = [i32]
        L.fhgs_status_string.restype = ctypes.c_char_p
        L.fhgs_default_params.argtypes = [ctypes.POINTER(Params)]
        L.fhgs_default_params.restype = None
        L.fhgs_proj_bytes.argtypes = [i64, i32]
        L.fhgs_proj_bytes.restype = i64
        L.fhgs_total_tiles.argtypes = [ctypes.POINTER(Camera), i32]
        L.fhgs_total_tiles.restype = i64
        L.fhgs_reserve.argtypes = [vp, i64, ctypes.POINTER(Camera), i32]
        L.fhgs_sync_status.argtypes = [vp, vp]
        L.fhgs_project.argtypes = [vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), i32,
                                   ctypes.POINTER(Params), vp, vp]
        L.fhgs_bin_sort.argtypes = [vp, i64, vp, ctypes.POINTER(Camera), i32, ctypes.POINTER(Params),
                                    ctypes.POINTER(Bins), vp]
        L.fhgs_render_fwd.argtypes = [vp, i64, vp, ctypes.POINTER(Bins), vp, i32, i32, ctypes.POINTER(Camera), i32,
                                      ctypes.POINTER(Params), f32p, f32p, f32p, vp, vp]
        L.fhgs_render_bwd.argtypes = [vp, ctypes.POINTER(Gaussians), vp, ctypes.POINTER(Bins), vp, i32, i32,
                                      ctypes.POINTER(Camera), i32, ctypes.POINTER(Params), f32p, vp, f32p, f32p,
                                      f32p, f32p, f32p, f32p, f32p, f32p, vp]
        L.fhgs_fuse_features.argtypes = [vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), i32,
                                         ctypes.POINTER(ctypes.c_void_p), i32, ctypes.POINTER(Params), f32p, f32p,
                                         f32p, ctypes.c_uint32, vp]
        L.fhgs_render_bwd_noalloc.argtypes = [ctypes.POINTER(Gaussians), vp, ctypes.POINTER(Bins), vp, i32, i32,
                                              ctypes.POINTER(Camera), i32, ctypes.POINTER(Params), f32p, vp, f32p,
                                              f32p, f32p, f32p, f32p, f32p, f32p, f32p, vp]
        L.fhgs_render_bwd_noalloc.restype = i32
        L.fhgs_noalloc_sync_status.argtypes = [vp]
        L.fhgs_noalloc_sync_status.restype = i32
        L.fhgs_debug_wait_probe.argtypes = [ctypes.c_uint64]
        L.fhgs_debug_wait_probe.restype = i32
        f32 = ctypes.c_float
        L.fhgs_ndfd_fwd.argtypes = [vp, i64, vp, ctypes.POINTER(Bins), vp, vp, i32, i32, ctypes.POINTER(Camera), i32,
                                    ctypes.POINTER(Params), f32, f32, f32p, f32p, vp, ctypes.POINTER(NdfdState), vp]
        L.fhgs_ndfd_bwd.argtypes = [vp, ctypes.POINTER(Gaussians), vp, ctypes.POINTER(Bins), vp, vp, i32, i32,
                                    ctypes.POINTER(Camera), i32, ctypes.POINTER(Params), f32, f32, f32p, f32p,
                                    f32p, f32p, f32p, f32p, f32p, ctypes.POINTER(NdfdState), vp]
        L.fhgs_point_features.argtypes = [vp, i64, f32p, ctypes.POINTER(Camera), i32, ctypes.POINTER(ctypes.c_void_p),
                                          i32, f32p, ctypes.POINTER(Params), f32p, vp, vp, vp]
        L.fhgs_l1_loss.argtypes = [vp, i64, f32p, f32p, f32, f32p, f32p, vp]
        L.fhgs_adam_state_floats.argtypes = [i64, i32]
        L.fhgs_adam_state_floats.restype = i64
        L.fhgs_adam_gaussians.argtypes = [vp, i64, i32] + [f32p] * 5 + [ctypes.POINTER(Grads), i32, f32p,
                                                                       ctypes.POINTER(Adam), f32p, f32p, vp]
        L.fhgs_activate_gaussians.argtypes = [vp, i64, f32p, f32p, f32p, f32p, vp]
        L.fhgs_sum.argtypes = [vp, i64, f32p, f32p, vp]
        L.fhgs_profile_enable.argtypes = [vp, i32]
        L.fhgs_profile_read.argtypes = [vp, ctypes.c_char_p, i64]
        L.fhgs_ffma_probe.argtypes = [i32, i32, vp]
        L.fhgs_ffma_probe.restype = i64
        L.fhgs_launch_count.argtypes = []
        L.fhgs_launch_count.restype = i64
        for name in ("fhgs_create", "fhgs_reserve", "fhgs_sync_status", "fhgs_project", "fhgs_bin_sort",
                     "fhgs_render_fwd", "fhgs_render_bwd", "fhgs_fuse_features", "fhgs_ndfd_fwd", "fhgs_ndfd_bwd",
                     "fhgs_point_features", "fhgs_l1_loss", "fhgs_adam_gaussians", "fhgs_profile_enable",
                     "fhgs_activate_gaussians", "fhgs_sum",
                     "fhgs_profile_read"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_params(sh_degree: int = 0, path: int = PATH_AUTO, bg=(0.0, 0.0, 0.0), **kw) -> Params:
    p = Params()
    lib().fhgs_default_params(ctypes.byref(p))
    p.sh_degree = int(sh_degree)
    p.path = int(path)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    p.bg[0], p.bg[1], p.bg[2] = (float(b) for b in bg)
    return p


def copy_params(p: Params) -> Params:
    q = Params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(Params))
    return q


def make_cameras(cams: Sequence[dict]):
    """Camera dicts (width, height, fx, fy, cx, cy, w2c 3x4) to a C array.
    Values are rounded to float32 exactly as the oracle's FP32 spec does."""
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].width, arr[i].height = int(c["width"]), int(c["height"])
        arr[i].fx, arr[i].fy = float(np.float32(c["fx"])), float(np.float32(c["fy"]))
        arr[i].cx, arr[i].cy = float(np.float32(c["cx"])), float(np.float32(c["cy"]))
        w = np.asarray(c["w2c"], np.float64).reshape(-1).astype(np.float32)
        for k in range(12):
            arr[i].world_to_cam[k] = float(w[k])
    return arr


class Context:
    """An fhgs_ctx on one CUDA device, with thin wrappers of every ABI call."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = ctypes.c_void_p()
        s = lib().fhgs_create(ctypes.byref(h), self.device)
        if s != OK:
            raise FhgsError(s, lib().fhgs_status_string(s).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().fhgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, s: int):
        if s != OK:
            raise FhgsError(s, lib().fhgs_last_error(self.h).decode())

    @staticmethod
    def stream_ptr(stream=None):
        st = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(st.cuda_stream)

    # --------------------------------------------------------- instrumentation
    def profile(self, enable: bool = True):
        self.check(lib().fhgs_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self.check(lib().fhgs_profile_read(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    @staticmethod
    def launch_count() -> int:
        return int(lib().fhgs_launch_count())

    # --------------------------------------------------------------- calls
    def reserve(self, max_n: int, cams):
        self.check(lib().fhgs_reserve(self.h, int(max_n), cams, len(cams)))

    def sync_status(self, stream=None) -> int:
        return lib().fhgs_sync_status(self.h, self.stream_ptr(stream))

    def project(self, g: Gaussians, cams, params: Params, proj: torch.Tensor, stream=None):
        self.check(lib().fhgs_project(self.h, ctypes.byref(g), cams, len(cams), ctypes.byref(params), _ptr(proj),
                                      self.stream_ptr(stream)))

    def bin_sort(self, n: int, proj, cams, params, bins: Bins, stream=None):
        self.check(lib().fhgs_bin_sort(self.h, int(n), _ptr(proj), cams, len(cams), ctypes.byref(params),
                                       ctypes.byref(bins), self.stream_ptr(stream)))

    def render_fwd(self, n, proj, bins, features, D, cams, params, rgb, feat, T, last, stream=None):
        ft = BF16 if (features is not None and features.dtype == torch.bfloat16) else F32
        self.check(lib().fhgs_render_fwd(self.h, int(n), _ptr(proj), ctypes.byref(bins), _ptr(features), ft, int(D),
                                         cams, len(cams), ctypes.byref(params), _ptr(rgb), _ptr(feat), _ptr(T),
                                         _ptr(last), self.stream_ptr(stream)))

    def render_bwd(self, g, proj, bins, features, D, cams, params, T, last, grgb, gfeat, out: dict, stream=None):
        ft = BF16 if (features is not None and features.dtype == torch.bfloat16) else F32
        self.check(lib().fhgs_render_bwd(self.h, ctypes.byref(g), _ptr(proj), ctypes.byref(bins), _ptr(features),
                                         ft, int(D), cams, len(cams), ctypes.byref(params), _ptr(T), _ptr(last),
                                         _ptr(grgb), _ptr(gfeat), _ptr(out["means"]), _ptr(out["scales"]),
                                         _ptr(out["quats"]), _ptr(out["opacities"]), _ptr(out["sh"]),
                                         _ptr(out.get("features")), self.stream_ptr(stream)))

    def fuse(self, g, views, maps: Sequence[torch.Tensor], D, params, num, den, out, flags, stream=None):
        ptrs = (ctypes.c_void_p * max(1, len(maps)))(*[m.data_ptr() for m in maps])
        self.check(lib().fhgs_fuse_features(self.h, ctypes.byref(g), views, len(views), ptrs, int(D),
                                            ctypes.byref(params), _ptr(num), _ptr(den), _ptr(out), int(flags),
                                            self.stream_ptr(stream)))


    def ndfd_fwd(self, n, proj, bins, features, feat_gt, D, cams, params, k, lam, Lgt, Lcf, ncontrib=None,
                 state=None, stream=None):
        """state: optional dict of F [P, D], T [P], last [P] tensors that
        receive the walk's end state (tensor-core kernels only)."""
        ft = BF16 if features.dtype == torch.bfloat16 else F32
        sv = None if state is None else ctypes.byref(_ndfd_state(state))
        self.check(lib().fhgs_ndfd_fwd(self.h, int(n), _ptr(proj), ctypes.byref(bins), _ptr(features), _ptr(feat_gt),
                                       ft, int(D), cams, len(cams), ctypes.byref(params), float(k), float(lam),
                                       _ptr(Lgt), _ptr(Lcf), _ptr(ncontrib), sv, self.stream_ptr(stream)))

    def ndfd_bwd(self, g, proj, bins, features, feat_gt, D, cams, params, k, lam, dLgt, dLcf, out: dict,
                 state=None, stream=None):
        ft = BF16 if features.dtype == torch.bfloat16 else F32
        sv = None if state is None else ctypes.byref(_ndfd_state(state))
        self.check(lib().fhgs_ndfd_bwd(self.h, ctypes.byref(g), _ptr(proj), ctypes.byref(bins), _ptr(features),
                                       _ptr(feat_gt), ft, int(D), cams, len(cams), ctypes.byref(params), float(k),
                                       float(lam), _ptr(dLgt), _ptr(dLcf), _ptr(out["means"]), _ptr(out["scales"]),
                                       _ptr(out["quats"]), _ptr(out["opacities"]), _ptr(out["sh"]), sv,
                                       self.stream_ptr(stream)))


def _ndfd_state(state: dict) -> NdfdState:
    return NdfdState(state["F"].data_ptr(), state["T"].data_ptr(), state["last"].data_ptr())


def point_features(ctx: "Context", means, views: Sequence[dict], maps: Sequence[torch.Tensor], u, params: Params,
                   stream=None):
    """fhgs_point_features: per point, the feature of its pixel in a view
    drawn (by u in [0, 1)) among the views that see it.  maps[v]: [H*W, D]
    float32 on the device.  Returns (features [n, D], view [n], pixel [n])."""
    n = int(means.shape[0])
    D = int(maps[0].shape[-1])
    dev = means.device
    out = torch.empty((n, D), dtype=torch.float32, device=dev)
    view = torch.empty(n, dtype=torch.int32, device=dev)
    pixel = torch.empty(n, dtype=torch.int32, device=dev)
    cams = make_cameras(views)
    ptrs = (ctypes.c_void_p * len(maps))(*[m.data_ptr() for m in maps])
    ctx.check(lib().fhgs_point_features(ctx.h, n, _ptr(means.contiguous()), cams, len(views), ptrs, D,
                                        _ptr(u.contiguous()), ctypes.byref(params), _ptr(out), _ptr(view),
                                        _ptr(pixel), Context.stream_ptr(stream)))
    return out, view, pixel


def l1_loss(ctx: "Context", a, b, loss=None, want_grad: bool = True, stream=None):
    """fhgs_l1_loss over all elements of a and b: returns (loss [1], grad)
    with loss = mean |a - b| (accumulated into `loss` when given)."""
    m = int(a.numel())
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=a.device)
    grad = torch.empty_like(a) if want_grad else None
    ctx.check(lib().fhgs_l1_loss(ctx.h, m, _ptr(a.contiguous()), _ptr(b.contiguous()), 1.0 / max(m, 1), _ptr(loss),
                                 _ptr(grad), Context.stream_ptr(stream)))
    return loss, grad


def adam_gaussians(ctx: "Context", raw: dict, grads, state, step: int, lr, sh_degree: int,
                   beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15, scales_out=None, opac_out=None,
                   stream=None):
    """fhgs_adam_gaussians: one Adam update of raw = {means, log_scales,
    quats, logit_opacities, sh} (in place) from the activated-parameter
    gradients {means, scales, quats, opacities, sh} -- one dict, or a list of
    up to four whose sum the kernel takes.  lr: five rates."""
    sets = [grads] if isinstance(grads, dict) else list(grads)
    arr = (Grads * len(sets))()
    for i, g in enumerate(sets):
        arr[i].means, arr[i].scales, arr[i].quats = _ptr(g["means"]), _ptr(g["scales"]), _ptr(g["quats"])
        arr[i].opacities, arr[i].sh = _ptr(g["opacities"]), _ptr(g["sh"])
    opt = Adam()
    for k in range(5):
        opt.lr[k] = float(lr[k])
    opt.beta1, opt.beta2, opt.eps, opt.step = beta1, beta2, eps, int(step)
    n = int(raw["means"].shape[0])
    ctx.check(lib().fhgs_adam_gaussians(
        ctx.h, n, int(sh_degree), _ptr(raw["means"]), _ptr(raw["log_scales"]), _ptr(raw["quats"]),
        _ptr(raw["logit_opacities"]), _ptr(raw["sh"]), arr, len(sets), _ptr(state), ctypes.byref(opt),
        _ptr(scales_out), _ptr(opac_out), Context.stream_ptr(stream)))


def activate_gaussians(ctx: "Context", log_scales, logit_opacities, stream=None):
    """fhgs_activate_gaussians: (exp(log_scales), sigmoid(logits)) on the device."""
    n = int(log_scales.shape[0])
    scales = torch.empty((n, 3), dtype=torch.float32, device=log_scales.device)
    opac = torch.empty(n, dtype=torch.float32, device=log_scales.device)
    ctx.check(lib().fhgs_activate_gaussians(ctx.h, n, _ptr(log_scales), _ptr(logit_opacities), _ptr(scales),
                                            _ptr(opac), Context.stream_ptr(stream)))
    return scales, opac


def sum_f32(ctx: "Context", x, out=None, stream=None):
    """fhgs_sum: the sum of all elements of x, as a device float[1]
    (accumulated into `out` when given)."""
    if out is None:
        out = torch.zeros(1, dtype=torch.float32, device=x.device)
    ctx.check(lib().fhgs_sum(ctx.h, int(x.numel()), _ptr(x.contiguous()), _ptr(out), Context.stream_ptr(stream)))
    return out


def adam_state(n: int, sh_degree: int, device) -> torch.Tensor:
    """A zeroed Adam state for n Gaussians (fhgs_adam_state_floats floats)."""
    return torch.zeros(int(lib().fhgs_adam_state_floats(int(n), int(sh_degree))), dtype=torch.float32,
                       device=device)


def render_bwd_noalloc(g, proj, bins, features, D, cams, params, T, last, grgb, gfeat, out: dict, stream=None) -> int:
    """fhgs_render_bwd_noalloc: the backward without a context and without
    allocating (scratch in a fixed device array).  Returns the status code."""
    ft = BF16 if (features is not None and features.dtype == torch.bfloat16) else F32
    return int(lib().fhgs_render_bwd_noalloc(ctypes.byref(g), _ptr(proj), ctypes.byref(bins), _ptr(features), ft,
                                             int(D), cams, len(cams), ctypes.byref(params), _ptr(T), _ptr(last),
                                             _ptr(grgb), _ptr(gfeat), _ptr(out["means"]), _ptr(out["scales"]),
                                             _ptr(out["quats"]), _ptr(out["opacities"]), _ptr(out["sh"]),
                                             _ptr(out.get("features")), Context.stream_ptr(stream)))


def noalloc_sync_status(stream=None) -> int:
    """fhgs_noalloc_sync_status: reads and clears the allocation-free
    backward's status word on the current device.  Returns the status code."""
    return int(lib().fhgs_noalloc_sync_status(Context.stream_ptr(stream)))


def debug_wait_probe(ns: int) -> None:
    """fhgs_debug_wait_probe: while ns > 0, every CTA of the tensor-core
    kernels launched afterwards runs out a bounded wait (ns) before doing
    anything, latches FHGS_ERR_TIMEOUT and returns.  0 turns it off."""
    s = int(lib().fhgs_debug_wait_probe(int(ns)))
    if s != OK:
        raise FhgsError(s, "fhgs_debug_wait_probe")


def gaussians_struct(means, scales, quats, opacities, sh) -> Gaussians:
    g = Gaussians()
    g.means, g.scales, g.quats = means.data_ptr(), scales.data_ptr(), quats.data_ptr()
    g.opacities, g.sh, g.n = opacities.data_ptr(), sh.data_ptr(), means.shape[0]
    return g


def _contig(t, dtype=torch.float32):
    return t.detach().to(dtype).contiguous()


class Rasterizer:
    """Forward/backward of the hot path on one device, keeping the buffers
    (projection, tile lists, instance capacity) between calls."""

    def __init__(self, device: int = 0, sh_degree: int = 0, path: int = PATH_AUTO, bg=(0.0, 0.0, 0.0),
                 keep_keys: bool = False, **params):
        self.ctx = Context(device)
        self.dev = torch.device("cuda", device)
        self.params = make_params(sh_degree=sh_degree, path=path, bg=bg, **params)
        self.params_bwd = None  # backward parameters when its D split differs
        self.keep_keys = keep_keys
        self.capacity = 0

    def set_path(self, path: int):
        self.params.path = int(path)
        if self.params_bwd is not None:
            self.params_bwd.path = int(path)

    def set_splits(self, fwd: int, bwd: int):
        """Feature columns per CTA of the tensor-core forward and backward
        (0 = the library's choice)."""
        self.params.d_split = int(fwd)
        self.params_bwd = copy_params(self.params)
        self.params_bwd.d_split = int(bwd)

    # --------------------------------------------------------------- steps
    def prepare(self, means, scales, quats, opacities, sh, cams: Sequence[dict], capacity: int | None = None,
                check: bool = True) -> dict:
        """Projection + binning.  Returns the state the render calls use."""
        ccams = make_cameras(cams)
        n = int(means.shape[0])
        g = gaussians_struct(means, scales, quats, opacities, sh)
        total_tiles = int(lib().fhgs_total_tiles(ccams, len(cams)))
        proj = torch.empty(int(lib().fhgs_proj_bytes(n, len(cams))), dtype=torch.uint8, device=self.dev)
        self.ctx.project(g, ccams, self.params, proj)
        if capacity is not None:
            self.capacity = max(self.capacity, int(capacity))
        if self.capacity == 0:
            self.capacity = max(1024, 16 * n * len(cams))
        while True:
            st = dict(n=n, g=g, cams=ccams, ncam=len(cams), proj=proj, total_tiles=total_tiles,
                      params=(means, scales, quats, opacities, sh),  # g points into these: keep them alive
                      gids=torch.empty(self.capacity, dtype=torch.int32, device=self.dev),
                      keys=torch.empty(self.capacity, dtype=torch.int64, device=self.dev) if self.keep_keys else None,
                      ranges=torch.empty((total_tiles, 2), dtype=torch.int32, device=self.dev),
                      count=torch.zeros(1, dtype=torch.int64, device=self.dev))
            st["bins"] = Bins(st["gids"].data_ptr(), _ptr(st["keys"]).value if st["keys"] is not None else None,
                              st["ranges"].data_ptr(), st["count"].data_ptr(), self.capacity)
            self.ctx.bin_sort(n, proj, ccams, self.params, st["bins"])
            if not check:
                return st
            cnt = int(st["count"].item())
            if cnt <= self.capacity:
                self.ctx.sync_status()  # clears a latched overflow from an earlier try
                st["n_instances"] = cnt
                return st
            self.capacity = int(cnt * 1.25) + 1024

    def forward(self, st: dict, features, cams: Sequence[dict] | None = None, want_feat: bool = True):
        P = sum(int(c.width) * int(c.height) for c in st["cams"])
        D = 0 if features is None else int(features.shape[1])
        rgb = torch.empty((P, 3), dtype=torch.float32, device=self.dev)
        feat = torch.empty((P, D), dtype=torch.float32, device=self.dev) if (D and want_feat) else None
        T = torch.empty(P, dtype=torch.float32, device=self.dev)
        last = torch.empty(P, dtype=torch.int32, device=self.dev)
        self.ctx.render_fwd(st["n"], st["proj"], st["bins"], features, D if feat is not None else 0, st["cams"],
                            self.params, rgb, feat, T, last)
        st.update(T=T, last=last, features=features, D=D)
        return rgb, feat

    def backward(self, st: dict, grad_rgb, grad_feat, want_feat_grad: bool = True) -> dict:
        n, D = st["n"], st["D"]
        K = (self.params.sh_degree + 1) ** 2
        out = dict(means=torch.empty((n, 3), device=self.dev), scales=torch.empty((n, 3), device=self.dev),
                   quats=torch.empty((n, 4), device=self.dev), opacities=torch.empty(n, device=self.dev),
                   sh=torch.empty((n, K, 3), device=self.dev),
                   features=torch.empty((n, D), device=self.dev) if (D and want_feat_grad) else None)
        params = self.params_bwd if self.params_bwd is not None else self.params
        self.ctx.render_bwd(st["g"], st["proj"], st["bins"], st["features"], D, st["cams"], params, st["T"],
                            st["last"], grad_rgb.contiguous(),
                            None if grad_feat is None else grad_feat.contiguous(), out)
        return out

    def ndfd_forward(self, st: dict, features, feat_gt, k: float = NDFD_K, lam: float = NDFD_LAMBDA,
                     ncontrib=None, save_state: bool = False):
        """Per-pixel NDFD losses (L_gt, L_cf), each [P] float32, over the
        prepared views; feat_gt is [P, D] in the features' dtype.  ncontrib,
        an optional [P] int32 tensor, receives each pixel's contributor count.
        save_state keeps the walk's end state (F_N [P, D] FP32, T, last) in
        st, where ndfd_backward reads it instead of rebuilding it; the
        CUDA-core kernels neither write nor read it."""
        P = sum(int(c.width) * int(c.height) for c in st["cams"])
        D = int(features.shape[1])
        Lgt = torch.empty(P, dtype=torch.float32, device=self.dev)
        Lcf = torch.empty(P, dtype=torch.float32, device=self.dev)
        state = None
        st.pop("ndfd_state", None)
        if save_state:
            state = dict(F=torch.empty((P, D), dtype=torch.float32, device=self.dev),
                         T=torch.empty(P, dtype=torch.float32, device=self.dev),
                         last=torch.empty(P, dtype=torch.int32, device=self.dev))
        self.ctx.ndfd_fwd(st["n"], st["proj"], st["bins"], features, feat_gt.contiguous(), D, st["cams"], self.params,
                          k, lam, Lgt, Lcf, ncontrib, state)
        if state is not None:
            st["ndfd_state"] = state
        return Lgt, Lcf

    def ndfd_backward(self, st: dict, features, feat_gt, grad_Lgt, grad_Lcf, k: float = NDFD_K,
                      lam: float = NDFD_LAMBDA) -> dict:
        """Gradients of sum_p grad_Lgt L_gt + grad_Lcf L_cf with respect to
        means, scales, quats, opacities (and sh: zeros)."""
        n, D = st["n"], int(features.shape[1])
        K = (self.params.sh_degree + 1) ** 2
        out = dict(means=torch.empty((n, 3), device=self.dev), scales=torch.empty((n, 3), device=self.dev),
                   quats=torch.empty((n, 4), device=self.dev), opacities=torch.empty(n, device=self.dev),
                   sh=torch.empty((n, K, 3), device=self.dev))
        self.ctx.ndfd_bwd(st["g"], st["proj"], st["bins"], features, feat_gt.contiguous(), D, st["cams"],
                          self.params, k, lam, grad_Lgt.contiguous(), grad_Lcf.contiguous(), out,
                          st.get("ndfd_state"))
        return out

    def fuse(self, means, scales, quats, opacities, sh, views: Sequence[dict], maps: Sequence[torch.Tensor],
             normalize: bool = False, num=None, den=None, accumulate: bool = False):
        n = int(means.shape[0])
        D = int(maps[0].shape[-1])
        g = gaussians_struct(means, scales, quats, opacities, sh)
        num = torch.zeros((n, D), device=self.dev) if num is None else num
        den = torch.zeros(n, device=self.dev) if den is None else den
        out = torch.empty((n, D), device=self.dev)
        flags = FUSE_FINALIZE | (FUSE_NORMALIZE if normalize else 0) | (FUSE_ACCUMULATE if accumulate else 0)
        self.ctx.fuse(g, make_cameras(views), [m.contiguous() for m in maps], D, self.params, num, den, out, flags)
        return out, num, den

    def fuse_accumulate(self, gaussians: tuple, views: Sequence[dict], maps: Sequence[torch.Tensor], num, den):
        """Add the views' fusion numerator and denominator into num/den (no
        division)."""
        g = gaussians_struct(*gaussians)
        D = int(num.shape[1])
        self.ctx.fuse(g, make_cameras(views), [m.contiguous() for m in maps], D, self.params, num, den, None,
                      FUSE_ACCUMULATE)

    def fuse_finalize(self, gaussians: tuple, num, den, normalize: bool = False):
        """f = num / den (0 where den == 0), optionally L2-normalised."""
        g = gaussians_struct(*gaussians)
        out = torch.empty_like(num)
        dummy = make_cameras([dict(width=1, height=1, fx=1.0, fy=1.0, cx=0.5, cy=0.5,
                                   w2c=np.eye(3, 4))])  # n_views = 0: only the division runs
        flags = FUSE_ACCUMULATE | FUSE_FINALIZE | (FUSE_NORMALIZE if normalize else 0)
        self.ctx.check(lib().fhgs_fuse_features(self.ctx.h, ctypes.byref(g), dummy, 0, None, int(num.shape[1]),
                                                ctypes.byref(self.params), _ptr(num), _ptr(den), _ptr(out),
                                                int(flags), self.ctx.stream_ptr(None)))
        return out


class CapturedStep:
    """A whole forward + backward step over fixed cameras, captured once in a
    CUDA graph and then replayed as one launch: projection, binning, both
    renders (all cameras of uneven size in one launch each) and the
    projection backward.  The caller writes new inputs into `inputs` (copy_)
    before replay(); every replay overwrites `outputs`.

    The instance capacity is fixed at capture (the instance count of the
    capture-time scene times `margin`); a replay whose scene needs more
    latches FHGS_ERR_CAPACITY, which rast.ctx.sync_status() reports."""

    def __init__(self, rast: Rasterizer, means, scales, quats, opacities, sh, features, grad_rgb, grad_feat,
                 cams: Sequence[dict], margin: float = 1.25, warmup: int = 2):
        self.rast = rast
        self.cams = list(cams)
        self.inputs = dict(means=_contig(means), scales=_contig(scales), quats=_contig(quats),
                           opacities=_contig(opacities), sh=_contig(sh),
                           features=None if features is None else features.detach().clone().contiguous(),
                           grad_rgb=_contig(grad_rgb),
                           grad_feat=None if grad_feat is None else _contig(grad_feat))
        x = self.inputs
        n = int(x["means"].shape[0])
        st = rast.prepare(x["means"], x["scales"], x["quats"], x["opacities"], x["sh"], self.cams)
        rast.capacity = int(st["n_instances"] * margin) + 1024
        del st
        rast.ctx.reserve(n, make_cameras(self.cams))
        side = torch.cuda.Stream(device=rast.dev)
        side.wait_stream(torch.cuda.current_stream(rast.dev))
        with torch.cuda.stream(side):
            for _ in range(max(1, warmup)):
                self._step()
        torch.cuda.current_stream(rast.dev).wait_stream(side)
        torch.cuda.synchronize(rast.dev)
        s = rast.ctx.sync_status()
        if s != OK:
            raise FhgsError(s, "device status after the warm-up steps")
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.outputs = self._step()

    def _step(self) -> dict:
        x, r = self.inputs, self.rast
        st = r.prepare(x["means"], x["scales"], x["quats"], x["opacities"], x["sh"], self.cams, check=False)
        rgb, feat = r.forward(st, x["features"])
        grads = r.backward(st, x["grad_rgb"], x["grad_feat"])
        return dict(rgb=rgb, feat=feat, T=st["T"], last=st["last"], ranges=st["ranges"], gids=st["gids"],
                    count=st["count"], grads=grads)

    def replay(self) -> dict:
        self.graph.replay()
        return self.outputs


class HostPipeline:
    """Forward + backward over inputs that live in (pinned) host memory, with
    the copies overlapped: step k's inputs go host -> device on a copy stream
    while step k-1 computes, and each step's outputs go device -> host on a
    second copy stream while the next step computes.  Device inputs and host
    outputs are double-buffered; events order every reuse.

    inputs: dict of pinned host tensors named means, scales, quats,
    opacities, sh, features, grad_rgb, grad_feat.  step() queues one step and
    returns the pinned host tensors it will fill (rgb, feat, then the
    gradients); they are valid after finish() or once the step two later has
    been queued and synchronised, and are reused by the step two later."""

    NAMES = ("means", "scales", "quats", "opacities", "sh", "features", "grad_rgb", "grad_feat")

    def __init__(self, rast: Rasterizer, cams: Sequence[dict], inputs: dict):
        self.rast, self.cams = rast, list(cams)
        dev = rast.dev
        self.h_in = {k: inputs[k] for k in self.NAMES}
        self.d_in = [{k: torch.empty_like(v, device=dev) for k, v in self.h_in.items()} for _ in range(2)]
        self.s_h2d = torch.cuda.Stream(device=dev)
        self.s_cmp = torch.cuda.Stream(device=dev)
        self.s_d2h = torch.cuda.Stream(device=dev)
        self.ev_in = [torch.cuda.Event() for _ in range(2)]  # inputs of slot j copied in
        self.ev_used = [None, None]                          # slot j's inputs consumed
        self.ev_out = [None, None]                           # host outputs of slot j copied out
        self.h_out = [None, None]
        self.k = 0

    def start(self):
        """Order the pipeline's streams after the current stream (e.g. after
        a timing event)."""
        cur = torch.cuda.current_stream(self.rast.dev)
        for st in (self.s_h2d, self.s_cmp, self.s_d2h):
            st.wait_stream(cur)

    def step(self):
        j = self.k % 2
        d = self.d_in[j]
        with torch.cuda.stream(self.s_h2d):
            if self.ev_used[j] is not None:
                self.s_h2d.wait_event(self.ev_used[j])
            for name, h in self.h_in.items():
                d[name].copy_(h, non_blocking=True)
            self.ev_in[j].record(self.s_h2d)
        with torch.cuda.stream(self.s_cmp):
            self.s_cmp.wait_event(self.ev_in[j])
            st = self.rast.prepare(d["means"], d["scales"], d["quats"], d["opacities"], d["sh"], self.cams,
                                   check=False)
            rgb, feat = self.rast.forward(st, d["features"])
            grads = self.rast.backward(st, d["grad_rgb"], d["grad_feat"])
            outs = [rgb, feat] + [v for v in grads.values() if v is not None]
            used = torch.cuda.Event()
            used.record(self.s_cmp)
            self.ev_used[j] = used
        if self.h_out[j] is None:
            self.h_out[j] = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
        with torch.cuda.stream(self.s_d2h):
            self.s_d2h.wait_event(used)
            if self.ev_out[j] is not None:
                self.s_d2h.wait_event(self.ev_out[j])
            for o, ho in zip(outs, self.h_out[j]):
                o.record_stream(self.s_d2h)
                ho.copy_(o, non_blocking=True)
            self.ev_out[j] = torch.cuda.Event()
            self.ev_out[j].record(self.s_d2h)
        for t in d.values():
            t.record_stream(self.s_cmp)
        self.k += 1
        return self.h_out[j]

    def finish(self):
        """Order the current stream after everything queued."""
        cur = torch.cuda.current_stream(self.rast.dev)
        for st in (self.s_h2d, self.s_cmp, self.s_d2h):
            cur.wait_stream(st)

    def bytes_per_step(self):
        h2d = sum(v.numel() * v.element_size() for v in self.h_in.values())
        d2h = sum(v.numel() * v.element_size() for v in (self.h_out[0] or []))
        return h2d, d2h


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, features, rast, cams):
        m, s, q, o, h = (_contig(t) for t in (means, scales, quats, opacities, sh))
        f = None if features is None else features.detach().contiguous()
        st = rast.prepare(m, s, q, o, h, cams)
        rgb, feat = rast.forward(st, f)
        ctx.rast, ctx.st = rast, st
        ctx.keep = (m, s, q, o, h, f)
        ctx.has_feat = f is not None
        return rgb, feat if feat is not None else torch.zeros(0, device=rgb.device)

    @staticmethod
    def backward(ctx, grad_rgb, grad_feat):
        rast, st = ctx.rast, ctx.st
        gf = grad_feat if (ctx.has_feat and grad_feat is not None and grad_feat.numel()) else None
        out = rast.backward(st, grad_rgb.float(), None if gf is None else gf.float(),
                            want_feat_grad=ctx.needs_input_grad[5])
        gfeat = out.get("features")
        if gfeat is not None and ctx.keep[5] is not None:
            gfeat = gfeat.to(ctx.keep[5].dtype)
        return out["means"], out["scales"], out["quats"], out["opacities"], out["sh"], gfeat, None, None


def render(means, scales, quats, opacities, sh, features, cams: Sequence[dict], rast: Rasterizer):
    """Differentiable render: returns rgb [P,3] and feat [P,D] (packed over
    cameras).  Gradients flow to every input, features included."""
    return _RenderFn.apply(means, scales, quats, opacities, sh, features, rast, list(cams))
