"""Python binding of libtgs, the GB300 tensor-core 3D Gaussian Splatting rasterizer.

Argument marshalling only: every step of the rendering path runs in the library's CUDA kernels.
PyTorch provides device memory and streams. The names mirror include/tgs.h:

    preprocess(scene, camera)                  -> Projected         (tgs_preprocess)
    bin_sort(proj, width, height, tiling)      -> Bins              (tgs_bin_sort)
    rasterize(proj, bins, width, height, ...)  -> (rgb, T, n_contrib) (tgs_rasterize)
    rasterize_backward(...)                    -> gradients         (tgs_rasterize_backward)
    render(scene, camera, ...)                 -> the three forward calls in sequence
    RasterizeFn                                -> torch.autograd.Function over rasterize

There is no CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

TILE = 16
PRECISION = {"fp32": 0, "fp16_tc": 1, "bf16_tc": 2}

TGS_OK = 0
TGS_ERR_INVALID_ARGUMENT = 1
TGS_ERR_CUDA = 2
TGS_ERR_CAPACITY = 3
TGS_ERR_UNSUPPORTED_DEVICE = 4
TGS_ERR_TIMEOUT = 5
TGS_ERR_BUSY = 6
TGS_ERR_NOT_FOUND = 7


class TgsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


# ------------------------------------------------------------------------------------------------
# ctypes mirrors of include/tgs.h

class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacities", C.c_void_p), ("sh", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("cam_pos", C.c_float * 3), ("near_z", C.c_float)]


class _Tiling(C.Structure):
    _fields_ = [("group_w", C.c_int32), ("group_h", C.c_int32), ("flags", C.c_int32)]


BIN_RANGE_ONLY = 1  # tgs_tiling.flags: no tile-membership test


class _Projected(C.Structure):
    _fields_ = [("mean2d", C.c_void_p), ("conic_opacity", C.c_void_p), ("rgb", C.c_void_p),
                ("depth", C.c_void_p), ("radius", C.c_void_p), ("rect", C.c_void_p)]


class _Bins(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("keys", C.c_void_p), ("vals", C.c_void_p), ("masks", C.c_void_p),
                ("ranges", C.c_void_p), ("num_entries", C.c_void_p)]


class _RasterOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("flags", C.c_int32), ("bg", C.c_float * 3),
                ("counters", C.c_void_p)]


RASTER_NO_CULL = 1


class _Frame(C.Structure):
    _fields_ = [("proj", C.POINTER(_Projected)), ("n", C.c_int64), ("bins", C.POINTER(_Bins)),
                ("width", C.c_int32), ("height", C.c_int32), ("out_rgb", C.c_void_p), ("out_T", C.c_void_p),
                ("ready", C.c_void_p), ("ready_value", C.c_int32), ("status", C.c_void_p),
                ("done", C.c_void_p), ("done_value", C.c_int32)]


BATCH_MAX_FRAMES = 32
BATCH_WORKSPACE_BYTES = 256


_P = C.c_void_p
_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes) of every exported function
class _ServeConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_inflight", C.c_int32), ("slots", C.c_int32),
                ("device", C.c_int32), ("precision", C.c_int32), ("tiling", _Tiling),
                ("bg", C.c_float * 3), ("request_timeout_ms", C.c_int32), ("max_gaussians", C.c_int64),
                ("max_width", C.c_int32), ("max_height", C.c_int32), ("max_entries", C.c_int64)]


SERVE_MAX_RESOLUTIONS = 16


class _FramesConfig(C.Structure):
    _fields_ = [("max_gaussians", C.c_int64), ("max_sh_degree", C.c_int32), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("max_entries", C.c_int64), ("tiling", _Tiling),
                ("precision", C.c_int32), ("bg", C.c_float * 3), ("sets", C.c_int32),
                ("device", C.c_int32)]


class _ServeResolutionStats(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("completed", C.c_int64),
                ("mean_ms", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


class _ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("rejected", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("regrown", C.c_int64), ("inflight", C.c_int64),
                ("hbm_bytes", C.c_int64), ("seconds", C.c_double), ("frames_per_second", C.c_double),
                ("num_resolutions", C.c_int32),
                ("res", _ServeResolutionStats * SERVE_MAX_RESOLUTIONS)]


SIGNATURES = {
    "tgs_status_string": (C.c_char_p, [C.c_int32]),
    "tgs_last_error_message": (C.c_char_p, []),
    "tgs_abi_version": (C.c_int32, []),
    "tgs_check_device": (C.c_int32, [C.c_int32]),
    "tgs_preprocess": (C.c_int32, [C.POINTER(_Scene), C.POINTER(_Camera), C.POINTER(_Projected), _P]),
    "tgs_bin_sort_workspace_size": (C.c_int32, [C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                                C.POINTER(_Tiling), C.POINTER(C.c_size_t)]),
    "tgs_bin_sort": (C.c_int32, [C.POINTER(_Projected), C.c_int64, C.c_int32, C.c_int32, C.POINTER(_Tiling),
                                 _P, C.c_size_t, C.POINTER(_Bins), C.POINTER(C.c_int64), _P]),
    "tgs_bin_sort_static": (C.c_int32, [C.POINTER(_Projected), C.c_int64, C.c_int32, C.c_int32,
                                        C.POINTER(_Tiling), C.POINTER(_Bins), C.POINTER(C.c_int64), _P]),
    "tgs_rasterize": (C.c_int32, [C.POINTER(_Projected), C.c_int64, C.POINTER(_Bins), C.c_int32, C.c_int32,
                                  C.POINTER(_Tiling), C.POINTER(_RasterOpts), _P, _P, _P, _P]),
    "tgs_rasterize_batch": (C.c_int32, [C.POINTER(_Frame), C.c_int32, C.POINTER(_Tiling), C.POINTER(_RasterOpts),
                                        C.c_int64, _P, _P]),
    "tgs_rasterize_backward": (C.c_int32, [C.POINTER(_Projected), C.c_int64, C.POINTER(_Bins), C.c_int32,
                                           C.c_int32, C.POINTER(_Tiling), C.POINTER(_RasterOpts), _P, _P,
                                           _P, _P, _P, _P, _P]),
    "tgs_last_device_error": (C.c_int32, [C.c_int32]),
    "tgs_set_lookback_limit": (C.c_int64, [C.c_int64]),
    "tgs_kernel_launch_count": (C.c_int64, []),
    "tgs_allocation_count": (C.c_int64, []),
    "tgs_serve_create": (C.c_int32, [C.POINTER(_ServeConfig), C.POINTER(_P)]),
    "tgs_serve_add_scene": (C.c_int32, [_P, C.POINTER(_Scene), C.POINTER(C.c_int32)]),
    "tgs_serve_remove_scene": (C.c_int32, [_P, C.c_int32]),
    "tgs_serve_submit": (C.c_int32, [_P, C.c_int32, C.POINTER(_Camera), _P, _P, C.POINTER(C.c_uint64)]),
    "tgs_serve_poll": (C.c_int32, [_P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "tgs_serve_wait": (C.c_int32, [_P, C.c_uint64, C.c_int32, C.POINTER(C.c_int32)]),
    "tgs_serve_pause": (C.c_int32, [_P, C.c_int32]),
    "tgs_serve_get_stats": (C.c_int32, [_P, C.POINTER(_ServeStats)]),
    "tgs_serve_destroy": (C.c_int32, [_P]),
    "tgs_frames_create": (C.c_int32, [C.POINTER(_FramesConfig), C.POINTER(_P)]),
    "tgs_frames_device_bytes": (C.c_int64, [_P]),
    "tgs_frames_render": (C.c_int32, [_P, C.POINTER(_Scene), C.POINTER(_Camera), C.c_int32, _P, _P, _P]),
    "tgs_frames_wait": (C.c_int32, [_P]),
    "tgs_frames_destroy": (C.c_int32, [_P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libtgs.so (building it first if its sources are newer). Raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != TGS_OK:
        lib = load()
        raise TgsError(status, f"{lib.tgs_status_string(status).decode()}: "
                               f"{lib.tgs_last_error_message().decode()}")


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------------------------------------
# Inputs

@dataclass
class DeviceScene:
    means: "object"      # torch [n,3] float32
    scales: "object"
    quats: "object"
    opacities: "object"
    sh: "object"
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @classmethod
    def from_host(cls, scene, device="cuda", pin: bool = False, non_blocking: bool = False):
        def t(a):
            x = torch.from_numpy(np.ascontiguousarray(a, np.float32))
            if pin:
                x = x.pin_memory()
            return x.to(device, non_blocking=non_blocking)
        return cls(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacities), t(scene.sh),
                   int(scene.sh_degree))

    def struct(self) -> _Scene:
        return _Scene(self.n, self.sh_degree, _ptr(self.means), _ptr(self.scales), _ptr(self.quats),
                      _ptr(self.opacities), _ptr(self.sh))


def camera_struct(cam) -> _Camera:
    c = _Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(9)
    for k in range(9):
        c.R[k] = float(R[k])
    t = np.asarray(cam.t, np.float32).reshape(3)
    p = np.asarray(cam.cam_pos, np.float32).reshape(3)
    for k in range(3):
        c.t[k] = float(t[k])
        c.cam_pos[k] = float(p[k])
    c.near_z = float(cam.near)
    return c


def _tiling(tiling, membership: bool = True) -> _Tiling:
    gw, gh = tiling[:2]
    return _Tiling(int(gw), int(gh), 0 if membership else BIN_RANGE_ONLY)


def group_grid(width, height, tiling):
    gw, gh = tiling
    tx, ty = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE
    return (tx + gw - 1) // gw, (ty + gh - 1) // gh


# ------------------------------------------------------------------------------------------------
# tgs_preprocess

@dataclass
class Projected:
    n: int
    mean2d: "object"         # [n,2] float32
    conic_opacity: "object"  # [n,4] float32
    rgb: "object"            # [n,3] float32
    depth: "object"          # [n] float32
    radius: "object"         # [n] int32
    rect: "object"           # [n,4] int32

    @classmethod
    def empty(cls, n, device="cuda"):
        f = dict(dtype=torch.float32, device=device)
        i = dict(dtype=torch.int32, device=device)
        return cls(n, torch.empty((n, 2), **f), torch.empty((n, 4), **f), torch.empty((n, 3), **f),
                   torch.empty((n,), **f), torch.empty((n,), **i), torch.empty((n, 4), **i))

    def struct(self) -> _Projected:
        return _Projected(_ptr(self.mean2d), _ptr(self.conic_opacity), _ptr(self.rgb), _ptr(self.depth),
                          _ptr(self.radius), _ptr(self.rect))


def preprocess(scene: DeviceScene, camera, out: Projected | None = None, stream=None) -> Projected:
    lib = load()
    if out is None:
        out = Projected.empty(scene.n, scene.means.device)
    s, c, o = scene.struct(), camera_struct(camera), out.struct()
    _check(lib.tgs_preprocess(C.byref(s), C.byref(c), C.byref(o), _stream(stream)))
    return out


# ------------------------------------------------------------------------------------------------
# tgs_bin_sort

@dataclass
class Bins:
    capacity: int
    tiling: tuple
    keys: "object"         # [capacity] int64 storage of uint64 keys
    vals: "object"         # [capacity] int32 storage of uint32 indices
    masks: "object"        # [capacity] int16 storage of uint16 masks
    ranges: "object"       # [G,2] int32 storage of uint32
    num_entries: "object"  # [1] int64 (device)
    workspace: "object"    # uint8 workspace
    entries: int = -1      # host copy of the count when known
    membership: bool = True  # the tile-membership test was on (tgs_tiling.flags)

    def struct(self) -> _Bins:
        return _Bins(self.capacity, _ptr(self.keys), _ptr(self.vals), _ptr(self.masks), _ptr(self.ranges),
                     _ptr(self.num_entries))


def workspace_size(n, capacity, width, height, tiling) -> int:
    lib = load()
    out = C.c_size_t(0)
    t = _tiling(tiling)
    _check(lib.tgs_bin_sort_workspace_size(int(n), int(capacity), int(width), int(height), C.byref(t),
                                           C.byref(out)))
    return int(out.value)


def allocate_bins(n, capacity, width, height, tiling, device="cuda", keys=True) -> Bins:
    GX, GY = group_grid(width, height, tiling)
    ws = workspace_size(n, capacity, width, height, tiling)
    cap = max(int(capacity), 1)
    return Bins(int(capacity), tuple(tiling),
                torch.empty(cap, dtype=torch.int64, device=device) if keys else None,
                torch.empty(cap, dtype=torch.int32, device=device),
                torch.empty(cap, dtype=torch.int16, device=device),
                torch.empty((GX * GY, 2), dtype=torch.int32, device=device),
                torch.zeros(1, dtype=torch.int64, device=device),
                torch.empty(max(ws, 256), dtype=torch.uint8, device=device))


def bin_sort(proj: Projected, width, height, tiling=(2, 2), bins: Bins | None = None, capacity=None,
             sync=True, stream=None, membership=True) -> Bins:
    """Bins and sorts. With sync=True the entry count is read back (one stream sync) and the
    capacity grows as needed; with sync=False the call is fully asynchronous and overflow leaves
    every range empty (check bins.num_entries). membership=False keeps every tile of each
    Gaussian's AABB range (TGS_BIN_RANGE_ONLY)."""
    lib = load()
    n = proj.n
    if bins is None:
        bins = allocate_bins(n, capacity if capacity is not None else max(1024, 8 * n), width, height,
                             tiling, proj.mean2d.device)
    t = _tiling(tiling, membership)
    bins.membership = bool(membership)
    while True:
        b = bins.struct()
        host = C.c_int64(0)
        st = lib.tgs_bin_sort(C.byref(proj.struct()), n, int(width), int(height), C.byref(t),
                              _ptr(bins.workspace), bins.workspace.numel(), C.byref(b),
                              C.byref(host) if sync else None, _stream(stream))
        if sync and st == TGS_ERR_CAPACITY:
            bins = allocate_bins(n, int(host.value * 1.25) + 1024, width, height, tiling,
                                 proj.mean2d.device, keys=bins.keys is not None)
            bins.membership = bool(membership)
            continue
        _check(st)
        if sync:
            bins.entries = int(host.value)
        return bins


def bin_sort_static(proj: Projected, width, height, bins: Bins, sync=True, stream=None) -> Bins:
    """tgs_bin_sort_static: the bin sort using the library's fixed scratch area instead of
    bins.workspace (for callers that must not allocate device memory). `bins` must already be
    allocated with enough capacity."""
    lib = load()
    t = _tiling(bins.tiling, bins.membership)
    host = C.c_int64(0)
    _check(lib.tgs_bin_sort_static(C.byref(proj.struct()), proj.n, int(width), int(height), C.byref(t),
                                   C.byref(bins.struct()), C.byref(host) if sync else None, _stream(stream)))
    if sync:
        bins.entries = int(host.value)
    return bins


# ------------------------------------------------------------------------------------------------
# tgs_rasterize / tgs_rasterize_backward

def rasterize(proj: Projected, bins: Bins, width, height, precision="fp16_tc", bg=(0.0, 0.0, 0.0),
              out=None, want_n_contrib=True, counters=None, stream=None, cull=True):
    """Returns (rgb [3,H,W], T [H,W], n_contrib [H,W] or None). cull=False sets
    TGS_RASTER_NO_CULL (FP16_TC keeps provably-pruned (Gaussian, tile) pairs)."""
    lib = load()
    dev = proj.mean2d.device
    if out is None:
        rgb = torch.empty((3, height, width), dtype=torch.float32, device=dev)
        T = torch.empty((height, width), dtype=torch.float32, device=dev)
        nc = torch.empty((height, width), dtype=torch.int32, device=dev) if want_n_contrib else None
    else:
        rgb, T, nc = out
    if counters is not None and (counters.dtype != torch.int64 or counters.numel() < 3
                                 or not counters.is_contiguous() or counters.device != dev):
        raise ValueError("counters must be a contiguous int64 tensor of 3 elements on the scene's device")
    o = _RasterOpts(PRECISION[precision], 0 if cull else RASTER_NO_CULL,
                    (C.c_float * 3)(*[float(v) for v in bg]), _ptr(counters))
    t = _tiling(bins.tiling)
    _check(lib.tgs_rasterize(C.byref(proj.struct()), proj.n, C.byref(bins.struct()), int(width), int(height),
                             C.byref(t), C.byref(o), _ptr(rgb), _ptr(T), _ptr(nc), _stream(stream)))
    return rgb, T, nc


@dataclass
class BatchFrame:
    """One frame of rasterize_batch: its projected Gaussians and bins, and where its image goes.
    ready / status are optional device int32 tensors of one element (readiness flag, status word)."""
    proj: Projected
    bins: Bins
    width: int
    height: int
    out_rgb: "object"        # [3,H,W] float32 (device)
    out_T: "object"          # [H,W] float32 (device)
    ready: "object" = None
    ready_value: int = 1
    status: "object" = None
    done: "object" = None
    done_value: int = 1


def rasterize_batch(frames, tiling=(2, 2), precision="fp16_tc", bg=(0.0, 0.0, 0.0), wait_limit_ns=0,
                    workspace=None, stream=None, cull=True):
    """tgs_rasterize_batch: every frame (of any scene and resolution) in one persistent tensor-core
    launch. Returns the workspace tensor (reusable by later calls on the same stream)."""
    lib = load()
    if not frames:
        raise ValueError("no frames")
    dev = frames[0].proj.mean2d.device
    if workspace is None:
        workspace = torch.empty(BATCH_WORKSPACE_BYTES, dtype=torch.uint8, device=dev)
    keep = []
    arr = (_Frame * len(frames))()
    for k, f in enumerate(frames):
        ps, bs = f.proj.struct(), f.bins.struct()
        keep += [ps, bs]
        arr[k] = _Frame(C.pointer(ps), f.proj.n, C.pointer(bs), int(f.width), int(f.height), _ptr(f.out_rgb),
                        _ptr(f.out_T), _ptr(f.ready), int(f.ready_value), _ptr(f.status), _ptr(f.done),
                        int(f.done_value))
    o = _RasterOpts(PRECISION[precision], 0 if cull else RASTER_NO_CULL,
                    (C.c_float * 3)(*[float(v) for v in bg]), None)
    t = _tiling(tiling)
    _check(lib.tgs_rasterize_batch(arr, len(frames), C.byref(t), C.byref(o), int(wait_limit_ns),
                                   _ptr(workspace), _stream(stream)))
    return workspace


def rasterize_backward(proj: Projected, bins: Bins, width, height, T, n_contrib, grad_rgb,
                       bg=(0.0, 0.0, 0.0), stream=None):
    """Returns (g_mean2d [n,2], g_conic_opacity [n,4], g_rgb [n,3])."""
    lib = load()
    n, dev = proj.n, proj.mean2d.device
    gm = torch.empty((n, 2), dtype=torch.float32, device=dev)
    gco = torch.empty((n, 4), dtype=torch.float32, device=dev)
    gc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    o = _RasterOpts(PRECISION["fp32"], 0, (C.c_float * 3)(*[float(v) for v in bg]), None)
    t = _tiling(bins.tiling)
    g = grad_rgb.contiguous()
    _check(lib.tgs_rasterize_backward(C.byref(proj.struct()), n, C.byref(bins.struct()), int(width),
                                      int(height), C.byref(t), C.byref(o), _ptr(T), _ptr(n_contrib), _ptr(g),
                                      _ptr(gm), _ptr(gco), _ptr(gc), _stream(stream)))
    return gm, gco, gc


def kernel_launch_count() -> int:
    return int(load().tgs_kernel_launch_count())


def last_device_error(reset=False) -> int:
    return int(load().tgs_last_device_error(1 if reset else 0))


def set_lookback_limit(ns: int) -> int:
    """Limit of one look-back wait of the bin sort for later calls (ns <= 0: the default, 1 s);
    returns the previous limit (tgs_set_lookback_limit)."""
    return int(load().tgs_set_lookback_limit(int(ns)))


def render(scene: DeviceScene, camera, tiling=(2, 2), precision="fp16_tc", bg=(0.0, 0.0, 0.0),
           bins: Bins | None = None, sync=True, stream=None):
    """preprocess -> bin_sort -> rasterize. Returns (rgb, T, n_contrib, proj, bins)."""
    proj = preprocess(scene, camera, stream=stream)
    bins = bin_sort(proj, camera.width, camera.height, tiling, bins=bins, sync=sync, stream=stream)
    rgb, T, nc = rasterize(proj, bins, camera.width, camera.height, precision, bg, stream=stream)
    return rgb, T, nc, proj, bins


class RasterizeFn(torch.autograd.Function):
    """Differentiable FP32 rasterization of projected Gaussians.

    apply(mean2d [n,2], conic_opacity [n,4], rgb [n,3], depth, radius, rect, bins, width, height, bg)
    -> image [3,H,W]. Backward gives gradients for mean2d, conic_opacity (a, b, c, opacity) and rgb.
    The bins must have been built from the same projected Gaussians."""

    @staticmethod
    def forward(ctx, mean2d, conic_opacity, rgb, depth, radius, rect, bins, width, height, bg):
        proj = Projected(mean2d.shape[0], mean2d.contiguous(), conic_opacity.contiguous(),
                         rgb.contiguous(), depth, radius, rect)
        img, T, nc = rasterize(proj, bins, width, height, "fp32", bg)
        ctx.save_for_backward(proj.mean2d, proj.conic_opacity, proj.rgb, T, nc)
        ctx.meta = (bins, width, height, bg, depth, radius, rect)
        return img

    @staticmethod
    def backward(ctx, grad_img):
        mean2d, co, rgb, T, nc = ctx.saved_tensors
        bins, width, height, bg, depth, radius, rect = ctx.meta
        proj = Projected(mean2d.shape[0], mean2d, co, rgb, depth, radius, rect)
        gm, gco, gc = rasterize_backward(proj, bins, width, height, T, nc, grad_img, bg)
        return gm, gco, gc, None, None, None, None, None, None, None


# ------------------------------------------------------------------------------------------------
# Graph-captured rendering

class Renderer:
    """Renders a resident scene from a fixed set of cameras with CUDA graphs.

    Per camera two graphs are captured: one for preprocess + bin sort (asynchronous, no host round
    trip) and one for rasterize, so a frame is two launches and the GPU never waits on the host
    between the frame's kernels. Every replay recomputes the frame from the scene in HBM; nothing is
    cached between frames. Capacities are sized once from a synchronous count per camera
    (x `margin`); a frame that outgrows its capacity renders background only and reports it through
    `overflowed()`.

    With `pipeline` (default) the preprocess + bin sort of a frame runs on a stream of its own buffer
    set (`sets` sets, taken round robin by camera index), so the preprocess + bin sort chains of the
    next `sets - 1` frames run side by side with each other and with the rasterization of the current
    frame; each set is reused only after the rasterization that read it. Rasterizations run in frame
    order on one stream. Frames are enqueued by render(); join() makes the current stream wait for
    every enqueued frame. Images are the same as without the pipeline.
    """

    def __init__(self, scene: DeviceScene, cameras, tiling=(2, 2), precision="fp16_tc",
                 bg=(0.0, 0.0, 0.0), margin=1.1, graphs=True, cull=True, pipeline=True, membership=True,
                 sets=3):
        self.cull = cull
        self.membership = membership
        self.scene, self.cameras = scene, list(cameras)
        self.tiling, self.precision, self.bg = tuple(tiling), precision, tuple(bg)
        self.pipeline = bool(pipeline)
        n = scene.n
        dev = scene.means.device
        nsets = max(2, int(sets)) if self.pipeline else 1
        self.proj_sets = [Projected.empty(n, dev) for _ in range(nsets)]
        self.proj = self.proj_sets[0]
        cap = 0
        for cam in self.cameras:
            preprocess(scene, cam, out=self.proj)
            cap = max(cap, bin_sort(self.proj, cam.width, cam.height, self.tiling,
                                    membership=membership).entries)
        W = max(c.width for c in self.cameras)
        H = max(c.height for c in self.cameras)
        # bin buffers are shared by the cameras of a set (ranges sized for the largest image)
        self.bin_sets = [allocate_bins(n, int(cap * margin) + 4096, W, H, self.tiling, keys=False)
                         for _ in range(nsets)]
        self.bins = self.bin_sets[0]
        self.out = [(torch.empty((3, c.height, c.width), device=dev),
                     torch.empty((c.height, c.width), device=dev)) for c in self.cameras]
        self.kernels_per_frame = []
        self.g_prep, self.g_raster = [], []
        # The preprocess + bin sort of the next frame runs at the highest stream priority: its chain of
        # short kernels then takes SM slots as the current frame's raster CTAs retire, instead of
        # queueing behind the whole raster grid.
        top = torch.cuda.Stream.priority_range()[1]
        self.s_prep = ([torch.cuda.Stream(device=dev, priority=top) for _ in range(nsets)]
                       if self.pipeline else None)
        self.s_raster = torch.cuda.Stream(device=dev) if self.pipeline else None
        self._set_free = [None] * nsets  # event after the last rasterization that read each set
        for k in range(len(self.cameras)):  # run every path once outside capture
            self._prep(k)
            self._raster(k)
        torch.cuda.synchronize()
        if graphs:
            side = torch.cuda.Stream()
            for k in range(len(self.cameras)):
                before = kernel_launch_count()
                gp, gr = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
                with torch.cuda.graph(gp, stream=side, capture_error_mode="relaxed"):
                    self._prep(k)
                with torch.cuda.graph(gr, stream=side, capture_error_mode="relaxed"):
                    self._raster(k)
                self.kernels_per_frame.append(kernel_launch_count() - before)
                self.g_prep.append(gp)
                self.g_raster.append(gr)
            torch.cuda.synchronize()

    def _set(self, k):
        return k % len(self.proj_sets)

    def _prep(self, k):
        cam = self.cameras[k]
        proj, bins = self.proj_sets[self._set(k)], self.bin_sets[self._set(k)]
        preprocess(self.scene, cam, out=proj)
        bin_sort(proj, cam.width, cam.height, self.tiling, bins=bins, sync=False,
                 membership=self.membership)

    def _raster(self, k):
        cam = self.cameras[k]
        proj, bins = self.proj_sets[self._set(k)], self.bin_sets[self._set(k)]
        rgb, T = self.out[k]
        rasterize(proj, bins, cam.width, cam.height, self.precision, self.bg, out=(rgb, T, None),
                  want_n_contrib=False, cull=self.cull)

    def render(self, k, events=None):
        """Enqueues the frame of camera k; returns (rgb [3,H,W], T [H,W]) (reused buffers, ready
        after join()). `events`, if given, are three CUDA events recorded before the preprocess,
        after the bin sort and after the rasterization."""
        cur = torch.cuda.current_stream()
        if not self.pipeline:
            if events:
                events[0].record(cur)
            self.g_prep[k].replay() if self.g_prep else self._prep(k)
            if events:
                events[1].record(cur)
            self.g_raster[k].replay() if self.g_raster else self._raster(k)
            if events:
                events[2].record(cur)
            return self.out[k]
        st = self._set(k)
        ready = torch.cuda.Event()
        ready.record(cur)  # the caller's work issued so far (e.g. a scene upload)
        sp = self.s_prep[st]
        with torch.cuda.stream(sp):
            sp.wait_event(ready)
            if self._set_free[st] is not None:
                sp.wait_event(self._set_free[st])
            if events:
                events[0].record(sp)
            self.g_prep[k].replay() if self.g_prep else self._prep(k)
            prepped = torch.cuda.Event()
            prepped.record(sp)
            if events:
                events[1].record(sp)
        with torch.cuda.stream(self.s_raster):
            self.s_raster.wait_event(prepped)
            self.g_raster[k].replay() if self.g_raster else self._raster(k)
            done = torch.cuda.Event()
            done.record(self.s_raster)
            if events:
                events[2].record(self.s_raster)
        self._set_free[st] = done
        return self.out[k]

    def join(self):
        """Makes the current stream wait for every frame enqueued so far."""
        if self.pipeline:
            cur = torch.cuda.current_stream()
            cur.wait_stream(self.s_raster)
            for sp in self.s_prep:
                cur.wait_stream(sp)

    def overflowed(self) -> bool:
        """True if the last frame of a buffer set needed more bin entries than the capacity
        (synchronizes)."""
        torch.cuda.synchronize()
        return any(int(b.num_entries.item()) > b.capacity for b in self.bin_sets)


# ------------------------------------------------------------------------------------------------
# Rendering service

class Server:
    """A tgs_server: resident scenes and asynchronous frame requests rendered by a native worker
    thread with `slots` frames in flight (see include/tgs.h, tgs_serve_*). Use as a context manager
    or call close()."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 64, slots: int = 4, device: int = 0,
                 precision: str = "fp16_tc", tiling=(2, 2), bg=(0.0, 0.0, 0.0), request_timeout_ms: int = 0,
                 max_gaussians: int = 1 << 18, max_size=(1024, 1024), max_entries: int = 1 << 22,
                 membership: bool = True):
        """Slot capacities (max_gaussians, max_size = (width, height), max_entries) are fixed here:
        the server allocates every slot buffer now, charged to the budget."""
        lib = load()
        cfg = _ServeConfig(int(hbm_budget_bytes), int(max_inflight), int(slots), int(device),
                           PRECISION[precision], _tiling(tiling, membership),
                           (C.c_float * 3)(*[float(v) for v in bg]), int(request_timeout_ms),
                           int(max_gaussians), int(max_size[0]), int(max_size[1]), int(max_entries))
        h = _P()
        _check(lib.tgs_serve_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self.device = device

    def _handle(self):
        if self._h is None:
            raise ValueError("server is closed")
        return self._h

    def add_scene(self, scene) -> int:
        """Copies a DeviceScene (or any object with the same array fields on the host as numpy)
        into the server; returns its id."""
        if isinstance(scene, DeviceScene):
            st = scene.struct()
            keep = scene
        else:  # host arrays: the library copies them with cudaMemcpyDefault
            arrs = [np.ascontiguousarray(getattr(scene, k), np.float32)
                    for k in ("means", "scales", "quats", "opacities", "sh")]
            keep = arrs
            st = _Scene(int(arrs[0].shape[0]), int(scene.sh_degree),
                        *[a.ctypes.data if a.size else None for a in arrs])
        sid = C.c_int32()
        _check(load().tgs_serve_add_scene(self._handle(), C.byref(st), C.byref(sid)))
        del keep
        return int(sid.value)

    def remove_scene(self, scene_id: int):
        _check(load().tgs_serve_remove_scene(self._handle(), int(scene_id)))

    def submit(self, scene_id: int, cam, out_rgb, out_T=None) -> int:
        """Admits a request; returns its ticket. out_rgb [3,H,W] (and out_T [H,W]) are device
        tensors that must stay alive until the request is done. Raises TgsError (BUSY when full)."""
        t = C.c_uint64()
        c = camera_struct(cam)
        _check(load().tgs_serve_submit(self._handle(), int(scene_id), C.byref(c), _ptr(out_rgb),
                                       _ptr(out_T), C.byref(t)))
        return int(t.value)

    def try_submit(self, scene_id: int, cam, out_rgb, out_T=None):
        """As submit, but returns None instead of raising when the server is full."""
        t = C.c_uint64()
        c = camera_struct(cam)
        st = load().tgs_serve_submit(self._handle(), int(scene_id), C.byref(c), _ptr(out_rgb),
                                     _ptr(out_T), C.byref(t))
        if st == TGS_ERR_BUSY:
            return None
        _check(st)
        return int(t.value)

    def poll(self, ticket: int):
        """None while running, else the request's status (the ticket is then released)."""
        done, res = C.c_int32(), C.c_int32()
        _check(load().tgs_serve_poll(self._handle(), C.c_uint64(ticket), C.byref(done), C.byref(res)))
        return int(res.value) if done.value else None

    def wait(self, ticket: int, timeout_ms: int = 10000) -> int:
        """The request's status; raises TgsError(TIMEOUT) if it is not done in time."""
        res = C.c_int32()
        _check(load().tgs_serve_wait(self._handle(), C.c_uint64(ticket), int(timeout_ms), C.byref(res)))
        return int(res.value)

    def pause(self, paused: bool = True):
        _check(load().tgs_serve_pause(self._handle(), 1 if paused else 0))

    def stats(self) -> dict:
        st = _ServeStats()
        _check(load().tgs_serve_get_stats(self._handle(), C.byref(st)))
        out = {k: getattr(st, k) for k, _ in _ServeStats._fields_ if k not in ("res", "num_resolutions")}
        out["resolutions"] = [{k: getattr(st.res[i], k) for k, _ in _ServeResolutionStats._fields_}
                              for i in range(st.num_resolutions)]
        return out

    def close(self):
        if self._h is not None:
            h, self._h = self._h, None
            _check(load().tgs_serve_destroy(h))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()



# ------------------------------------------------------------------------------------------------
# Frame sequences from host memory

def _host_f32(a):
    """A contiguous float32 host array (numpy or CPU torch tensor) and its address."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError("host arrays must be contiguous float32 CPU tensors")
        return a, a.data_ptr()
    a = np.ascontiguousarray(a, np.float32)
    return a, a.ctypes.data


class Frames:
    """A tgs_frames object (include/tgs.h, tgs_frames_*): a scene in host memory rendered from a
    list of cameras into host images, the host <-> device copies overlapped with the kernels (two
    device copies of the scene, `sets` buffer sets in flight). Every buffer is allocated here.
    Use as a context manager or call close()."""

    def __init__(self, max_gaussians: int, max_size=(1920, 1080), max_entries: int = 1 << 22,
                 tiling=(2, 2), precision: str = "fp16_tc", bg=(0.0, 0.0, 0.0), sets: int = 3,
                 max_sh_degree: int = 3, device: int = 0, membership: bool = True):
        lib = load()
        cfg = _FramesConfig(int(max_gaussians), int(max_sh_degree), int(max_size[0]), int(max_size[1]),
                            int(max_entries), _tiling(tiling, membership), PRECISION[precision],
                            (C.c_float * 3)(*[float(v) for v in bg]), int(sets), int(device))
        h = _P()
        _check(lib.tgs_frames_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._keep = []  # host arrays of calls not yet waited for

    def _handle(self):
        if self._h is None:
            raise TgsError(TGS_ERR_INVALID_ARGUMENT, "frames object closed")
        return self._h

    @property
    def device_bytes(self) -> int:
        return int(load().tgs_frames_device_bytes(self._handle()))

    def render(self, scene, cams, out_rgb, out_T=None, stream=None):
        """Enqueues one call: `scene` has host arrays means, scales, quats, opacities, sh (numpy or
        CPU tensors; page-locked CPU tensors make the copies asynchronous) and sh_degree; out_rgb is
        a host float32 [len(cams), 3, H, W] (out_T [len(cams), H, W] or None). The arrays are kept
        alive until wait(). `stream` (a torch CUDA stream; None = the default stream) is made to wait
        for the call."""
        cams = list(cams)
        arrs = [_host_f32(getattr(scene, k)) for k in ("means", "scales", "quats", "opacities", "sh")]
        n = int(np.prod(arrs[0][0].shape)) // 3
        st = _Scene(n, int(scene.sh_degree), *[p if n else None for _, p in arrs])
        cs = (_Camera * max(1, len(cams)))(*[camera_struct(c) for c in cams])
        rgb, prgb = _host_f32(out_rgb)
        T, pT = _host_f32(out_T) if out_T is not None else (None, None)
        if rgb is not out_rgb or (out_T is not None and T is not out_T):
            raise ValueError("out_rgb / out_T must be contiguous float32 host arrays (written in place)")
        s = C.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(load().tgs_frames_render(self._handle(), C.byref(st), cs, len(cams), prgb, pT, s))
        self._keep.append((arrs, rgb, T))

    def wait(self):
        """Blocks until every enqueued call has completed; raises TgsError (CAPACITY, TIMEOUT) as
        tgs_frames_wait reports."""
        try:
            _check(load().tgs_frames_wait(self._handle()))
        finally:
            self._keep.clear()

    def close(self):
        if self._h is not None:
            _check(load().tgs_frames_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
