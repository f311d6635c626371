"""FP64 CPU oracle of the TensorGS rasterizer (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import this package. The rendering library (`paper_2605_17855_gb300`) never imports it and
shares no code with it; the only inputs both sides see come from `paper_2605_17855_gb300.scenes`,
which draws random inputs and holds none of the method's arithmetic.

Pins: every function here is checked against something other than itself in
tests/test_oracle_pins.py (closed forms, invariants, brute force, library routines).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("cam_pos", C.c_double * 3), ("near_z", C.c_double)]


_P = C.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_sh_basis.argtypes = [_P, _P]
            lib.orc_preprocess.argtypes = [C.c_int64, C.c_int32, _P, _P, _P, _P, _P, C.POINTER(OrcCamera),
                                           _P, _P, _P, _P, _P, _P, _P]
            lib.orc_project_cov.argtypes = [_P, _P, _P, C.POINTER(OrcCamera), _P]
            lib.orc_tile_rect.argtypes = [C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_int32, _P]
            lib.orc_tile_rect.restype = C.c_int32
            lib.orc_bin_count.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32,
                                          C.c_int32]
            lib.orc_bin_count.restype = C.c_int64
            lib.orc_bin.argtypes = [C.c_int64, _P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int32, _P, _P, _P, _P]
            lib.orc_blend.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P,
                                      _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P]
            lib.orc_blend_backward.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                               _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int64, _P,
                                               _P, _P, _P, _P]
            lib.orc_num_threads.restype = C.c_int32
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera_struct(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    for k, v in enumerate(np.asarray(cam.R, np.float32).reshape(9)):
        c.R[k] = float(v)
    for k in range(3):
        c.t[k] = float(np.asarray(cam.t, np.float32)[k])
        c.cam_pos[k] = float(np.asarray(cam.cam_pos, np.float32)[k])
    c.near_z = float(np.float32(cam.near))
    return c


def num_threads() -> int:
    return int(_load().orc_num_threads())


def sh_basis(d) -> np.ndarray:
    d = _f64(d).reshape(3)
    out = np.zeros(16)
    _load().orc_sh_basis(_ptr(d), _ptr(out))
    return out


@dataclass
class Projected:
    mean2d: np.ndarray   # [n, 2] float64
    conic: np.ndarray    # [n, 3] float64 (a, b, c) of the inverse projected covariance
    opacity: np.ndarray  # [n] float64
    rgb: np.ndarray      # [n, 3] float64
    depth: np.ndarray    # [n] float64
    radius: np.ndarray   # [n] int32, 0 = culled
    rect: np.ndarray     # [n, 4] int32 tile range (tx0, ty0, tx1, ty1), exclusive max


def preprocess(scene, cam) -> Projected:
    lib = _load()
    n = scene.n
    means, scales = _f32(scene.means, (n, 3)), _f32(scene.scales, (n, 3))
    quats, opac = _f32(scene.quats, (n, 4)), _f32(scene.opacities, (n,))
    sh = _f32(scene.sh)
    out = Projected(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3)), np.zeros(n),
                    np.zeros(n, np.int32), np.zeros((n, 4), np.int32))
    cs = camera_struct(cam)
    lib.orc_preprocess(n, int(scene.sh_degree), _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                       _ptr(sh), C.byref(cs), _ptr(out.mean2d), _ptr(out.conic), _ptr(out.opacity),
                       _ptr(out.rgb), _ptr(out.depth), _ptr(out.radius), _ptr(out.rect))
    return out


def project_cov(mean, scale, quat, cam) -> np.ndarray:
    out = np.zeros(3)
    cs = camera_struct(cam)
    _load().orc_project_cov(_ptr(_f32(mean)), _ptr(_f32(scale)), _ptr(_f32(quat)), C.byref(cs), _ptr(out))
    return out


def tile_rect(mx, my, r, width, height):
    rect = np.zeros(4, np.int32)
    ok = _load().orc_tile_rect(float(mx), float(my), int(r), int(width), int(height), _ptr(rect))
    return bool(ok), rect


def group_grid(width, height, gw, gh):
    tx = (width + TILE - 1) // TILE
    ty = (height + TILE - 1) // TILE
    return tx, ty, (tx + gw - 1) // gw, (ty + gh - 1) // gh


@dataclass
class Bins:
    keys: np.ndarray    # [E] uint64: (gid << 32) | float bits of depth
    vals: np.ndarray    # [E] uint32 splat index
    masks: np.ndarray   # [E] uint16 tile-membership bits
    ranges: np.ndarray  # [G, 2] uint32 [start, end)
    gw: int
    gh: int

    @property
    def num_entries(self) -> int:
        return int(self.keys.shape[0])


def bin_sort(mean2d, radius, depth, width, height, gw=2, gh=2, conic=None, opacity=None) -> Bins:
    """Group entries + masks, sorted by (group, depth, index). Takes the projected mean, radius and
    depth of either side (float32 inputs are widened exactly). With conic [n,3] and opacity [n]
    (float32 values) a tile of a splat's range is kept only if the splat can reach alpha >= 1/255
    in it (the membership test, taken in FP32 as the kernels take it); without them every tile of
    the range is kept."""
    lib = _load()
    mean2d, depth = _f64(mean2d).reshape(-1, 2), _f64(depth).reshape(-1)
    radius = np.ascontiguousarray(radius, np.int32).reshape(-1)
    n = radius.shape[0]
    if (conic is None) != (opacity is None):
        raise ValueError("conic and opacity go together")
    if conic is not None:
        conic = _f64(np.asarray(conic, np.float32)).reshape(n, 3)
        opacity = _f64(np.asarray(opacity, np.float32)).reshape(n)
    E = int(lib.orc_bin_count(n, _ptr(mean2d), _ptr(radius), _ptr(conic), _ptr(opacity), width, height,
                              gw, gh))
    _, _, GX, GY = group_grid(width, height, gw, gh)
    keys = np.zeros(max(E, 1), np.uint64)
    vals = np.zeros(max(E, 1), np.uint32)
    masks = np.zeros(max(E, 1), np.uint16)
    ranges = np.zeros((GX * GY, 2), np.uint32)
    lib.orc_bin(n, _ptr(mean2d), _ptr(radius), _ptr(depth), _ptr(conic), _ptr(opacity), width, height,
                gw, gh, _ptr(keys), _ptr(vals), _ptr(masks), _ptr(ranges))
    return Bins(keys[:E], vals[:E], masks[:E], ranges, gw, gh)


@dataclass
class Image:
    rgb: np.ndarray        # [H, W, 3] (or [npix, 3] for a pixel list)
    T: np.ndarray          # [H, W] final transmittance
    n_contrib: np.ndarray  # [H, W] int32: 1-based list position of the last blended entry, 0 = none
    margin: np.ndarray     # [H, W] smallest relative distance of a threshold decision
    evaluated: int         # (pixel, entry) pairs evaluated before termination
    guard: int             # power > 0 firings (expected 0)
    passing: int = 0       # evaluated pairs with alpha >= 1/255 (one exponential each)


def blend(width, height, mean2d, conic, opacity, rgb, bins: Bins, bg=(0.0, 0.0, 0.0), pixels=None) -> Image:
    """Front-to-back blend of every pixel, or of the (x, y) pairs in `pixels`."""
    lib = _load()
    mean2d, conic = _f64(mean2d).reshape(-1, 2), _f64(conic).reshape(-1, 3)
    opacity, rgb = _f64(opacity).reshape(-1), _f64(rgb).reshape(-1, 3)
    bgv = _f64(bg).reshape(3)
    vals = np.ascontiguousarray(bins.vals, np.uint32)
    masks = np.ascontiguousarray(bins.masks, np.uint16)
    ranges = np.ascontiguousarray(bins.ranges, np.uint32)
    if pixels is None:
        shape, npix, pix = (height, width), width * height, None
    else:
        pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        shape, npix = (pix.shape[0],), pix.shape[0]
    out = np.zeros(npix * 3)
    T = np.zeros(npix)
    nc = np.zeros(npix, np.int32)
    mg = np.zeros(npix)
    counters = np.zeros(3, np.int64)
    lib.orc_blend(width, height, bins.gw, bins.gh, _ptr(mean2d), _ptr(conic), _ptr(opacity), _ptr(rgb),
                  _ptr(vals), _ptr(masks), _ptr(ranges), _ptr(bgv), _ptr(pix), npix, _ptr(out), _ptr(T),
                  _ptr(nc), _ptr(mg), _ptr(counters))
    return Image(out.reshape(*shape, 3), T.reshape(shape), nc.reshape(shape), mg.reshape(shape),
                 int(counters[0]), int(counters[1]), int(counters[2]))


@dataclass
class Grads:
    mean2d: np.ndarray
    conic: np.ndarray
    opacity: np.ndarray
    rgb: np.ndarray


def blend_backward(width, height, mean2d, conic, opacity, rgb, bins: Bins, grad_rgb,
                   bg=(0.0, 0.0, 0.0), pixels=None) -> Grads:
    lib = _load()
    mean2d, conic = _f64(mean2d).reshape(-1, 2), _f64(conic).reshape(-1, 3)
    opacity, rgb = _f64(opacity).reshape(-1), _f64(rgb).reshape(-1, 3)
    n = opacity.shape[0]
    bgv = _f64(bg).reshape(3)
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
    npix = width * height if pix is None else pix.shape[0]
    g = _f64(grad_rgb).reshape(npix, 3)
    out = Grads(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3)))
    lib.orc_blend_backward(width, height, bins.gw, bins.gh, n, _ptr(mean2d), _ptr(conic), _ptr(opacity),
                           _ptr(rgb), _ptr(np.ascontiguousarray(bins.vals, np.uint32)),
                           _ptr(np.ascontiguousarray(bins.masks, np.uint16)),
                           _ptr(np.ascontiguousarray(bins.ranges, np.uint32)), _ptr(bgv), _ptr(pix), npix,
                           _ptr(g), _ptr(out.mean2d), _ptr(out.conic), _ptr(out.opacity), _ptr(out.rgb))
    return out


def render(scene, cam, gw=2, gh=2, bg=(0.0, 0.0, 0.0), membership=True):
    """Full oracle frame: preprocess -> bin/sort -> blend. Returns (Projected, Bins, Image)."""
    pr = preprocess(scene, cam)
    extra = dict(conic=pr.conic, opacity=pr.opacity) if membership else {}
    bins = bin_sort(pr.mean2d, pr.radius, pr.depth, cam.width, cam.height, gw, gh, **extra)
    img = blend(cam.width, cam.height, pr.mean2d, pr.conic, pr.opacity, pr.rgb, bins, bg)
    return pr, bins, img


def psnr(a, b) -> float:
    """10 log10(1 / MSE) of two images clamped to [0, 1]."""
    a = np.clip(np.asarray(a, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(b, np.float64), 0.0, 1.0)
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)
