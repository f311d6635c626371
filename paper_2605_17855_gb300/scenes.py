"""Seeded synthetic Gaussian scenes and pinhole cameras.

This module only draws inputs. It holds no projection, binning, sorting or blending arithmetic, so
the CUDA path and the FP64 oracle consume the very same float32 arrays. Every generator is fully
determined by its seed.

The workloads stand in for the captured scenes the paper evaluates on (Section 5.1, Table 4:
Tanks&Temples, Deep Blending, Synthetic-NeRF, Synthetic-NSVF), whose trained Gaussian models are not
available. The workloads:

  box_2k_128                  2,000 splats in a camera-space box, SH degree 0, 128x128, one camera (seed 0)
  mixture_1p5m_1600x1064      1.5M splats from a 256-component mixture, SH degree 3, 1600x1064, 8 orbit
                              cameras (seed 2)
  clusters_6m_3840x2160       6M splats in 64 tight clusters with 5% needles, SH degree 3, 3840x2160
                              (seed 3)
  box_500k_1024_8cams         500k splats from the box generator, 8 jittered cameras at 1024x1024 (seed 4)
  resident_scenes_200k_800k_1p5m_3m  four scenes of 200k/800k/1.5M/3M splats from the box generator,
                              SH degree 3 (seeds 5..8)

Conventions (shared by both sides):
  * quaternions are (w, x, y, z) and unit norm;
  * scales are linear standard deviations along the splat's local axes;
  * SH coefficients are laid out [n, (d+1)^2, 3], coefficient-major, index l*l + (m + l);
  * cameras map world to camera space as p_c = R p_w + t with camera x right, y down, z forward;
    pixel (i, j) is sampled at image coordinates (i, j); the principal point is ((W-1)/2, (H-1)/2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NEAR_Z = 0.2
# Value of the constant (l = 0) real spherical harmonic. Used only to turn a desired base colour
# into the DC coefficient that produces it.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclass
class Scene:
    means: np.ndarray      # [n, 3] float32, world space
    scales: np.ndarray     # [n, 3] float32, linear standard deviations
    quats: np.ndarray      # [n, 4] float32, (w, x, y, z), unit norm
    opacities: np.ndarray  # [n] float32 in (0, 1)
    sh: np.ndarray         # [n, (d+1)^2, 3] float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def nbytes(self) -> int:
        return int(self.means.nbytes + self.scales.nbytes + self.quats.nbytes
                   + self.opacities.nbytes + self.sh.nbytes)

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.means[idx]), np.ascontiguousarray(self.scales[idx]),
                     np.ascontiguousarray(self.quats[idx]), np.ascontiguousarray(self.opacities[idx]),
                     np.ascontiguousarray(self.sh[idx]), self.sh_degree)


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray        # [3, 3] float32, world -> camera rotation (row-major)
    t: np.ndarray        # [3] float32
    cam_pos: np.ndarray  # [3] float32, camera centre in world coordinates
    near: float = NEAR_Z

    @property
    def pixels(self) -> int:
        return self.width * self.height


def focal_from_hfov(width: int, hfov_deg: float) -> float:
    return float(np.float32(0.5 * width / math.tan(math.radians(hfov_deg) / 2)))


def _camera(width, height, R, t, hfov_deg=60.0) -> Camera:
    f = focal_from_hfov(width, hfov_deg)
    R32 = np.asarray(R, np.float32).reshape(3, 3)
    t32 = np.asarray(t, np.float32).reshape(3)
    pos = -(R32.astype(np.float64).T @ t32.astype(np.float64))
    return Camera(int(width), int(height), f, f, float(np.float32((width - 1) / 2)),
                  float(np.float32((height - 1) / 2)), R32, t32, pos.astype(np.float32))


def identity_camera(width: int, height: int, hfov_deg: float = 60.0) -> Camera:
    """Camera at the origin looking down +z (world space == camera space)."""
    return _camera(width, height, np.eye(3), np.zeros(3), hfov_deg)


def look_at_camera(eye, target, width: int, height: int, hfov_deg: float = 60.0,
                   up=(0.0, 1.0, 0.0)) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    down = -(up - np.dot(up, fwd) * fwd)
    down /= np.linalg.norm(down)
    right = np.cross(down, fwd)
    R = np.stack([right, down, fwd])
    t = -R @ eye
    return _camera(width, height, R, t, hfov_deg)


def orbit_cameras(count: int, radius: float, width: int, height: int, hfov_deg: float = 60.0,
                  yaw_offset_deg: float = 0.0):
    """`count` equatorial cameras on a circle of `radius` about the origin, looking at it, up +y.
    Camera k sits at yaw k * 360/count degrees; yaw 0 is at (0, 0, -radius)."""
    cams = []
    for k in range(count):
        yaw = math.radians(yaw_offset_deg + k * 360.0 / count)
        eye = (radius * math.sin(yaw), 0.0, -radius * math.cos(yaw))
        cams.append(look_at_camera(eye, (0.0, 0.0, 0.0), width, height, hfov_deg))
    return cams


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh_from_colour(rng, colour, degree, rest_std=0.1):
    n = colour.shape[0]
    sh = np.zeros((n, (degree + 1) ** 2, 3), np.float32)
    sh[:, 0, :] = (colour - 0.5) / _Y00
    if degree > 0:
        sh[:, 1:, :] = rest_std * rng.standard_normal((n, (degree + 1) ** 2 - 1, 3))
    return sh


def box_scene(n: int, seed: int = 0, sh_degree: int = 0, log_scale_mean: float = -3.5,
              log_scale_std: float = 0.5, opacity_logit_std: float = 1.5) -> Scene:
    """Box generator: means uniform in [-1,1]^2 x [2,6] (camera-space box of the identity camera),
    log-scales ~ N(mean, std) per axis, uniform unit quaternions, opacity = sigmoid(N(0, 1.5)),
    base colour uniform in [0,1] (higher SH bands ~ N(0, 0.1) when sh_degree > 0)."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3), np.float64)
    means[:, 0:2] = rng.uniform(-1.0, 1.0, (n, 2))
    means[:, 2] = rng.uniform(2.0, 6.0, n)
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, (n, 3)))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, opacity_logit_std, n))
    colour = rng.uniform(0.0, 1.0, (n, 3))
    sh = _sh_from_colour(rng, colour, sh_degree)
    return Scene(means.astype(np.float32), scales.astype(np.float32), quats,
                 opac.astype(np.float32), sh, sh_degree)


def _mixture_means(rng, n, components, cluster_std, radius):
    u = rng.standard_normal((components, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    centres = u * (radius * rng.uniform(0.0, 1.0, (components, 1)) ** (1.0 / 3.0))
    comp = rng.integers(0, components, n)
    pts = centres[comp] + cluster_std * rng.standard_normal((n, 3))
    out = np.linalg.norm(pts, axis=1) > radius
    while np.any(out):  # redraw the few samples that left the ball
        k = int(out.sum())
        pts[out] = centres[comp[out]] + cluster_std * rng.standard_normal((k, 3))
        out = np.linalg.norm(pts, axis=1) > radius
    return pts


def mixture_scene(n: int, seed: int, components: int = 256, cluster_std: float = 0.3,
                  radius: float = 4.0, log_scale_mean: float = -4.5, log_scale_std: float = 0.8,
                  opacity_logit_std: float = 2.0, sh_degree: int = 3,
                  needle_fraction: float = 0.0, needle_ratio: float = 100.0) -> Scene:
    """Mixture generator: means from an equal-weight Gaussian mixture whose centres are uniform in the
    ball of `radius` (samples redrawn until inside it); log-scales ~ N(mean, std) per axis; opacity =
    sigmoid(N(0, std)); SH DC ~ U[0,1] (raw coefficient), higher bands ~ N(0, 0.1). A
    `needle_fraction` of splats get scales (10 s, s/10, s/10), an axis ratio of `needle_ratio`."""
    rng = np.random.default_rng(seed)
    means = _mixture_means(rng, n, components, cluster_std, radius)
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, (n, 3)))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, opacity_logit_std, n))
    sh = np.zeros((n, (sh_degree + 1) ** 2, 3), np.float32)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if sh_degree > 0:
        sh[:, 1:, :] = 0.1 * rng.standard_normal((n, (sh_degree + 1) ** 2 - 1, 3))
    if needle_fraction > 0:
        k = int(round(needle_fraction * n))
        idx = rng.choice(n, k, replace=False)
        s = scales[idx, 0]
        f = math.sqrt(needle_ratio)
        scales[idx] = np.stack([s * f, s / f, s / f], axis=1)
    return Scene(means.astype(np.float32), scales.astype(np.float32), quats,
                 opac.astype(np.float32), sh, sh_degree)


# ----------------------------------------------------------------------------------------------
# The five workload configurations.

def box_2k_128():
    """2,000 splats, seed 0, SH degree 0, 128x128, 60 deg horizontal FOV, identity camera."""
    return box_scene(2000, seed=0, sh_degree=0), [identity_camera(128, 128, 60.0)]


def mixture_1p5m_1600x1064(n: int = 1_500_000, cams: int = 8, width: int = 1600, height: int = 1064):
    """1.5M-splat mixture scene (256 clusters, std 0.3, radius 4), SH degree 3, eight orbit
    cameras at radius 5 rendering 1600x1064."""
    return (mixture_scene(n, seed=2, components=256, cluster_std=0.3, radius=4.0,
                          log_scale_mean=-4.5, log_scale_std=0.8, opacity_logit_std=2.0, sh_degree=3),
            orbit_cameras(cams, 5.0, width, height))


def clusters_6m_3840x2160(n: int = 6_000_000, cams: int = 4, width: int = 3840, height: int = 2160):
    """6M splats in 64 tight clusters (std 0.15) with 5% needles (axis ratio 100:1), SH degree 3,
    four orbit views at radius 5 rendering 3840x2160."""
    return (mixture_scene(n, seed=3, components=64, cluster_std=0.15, radius=4.0,
                          log_scale_mean=-4.5, log_scale_std=0.8, opacity_logit_std=2.0, sh_degree=3,
                          needle_fraction=0.05, needle_ratio=100.0),
            orbit_cameras(cams, 5.0, width, height))


def box_500k_1024_8cams(n: int = 500_000, cams: int = 8, size: int = 1024):
    """500k splats from the box generator; eight cameras yaw-jittered by up to +-10 degrees about the
    scene centre (0, 0, 4) at 1024x1024."""
    scene = box_scene(n, seed=4, sh_degree=0)
    rng = np.random.default_rng(1004)
    out = []
    for k in range(cams):
        yaw = math.radians(rng.uniform(-10.0, 10.0)) if k else 0.0
        centre = np.array([0.0, 0.0, 4.0])
        eye = centre + 4.0 * np.array([math.sin(yaw), 0.0, -math.cos(yaw)])
        out.append(look_at_camera(eye, centre, size, size, 60.0))
    return scene, out


def resident_scenes_200k_800k_1p5m_3m(sizes=(200_000, 800_000, 1_500_000, 3_000_000)):
    """Four resident scenes from the box generator with SH degree 3."""
    return [box_scene(n, seed=5 + i, sh_degree=3) for i, n in enumerate(sizes)]


SERVING_RESOLUTIONS = ((640, 480), (1280, 720), (1920, 1080), (2 * 2048, 2048))
