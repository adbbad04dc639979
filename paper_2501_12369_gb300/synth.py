"""Seeded synthetic inputs: splat sets, pinhole cameras and target images.

This module only draws random numbers and builds camera poses. It holds none
of the rasterizer's arithmetic (no projection, no kernel, no compositing), so
both the CUDA path and the CPU oracle can take their inputs from it.

Every array is float32, C-contiguous, in the layouts the C ABI expects:
means [N,3], scales [N,3] (activated, > 0), quats [N,4] as (w, x, y, z),
opacities [N] (activated, in (0,1)), sh [N, (D+1)^2, 3].

The workloads stand in for the scenes the paper trains on (Mip-NeRF 360,
Tanks&Temples, Deep Blending; Sec. 5); no item of those datasets is used.
Scene sizes follow the paper's scale (a few million primitives, Table 3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Half range of the degree-0 SH coefficient whose decoded colour spans [0, 1]:
# 0.5 / (1 / (2 sqrt(pi))).
DC_HALF_RANGE = 0.5 * 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Splats:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Splats":
        idx = np.asarray(idx)
        return Splats(*(np.ascontiguousarray(a[idx]) for a in
                        (self.means, self.scales, self.quats, self.opacities, self.sh)),
                      self.sh_degree)

    def astuple(self):
        return (self.means, self.scales, self.quats, self.opacities, self.sh)


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray  # [4,4] float32, world -> camera, row-major, OpenCV axes
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    width: int
    height: int
    bg: tuple = (0.0, 0.0, 0.0)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera matrix with camera x right, y down, z forward."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:  # looking along the up axis
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f])
    m = np.eye(4)
    m[:3, :3] = rot
    m[:3, 3] = -rot @ eye
    return _f32(m)


def pinhole(eye, width, height, fx, fy=None, near=0.2, bg=(0.0, 0.0, 0.0), target=(0, 0, 0)) -> Camera:
    fy = fx if fy is None else fy
    return Camera(look_at(eye, target), float(fx), float(fy), width / 2.0, height / 2.0,
                  float(near), int(width), int(height), tuple(float(b) for b in bg))


def crop_camera(cam: Camera, x0: int, y0: int, width: int, height: int) -> Camera:
    """The same pinhole seen through a width x height window starting at pixel (x0, y0)."""
    return dataclasses.replace(cam, cx=cam.cx - x0, cy=cam.cy - y0, width=int(width), height=int(height))


def fibonacci_cameras(count, radius, width, height, fx, near=0.2):
    """Cameras on a Fibonacci sphere looking at the origin."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(count):
        y = 1.0 - 2.0 * (i + 0.5) / count
        r = math.sqrt(max(0.0, 1.0 - y * y))
        phi = i * golden
        eye = (radius * r * math.cos(phi), radius * y, radius * r * math.sin(phi))
        cams.append(pinhole(eye, width, height, fx, near=near))
    return cams


def random_pose_cameras(count, radius, resolutions, fx_per_width, seed, near=0.2):
    """Cameras at uniformly random directions on a sphere, resolution drawn from a list."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cams = []
    for _ in range(count):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        cams.append(pinhole(radius * v, w, h, fx_per_width * w, near=near))
    return cams


def _finish(rng, n, means, log_lo, log_hi, sh_degree, dc_only_rgb=True):
    scales = np.exp(rng.uniform(log_lo, log_hi, size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = rng.uniform(-DC_HALF_RANGE, DC_HALF_RANGE, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, size=(n, k - 1, 3))
    return Splats(_f32(means), _f32(scales), _f32(q), _f32(opac), _f32(sh), sh_degree)


def uniform_cube_scene(n=1024, seed=0, sh_degree=0, half=1.0, log_scale=(-4.0, -2.0)) -> Splats:
    """Means uniform in [-half, half]^3; the small forward-render workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-half, half, size=(n, 3))
    return _finish(rng, n, means, log_scale[0], log_scale[1], sh_degree)


def cluster_scene(n, seed=0, sh_degree=3, clusters=20, box=5.0, log_scale=(-5.0, -2.0)) -> Splats:
    """Means from a mixture of anisotropic Gaussian clusters clipped to a [-box, box]^3 volume."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-box, box, size=(clusters, 3))
    sig = rng.uniform(0.3, 1.5, size=(clusters, 3))
    rots = []
    for _ in range(clusters):
        qm, rm = np.linalg.qr(rng.normal(size=(3, 3)))
        qm = qm * np.sign(np.diag(rm))
        rots.append(qm)
    rots = np.stack(rots)
    which = rng.integers(clusters, size=n)
    z = rng.normal(size=(n, 3)) * sig[which]
    means = centres[which] + np.einsum("nij,nj->ni", rots[which], z)
    means = np.clip(means, -box, box)
    return _finish(rng, n, means, log_scale[0], log_scale[1], sh_degree)


def random_target(height, width, seed=1) -> np.ndarray:
    """Target image, planar [3, H, W], uniform in [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _f32(rng.uniform(0.0, 1.0, size=(3, height, width)))


def random_image_grad(height, width, seed=2, scale=1.0) -> np.ndarray:
    """An upstream image gradient, planar [3, H, W], uniform in [-scale, scale]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _f32(rng.uniform(-scale, scale, size=(3, height, width)))


# Named workloads, by what they are.
def small_forward_workload():
    """1,024 splats in [-1,1]^3, SH degree 0, one 64x64 camera at (0,0,4), fx=fy=64."""
    return uniform_cube_scene(1024, seed=0), pinhole((0.0, 0.0, 4.0), 64, 64, 64.0)


def scene_500k_720p():
    """500k clustered splats, SH degree 3, one 1280x720 camera (fx=1000) on the radius-6 sphere."""
    splats = cluster_scene(500_000, seed=0)
    cam = fibonacci_cameras(100, 6.0, 1280, 720, 1000.0)[0]
    return splats, cam


def scene_3m_1080p(num_cameras=100):
    """3M clustered splats, SH degree 3, 100 cameras 1920x1080 (fx=1500) on the radius-6 sphere."""
    splats = cluster_scene(3_000_000, seed=0)
    cams = fibonacci_cameras(num_cameras, 6.0, 1920, 1080, 1500.0)
    return splats, cams


MULTIVIEW_RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080))


def scene_1m_multiview(num_cameras=64, seed=0):
    """1M clustered splats, SH degree 3, cameras at random directions on the radius-5 sphere with
    resolutions drawn from 640x360 / 1280x720 / 1920x1080 (fx = 0.78125 x width, the 1500 / 1920
    of the 1080p workload)."""
    splats = cluster_scene(1_000_000, seed=seed)
    cams = random_pose_cameras(num_cameras, 5.0, MULTIVIEW_RESOLUTIONS, 1500.0 / 1920.0, seed=seed + 1)
    return splats, cams
