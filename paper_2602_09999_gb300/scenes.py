"""Seeded synthetic inputs shaped like the paper's training workloads.

This module holds none of the method's arithmetic: it only draws Gaussian
parameters, cameras and target images.  Both the CUDA path and the FP64
oracle receive exactly these float32 arrays.

The paper trains on Mip-NeRF360, Tanks&Temples and Deep Blending (Sec. 4.1),
which are not available here.  Seeded synthetic scenes stand in for them and
keep only the shapes the paper reports: a few million Gaussians with SH
degree 3 (Sec. 4.2: about 3.8M outdoors, 1.3M indoors), 16x16 tiles and
about one megapixel per view.

Parameter layout (structure of arrays, float32, n Gaussians):
  means [n,3], log_scales [n,3], quats [n,4] (w,x,y,z, unnormalised),
  opacity [n] (logits), sh_dc [n,3], sh_rest [n,15,3].
Cameras are pinhole with OpenCV axes (x right, y down, z forward),
world->camera rotation R (row-major) and translation t, focal lengths from a
60 degree horizontal field of view and the principal point at the image
centre.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PARAM_NAMES = ("means", "log_scales", "quats", "opacity", "sh_dc", "sh_rest")
NEAR_PLANE = 0.2


@dataclass
class Camera:
    R: np.ndarray          # [3,3] float32, world -> camera, row-major
    t: np.ndarray          # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = NEAR_PLANE
    cam_pos: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    time: float = 0.0      # timestamp of the view (dynamic Gaussians)

    @property
    def tiles(self):
        return (self.width + 15) // 16, (self.height + 15) // 16


def look_at(eye, target, width, height, fov_x_deg=60.0, up=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; world up is +y."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    f = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return Camera(R=R, t=t, fx=float(np.float32(f)), fy=float(np.float32(f)),
                  cx=float(np.float32(width / 2.0)), cy=float(np.float32(height / 2.0)),
                  width=int(width), height=int(height), near=NEAR_PLANE,
                  cam_pos=eye.astype(np.float32))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n):
    dc = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    rest = (0.05 * rng.standard_normal((n, 15, 3))).astype(np.float32)
    return dc, rest


def tiny_scene(n=10_000, seed=0):
    """Tiny scene: means U[-1,1]^3, log-scales N(-4,0.5), unit quaternions
    from N(0,I4), opacity logits N(0,1), SH DC U(0,1), rest N(0,0.05)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.normal(-4.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n).astype(np.float32)
    dc, rest = _sh(rng, n)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity=opacity, sh_dc=dc,
                sh_rest=rest)


def tiny_camera(width=256, height=256):
    return look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), width, height)


def _random_rotations(rng, k):
    q = rng.standard_normal((k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def outdoor_scene(n=3_000_000, seed=0):
    """Outdoor-shaped scene: 90% from a mixture of 64 anisotropic 3D
    Gaussians (centres at random directions times 20 u^2, per-axis std
    U(0.2,2)(1 + r/10), random rotations, Dirichlet(1) weights), 10% on a
    shell of radius U(18,20); log-scales N(-4.5,1), opacity logits
    N(-1,1.5), SH degree 3."""
    rng = np.random.default_rng(seed)
    k = 64
    dirs = rng.standard_normal((k, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radius = 20.0 * rng.uniform(0.0, 1.0, k) ** 2
    centres = dirs * radius[:, None]
    stds = rng.uniform(0.2, 2.0, (k, 3)) * (1.0 + radius[:, None] / 10.0)
    rots = _random_rotations(rng, k)
    weights = rng.dirichlet(np.ones(k))
    n_mix = int(round(0.9 * n))
    comp = rng.choice(k, size=n_mix, p=weights)
    local = rng.standard_normal((n_mix, 3)) * stds[comp]
    mix = centres[comp] + np.einsum("nij,nj->ni", rots[comp], local)
    n_shell = n - n_mix
    sd = rng.standard_normal((n_shell, 3))
    sd /= np.linalg.norm(sd, axis=1, keepdims=True)
    shell = sd * rng.uniform(18.0, 20.0, n_shell)[:, None]
    means = np.concatenate([mix, shell]).astype(np.float32)
    perm = rng.permutation(n)
    means = means[perm]
    log_scales = rng.normal(-4.5, 1.0, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(-1.0, 1.5, n).astype(np.float32)
    dc, rest = _sh(rng, n)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity=opacity, sh_dc=dc,
                sh_rest=rest)


def orbit_cameras(count=100, width=1237, height=822, radius=6.0, seed=1):
    """Cameras on a seeded orbit of the origin: azimuth U(0, 2pi),
    elevation U(-10, 30) degrees."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(count):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(-10.0, 30.0))
        eye = radius * np.array([math.cos(el) * math.cos(az), math.sin(el),
                                 math.cos(el) * math.sin(az)])
        cams.append(look_at(eye, (0.0, 0.0, 0.0), width, height))
    return cams


def indoor_scene(n=2_500_000, seed=0):
    """Indoor-shaped scene in the box [-5,5]x[-2,2]x[-4,4]: 60% within 0.1 of
    the six faces (face chosen by area, offset U(0,0.1) inward), 40% uniform;
    log-scales N(-4,0.8), opacity logits N(-1,1.5), SH degree 3."""
    rng = np.random.default_rng(seed)
    half = np.array([5.0, 2.0, 4.0])
    n_wall = int(round(0.6 * n))
    areas = np.array([half[1] * half[2], half[1] * half[2], half[0] * half[2],
                      half[0] * half[2], half[0] * half[1], half[0] * half[1]])
    face = rng.choice(6, size=n_wall, p=areas / areas.sum())
    pts = rng.uniform(-half, half, (n_wall, 3))
    axis = face // 2
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    off = rng.uniform(0.0, 0.1, n_wall)
    pts[np.arange(n_wall), axis] = sign * (half[axis] - off)
    inner = rng.uniform(-half, half, (n - n_wall, 3))
    means = np.concatenate([pts, inner]).astype(np.float32)
    means = means[rng.permutation(n)]
    log_scales = rng.normal(-4.0, 0.8, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(-1.0, 1.5, n).astype(np.float32)
    dc, rest = _sh(rng, n)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity=opacity, sh_dc=dc,
                sh_rest=rest)


def indoor_cameras(count=8, width=1264, height=832, seed=2):
    """In-room cameras: eyes uniform in the box shrunk by 1, yaw U(0, 2pi),
    pitch U(-15, 15) degrees."""
    rng = np.random.default_rng(seed)
    half = np.array([4.0, 1.0, 3.0])
    cams = []
    for _ in range(count):
        eye = rng.uniform(-half, half)
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        pitch = math.radians(rng.uniform(-15.0, 15.0))
        d = np.array([math.cos(pitch) * math.cos(yaw), math.sin(pitch),
                      math.cos(pitch) * math.sin(yaw)])
        cams.append(look_at(eye, eye + d, width, height))
    return cams


UNEVEN_SIZES = ((1237, 822), (960, 640), (1600, 1064), (640, 426))


def uneven_cameras(sizes=UNEVEN_SIZES, radius=6.0, seed=3):
    """Orbit cameras of uneven resolutions (the precision-variant batch)."""
    cams = []
    rng = np.random.default_rng(seed)
    for (w, h) in sizes:
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(-10.0, 30.0))
        eye = radius * np.array([math.cos(el) * math.cos(az), math.sin(el),
                                 math.cos(el) * math.sin(az)])
        cams.append(look_at(eye, (0.0, 0.0, 0.0), w, h))
    return cams


def target_image(width, height, view=0):
    """Target image [3,H,W], i.i.d. U(0,1) per pixel and channel, seed 1000 + view."""
    rng = np.random.default_rng(1000 + view)
    return rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def small_scene(n, seed, spread=1.0, log_scale_mean=-2.5, log_scale_std=0.4,
                opacity_mean=0.0, opacity_std=1.0, depth=4.0):
    """Small scenes for parity tests: means U[-spread,spread]^2 in x,y around
    the origin and U(-spread,spread)/2 in z."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n),
                      rng.uniform(-spread / 2, spread / 2, n)], 1).astype(np.float32)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(opacity_mean, opacity_std, n).astype(np.float32)
    dc, rest = _sh(rng, n)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity=opacity, sh_dc=dc,
                sh_rest=rest)


# ---------------------------------------------------------------------------
# dynamic (4D) workload: Gaussians with a linear velocity and a temporal
# centre (the linear-velocity form of the conditional Gaussian, Sec. 3.4)
# ---------------------------------------------------------------------------
DYN_TIMESTAMPS = 150
DYN_SIGMA_T = 0.1


def dynamic_scene(n=600_000, seed=5, radius=1.5):
    """Object-centred dynamic scene (shaped like the synthetic objects the
    paper's 4D experiments use): means N(0, 0.5^2 I) inside a ball of
    `radius`, log-scales N(-4.5, 0.6), opacity logits N(-1, 1.5), SH as
    elsewhere; velocity N(0, 0.05^2 I), temporal centre U(0, 1),
    sigma_t = 0.1."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, 0.5, (n, 3))
    r = np.linalg.norm(means, axis=1, keepdims=True)
    means = np.where(r > radius, means * (radius / np.maximum(r, 1e-12)), means).astype(np.float32)
    log_scales = rng.normal(-4.5, 0.6, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(-1.0, 1.5, n).astype(np.float32)
    dc, rest = _sh(rng, n)
    velocity = rng.normal(0.0, 0.05, (n, 3)).astype(np.float32)
    t0 = rng.uniform(0.0, 1.0, n).astype(np.float32)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity=opacity, sh_dc=dc,
                sh_rest=rest, velocity=velocity, t0=t0, sigma_t=DYN_SIGMA_T)


def dynamic_cameras(count=6, seed=6, radius=4.0, min_size=(800, 800), max_size=(1352, 1014),
                    timestamps=DYN_TIMESTAMPS, sizes=None):
    """Views of the dynamic scene: on a sphere of `radius` around the object
    (azimuth U(0, 2pi), elevation U(-20, 40) degrees), each at a random one of
    `timestamps` evenly spaced times in [0, 1] and, unless `sizes` is given,
    a random resolution between min_size and max_size."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(count):
        az = rng.uniform(0.0, 2.0 * np.pi)
        el = np.deg2rad(rng.uniform(-20.0, 40.0))
        eye = radius * np.array([np.cos(el) * np.sin(az), -np.sin(el), np.cos(el) * np.cos(az)])
        if sizes is not None:
            w, h = sizes[i % len(sizes)]
        else:
            w = int(rng.integers(min_size[0], max_size[0] + 1))
            h = int(rng.integers(min_size[1], max_size[1] + 1))
        cam = look_at(eye, (0.0, 0.0, 0.0), w, h)
        cam.time = float(rng.integers(0, timestamps)) / (timestamps - 1)
        cams.append(cam)
    return cams
