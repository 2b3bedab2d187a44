"""Seeded synthetic inputs for the SteepGS splitting path.

This module only draws random numbers and builds camera poses.  It holds none
of the method's arithmetic (no projection, compositing, gradients, splitting
matrices or eigen-solves), so that the CPU oracle (``oracle/``) and the CUDA
path (``paper_2505_05587_gb300``) can both consume exactly the same inputs
without sharing any code of the method.

Every array is produced as float32 (the parameter precision of the product);
the oracle promotes those exact values to float64.

Conventions (a reading of the paper, which leaves them open):
  * Gaussian parameters are stored structure-of-arrays:
      means [N,3], log_scales [N,3], quats [N,4] as (w,x,y,z),
      opacity_logit [N], sh [N,K,3] with K = (sh_degree+1)^2.
  * Cameras map world to camera coordinates as x_cam = R x_world + t with
    OpenCV axes (x right, y down, z forward); R is row-major 3x3.
  * Pixels are sampled at integer coordinates; images are [H,W,3] float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Scene-representation sizes (Section 3, "Scene Representation").
SH_COEFFS = {0: 1, 1: 4, 2: 9, 3: 16}


@dataclass
class Scene:
    means: np.ndarray          # [N,3] f32
    log_scales: np.ndarray     # [N,3] f32
    quats: np.ndarray          # [N,4] f32 (w,x,y,z), not necessarily unit
    opacity_logit: np.ndarray  # [N]   f32
    sh: np.ndarray             # [N,K,3] f32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def copy(self) -> "Scene":
        return Scene(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                     self.opacity_logit.copy(), self.sh.copy(), self.sh_degree)


@dataclass
class Camera:
    R: np.ndarray       # [3,3] f32 world->camera rotation (row-major)
    t: np.ndarray       # [3]   f32 world->camera translation
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near_z: float = 0.2


@dataclass
class Settings:
    """Rasterisation constants (3D Gaussian Splatting conventions where the
    paper is silent): 16x16 tiles, alpha clamped to [1/255, 0.99], compositing
    stops below transmittance 1e-4, 3-sigma radius, 0.3 px^2 dilation, the
    projection Jacobian clamped at 1.3 x the half field of view."""
    tile_w: int = 16
    tile_h: int = 16
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    radius_sigma: float = 3.0
    dilation: float = 0.3
    fov_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)

    def smooth(self) -> "Settings":
        """Smooth mode: no skip, no early stop, no alpha clamp, wide support."""
        return Settings(self.tile_w, self.tile_h, 0.0, 1.0, 0.0, 8.0,
                        self.dilation, self.fov_clamp, self.bg)


# ---------------------------------------------------------------------------
# Random draws
# ---------------------------------------------------------------------------

def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    # Uniform on S^3: normalised 4-D standard normal.
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def tiny_scene(seed: int = 0, n: int = 256) -> Scene:
    """Tiny oracle scene: means U([-1,1]^2 x [2,4]); log-scales N(-3,0.5);
    uniform unit quaternions; opacity logit N(0,1); SH degree 0 with the DC
    coefficient uniform in [-sqrt(pi), sqrt(pi)] (an RGB uniform in [0,1]
    under the degree-0 colour map)."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3))
    means[:, 0:2] = rng.uniform(-1.0, 1.0, (n, 2))
    means[:, 2] = rng.uniform(2.0, 4.0, n)
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = _unit_quats(rng, n)
    logit = rng.normal(0.0, 1.0, n)
    dc_lim = math.sqrt(math.pi)
    sh = rng.uniform(-dc_lim, dc_lim, (n, 1, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logit.astype(np.float32),
                 sh.astype(np.float32), 0)


def cluster_means(rng: np.random.Generator, n: int, n_clusters: int = 64,
                  box: float = 5.0) -> np.ndarray:
    """Mixture of anisotropic Gaussian clusters inside [-box, box]^3: centres
    uniform in the box, per-axis std U(0.2, 1.5) under a random rotation, equal
    weights; samples falling outside the box are redrawn."""
    centres = rng.uniform(-box, box, (n_clusters, 3))
    stds = rng.uniform(0.2, 1.5, (n_clusters, 3))
    rots = np.empty((n_clusters, 3, 3))
    for k in range(n_clusters):
        a = rng.standard_normal((3, 3))
        qm, r = np.linalg.qr(a)
        qm = qm * np.sign(np.diag(r))[None, :]
        rots[k] = qm
    out = np.empty((n, 3))
    filled = 0
    while filled < n:
        m = n - filled
        lab = rng.integers(0, n_clusters, m)
        z = rng.standard_normal((m, 3)) * stds[lab]
        pts = centres[lab] + np.einsum("mij,mj->mi", rots[lab], z)
        ok = np.all(np.abs(pts) <= box, axis=1)
        pts = pts[ok]
        out[filled:filled + pts.shape[0]] = pts
        filled += pts.shape[0]
    return out


def cluster_scene(seed: int = 0, n: int = 1_000_000, sh_degree: int = 3) -> Scene:
    """Scene-scale distributions: cluster-mixture means; log-scales N(-4.5,0.7);
    uniform unit quaternions; opacity logit N(-1,1.5); SH coefficients
    N(0,0.2) with the DC coefficient N(0.5,0.2)."""
    rng = np.random.default_rng(seed)
    means = cluster_means(rng, n)
    log_scales = rng.normal(-4.5, 0.7, (n, 3))
    quats = _unit_quats(rng, n)
    logit = rng.normal(-1.0, 1.5, n)
    k = SH_COEFFS[sh_degree]
    sh = rng.normal(0.0, 0.2, (n, k, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.2, (n, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logit.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


def target_image(seed: int, height: int, width: int) -> np.ndarray:
    """Ground-truth stand-in: every channel uniform in [0,1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (height, width, 3)).astype(np.float32)


# ---------------------------------------------------------------------------
# Cameras
# ---------------------------------------------------------------------------

def camera_identity(width: int, height: int, fx: float, fy: float | None = None,
                    centre=(0.0, 0.0, 0.0)) -> Camera:
    """Camera at `centre` looking down +z (R = I, t = -centre)."""
    fy = fx if fy is None else fy
    R = np.eye(3)
    t = -np.asarray(centre, dtype=np.float64)
    return Camera(R.astype(np.float32), t.astype(np.float32), float(fx), float(fy),
                  width / 2.0, height / 2.0, width, height)


def camera_lookat(centre, target, width: int, height: int, fx: float,
                  fy: float | None = None) -> Camera:
    """OpenCV look-at: z toward the target, y along world +y ("up" is -y),
    with a fallback down-vector when the view is parallel to it."""
    fy = fx if fy is None else fy
    c = np.asarray(centre, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    right = np.cross(down, f)
    if np.linalg.norm(right) < 1e-6:
        down = np.array([0.0, 0.0, 1.0])
        right = np.cross(down, f)
    right /= np.linalg.norm(right)
    y = np.cross(f, right)
    R = np.stack([right, y, f])
    t = -R @ c
    return Camera(R.astype(np.float32), t.astype(np.float32), float(fx), float(fy),
                  width / 2.0, height / 2.0, width, height)


SCENE_VIEW = (1237, 822)
RING_RESOLUTIONS = [(1957, 1091), (1600, 1060), (1237, 822), (980, 545), (980, 545),
                    (800, 600), (800, 600), (800, 600)]
SERVE_RESOLUTIONS = [(640, 480), (1237, 822), (1920, 1080)]


def scene_camera(width: int = 1237, height: int = 822, radius: float = 6.0) -> Camera:
    """Single scene-scale view: camera at distance `radius` on -z, looking at the
    origin, fx = fy = width."""
    return camera_lookat((0.0, 0.0, -radius), (0.0, 0.0, 0.0), width, height, width)


def ring_cameras(radius: float = 6.0, resolutions=None) -> list[Camera]:
    """Views on a horizontal ring: centre_k = r (sin phi_k, 0, -cos phi_k),
    phi_k = 2 pi k / K, looking at the origin, fx = fy = width."""
    res = RING_RESOLUTIONS if resolutions is None else resolutions
    k_views = len(res)
    cams = []
    for k, (w, h) in enumerate(res):
        phi = 2.0 * math.pi * k / k_views
        c = (radius * math.sin(phi), 0.0, -radius * math.cos(phi))
        cams.append(camera_lookat(c, (0.0, 0.0, 0.0), w, h, w))
    return cams


def offset_cameras(width: int = 128, height: int = 128, fx: float = 128.0,
                   offset: float = 0.25) -> list[Camera]:
    """Four views at the origin shifted by (+-offset, +-offset, 0), looking down +z."""
    cams = []
    for sx in (-1.0, 1.0):
        for sy in (-1.0, 1.0):
            cams.append(camera_identity(width, height, fx, centre=(sx * offset, sy * offset, 0.0)))
    return cams


def sphere_camera(rng: np.random.Generator, width: int, height: int,
                  radius: float = 6.0) -> Camera:
    """Random pose on the radius sphere (normalised 3-D normal direction),
    looking at the origin."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    return camera_lookat(radius * d, (0.0, 0.0, 0.0), width, height, width)


@dataclass
class Request:
    arrival_s: float
    scene: int
    camera: Camera


def request_stream(seed: int, n_requests: int, rate_hz: float, n_scenes: int,
                   resolutions=None) -> list[Request]:
    """Poisson arrivals at `rate_hz`; scene uniform; pose uniform on the sphere;
    resolution uniform over `resolutions`."""
    res = SERVE_RESOLUTIONS if resolutions is None else resolutions
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    times = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        w, h = res[int(rng.integers(0, len(res)))]
        s = int(rng.integers(0, n_scenes))
        out.append(Request(float(times[i]), s, sphere_camera(rng, w, h)))
    return out


def subset(scene: Scene, idx) -> Scene:
    return Scene(scene.means[idx].copy(), scene.log_scales[idx].copy(),
                 scene.quats[idx].copy(), scene.opacity_logit[idx].copy(),
                 scene.sh[idx].copy(), scene.sh_degree)
