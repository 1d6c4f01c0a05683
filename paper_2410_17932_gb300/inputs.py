"""Seeded synthetic inputs for the foveated-periphery Gaussian-splatting path.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It only draws random numbers and builds camera poses; it holds
none of the renderer's arithmetic (no projection, no SH evaluation, no
compositing).

The scenes stand in for the trained MipNeRF-360 / Tanks&Temples scenes that the
paper renders (Sec. 5); they keep the paper's primitive counts (0.3-0.5 M
periphery Gaussians, Sec. 4 "Training"; 3 M as a dense case) and its per-eye
resolution of 2016 x 2240 (Sec. 5.1, Tab. 1) with a 512 x 512 foveal crop
(Sec. 4 "Fovea Size in Pixels").

Layouts (all float32, C-contiguous, structure of arrays):
  means          [N, 3]   world-space centres
  log_scales     [N, 3]   per-axis log standard deviations
  quats          [N, 4]   rotation quaternions (w, x, y, z), not normalised
  opacity_logits [N]      opacity before the sigmoid
  sh             [N, K, 3] SH coefficients, K = (degree + 1)^2, band-major
A camera maps x_cam = R @ x_world + t, +z forward, +y down; pixel (i, j) has
its centre at (i + 0.5, j + 0.5).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 20241017


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.means[idx]),
                     np.ascontiguousarray(self.log_scales[idx]),
                     np.ascontiguousarray(self.quats[idx]),
                     np.ascontiguousarray(self.opacity_logits[idx]),
                     np.ascontiguousarray(self.sh[idx]), self.sh_degree)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.means, self.log_scales, self.quats,
                                      self.opacity_logits, self.sh))


@dataclasses.dataclass
class Camera:
    R: np.ndarray            # [3, 3] world -> camera rotation
    t: np.ndarray            # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2
    scene: int = 0
    # Half-field-of-view tangents of the full frame this view belongs to.  They
    # bound the projection-Jacobian clamp; a foveal crop keeps its parent's
    # values so that it sees the same splats as the matching window.
    tan_fovx: float = 0.0
    tan_fovy: float = 0.0

    def __post_init__(self):
        self.R = np.ascontiguousarray(self.R, dtype=np.float32).reshape(3, 3)
        self.t = np.ascontiguousarray(self.t, dtype=np.float32).reshape(3)
        if self.tan_fovx == 0.0:
            self.tan_fovx = self.width / (2.0 * self.fx)
        if self.tan_fovy == 0.0:
            self.tan_fovy = self.height / (2.0 * self.fy)

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """Off-axis pinhole view of the window [x0, x0+w) x [y0, y0+h)."""
        return Camera(self.R.copy(), self.t.copy(), self.fx, self.fy,
                      self.cx - x0, self.cy - y0, w, h, self.znear, self.scene,
                      self.tan_fovx, self.tan_fovy)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float32)
    # uniform random unit quaternions: a normalised Gaussian 4-vector
    q /= np.linalg.norm(q, axis=1, keepdims=True).astype(np.float32)
    return q


def uniform_box_scene(n: int, seed: int, xy=(-1.0, 1.0), z=(2.0, 6.0),
                      log_scale=(-3.5, 0.5), opacity=(0.0, 1.0),
                      sh_degree: int = 0, sh_hi_std: float = 0.05) -> Scene:
    """Means uniform in a box in front of the camera (the 200x200 plain case)."""
    rng = _rng(seed)
    means = np.empty((n, 3), np.float32)
    means[:, 0] = rng.uniform(xy[0], xy[1], n)
    means[:, 1] = rng.uniform(xy[0], xy[1], n)
    means[:, 2] = rng.uniform(z[0], z[1], n)
    log_scales = rng.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32)
    quats = _random_quats(rng, n)
    opacity_logits = rng.normal(opacity[0], opacity[1], n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.empty((n, K, 3), np.float32)
    # DC coefficients ~ U[0, 1]; higher bands ~ N(0, sh_hi_std)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_hi_std, (n, K - 1, 3))
    return Scene(means, log_scales, quats, opacity_logits, sh, sh_degree)


def _room_clusters(rng, n_clusters: int, room: float):
    """Cluster geometry of the room generator: centres ~ U(room), unit plane
    normals, two in-plane axes and in-plane extents ~ U[0.3, 3] m."""
    centres = rng.uniform(-room, room, (n_clusters, 3))
    normals = rng.standard_normal((n_clusters, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    helper = np.where(np.abs(normals[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    ax_u = np.cross(normals, helper)
    ax_u /= np.linalg.norm(ax_u, axis=1, keepdims=True)
    ax_v = np.cross(normals, ax_u)
    ext = rng.uniform(0.3, 3.0, (n_clusters, 2))
    return centres, normals, ax_u, ax_v, ext


def _cluster_points(rng, clusters, n: int, room: float, thick: float = 0.02) -> np.ndarray:
    """n points assigned uniformly to the clusters, Gaussian in-plane spread, 2 cm thickness."""
    centres, normals, ax_u, ax_v, ext = clusters
    cl = rng.integers(0, len(centres), n)
    g = rng.standard_normal((n, 3))
    pts = (centres[cl]
           + ax_u[cl] * (g[:, :1] * ext[cl, :1])
           + ax_v[cl] * (g[:, 1:2] * ext[cl, 1:2])
           + normals[cl] * (g[:, 2:3] * thick))
    return np.clip(pts, -room, room).astype(np.float32)


def clustered_room_scene(n: int, seed: int, log_scale=(-4.0, 0.7),
                         opacity=(0.0, 1.0), n_clusters: int = 256,
                         room: float = 10.0, sh_degree: int = 3,
                         sh_hi_std: float = 0.05) -> Scene:
    """Splats on 256 thin anisotropic planar clusters inside a 20 m room.

    Each cluster has a centre ~ U(room), a random plane normal, two in-plane
    axes, in-plane extents ~ U[0.3, 3] m and a 2 cm thickness; splats are
    assigned uniformly to clusters and clipped to the room.
    """
    rng = _rng(seed)
    clusters = _room_clusters(rng, n_clusters, room)
    means = _cluster_points(rng, clusters, n, room)
    log_scales = rng.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32)
    quats = _random_quats(rng, n)
    opacity_logits = rng.normal(opacity[0], opacity[1], n).astype(np.float32)
    K = (sh_degree + 1) ** 2
    sh = np.empty((n, K, 3), np.float32)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_hi_std, (n, K - 1, 3)).astype(np.float32)
    return Scene(means, log_scales, quats, opacity_logits, sh, sh_degree)


def neural_points(n: int, seed: int, cluster_seed: int, n_clusters: int = 256,
                  room: float = 10.0) -> np.ndarray:
    """[n, 3] float32 neural-point positions on the planar clusters of the room
    generator seeded with `cluster_seed` (the same surfaces as that scene's
    Gaussians), drawn with their own seed."""
    clusters = _room_clusters(_rng(cluster_seed), n_clusters, room)
    return _cluster_points(_rng(seed), clusters, n, room)


def synthetic_depth_map(width: int, height: int, seed: int, n_rects: int = 24):
    """A float32 Eq. 1 depth map and final transmittance of `n_rects` layered
    fronto-slanted planar patches: per pixel, depth = z_surface * (1 - T) as a
    single surface of opacity 1 - T would give; the background has T = 1."""
    rng = _rng(seed)
    z = np.zeros((height, width), np.float64)
    T = np.ones((height, width), np.float64)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    for _ in range(n_rects):
        x0, y0 = rng.integers(0, width), rng.integers(0, height)
        w, h = rng.integers(1, width // 2 + 2), rng.integers(1, height // 2 + 2)
        a = rng.choice([rng.uniform(0.0, 0.3), rng.uniform(0.3, 0.7), rng.uniform(0.7, 0.9999)])
        z0, gx, gy = rng.uniform(1.0, 8.0), rng.normal(0, 2e-3), rng.normal(0, 2e-3)
        sel = (xx >= x0) & (xx < x0 + w) & (yy >= y0) & (yy < y0 + h)
        z[sel] = np.maximum(0.3, z0 + gx * (xx[sel] - x0) + gy * (yy[sel] - y0))
        T[sel] = 1.0 - a
    depth = (z * (1.0 - T)).astype(np.float32)
    return depth, T.astype(np.float32)


def _yaw_pitch(yaw: float, pitch: float) -> np.ndarray:
    """World->camera rotation for a head that turned by yaw (about y), pitch (about x)."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    Ry = np.array([[cy_, 0.0, -sy_], [0.0, 1.0, 0.0], [sy_, 0.0, cy_]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, cp, sp], [0.0, -sp, cp]])
    return Rx @ Ry


VR_W, VR_H = 2016, 2240
VR_FX = (VR_W / 2) / math.tan(math.radians(50.0))   # 100-degree horizontal FOV
IPD = 0.063


def stereo_eyes(seed: int, head=(0.0, 0.0, 0.0), width=VR_W, height=VR_H,
                scene: int = 0, pitch_std: float = 0.15) -> List[Camera]:
    """Two eyes 63 mm apart along the head's x axis, seeded head yaw and pitch."""
    rng = _rng(seed)
    yaw = rng.uniform(-math.pi, math.pi)
    pitch = rng.normal(0.0, pitch_std)
    R = _yaw_pitch(yaw, pitch)
    fx = (width / 2) / math.tan(math.radians(50.0))
    cams = []
    for side in (-1.0, 1.0):
        eye = np.asarray(head, np.float64) + side * (IPD / 2) * R[0]   # camera x axis in world
        t = -R @ eye
        cams.append(Camera(R, t, fx, fx, width / 2.0, height / 2.0, width, height,
                           scene=scene))
    return cams


def foveal_crop(cam: Camera, seed: int, size: int = 512, tile: int = 16,
                aligned: bool = True) -> Camera:
    """A size x size foveal window around a seeded gaze point, as an off-axis view."""
    rng = _rng(seed)
    gx = rng.uniform(size / 2, cam.width - size / 2)
    gy = rng.uniform(size / 2, cam.height - size / 2)
    x0 = int(gx - size / 2)
    y0 = int(gy - size / 2)
    if aligned:
        x0 -= x0 % tile
        y0 -= y0 % tile
    else:
        x0 += (1 if x0 % tile == 0 else 0)
    x0 = max(0, min(x0, cam.width - size))
    y0 = max(0, min(y0, cam.height - size))
    return cam.crop(x0, y0, size, size)


def identity_camera(width=200, height=200, f=200.0, scene: int = 0) -> Camera:
    return Camera(np.eye(3), np.zeros(3), f, f, width / 2.0, height / 2.0, width,
                  height, scene=scene)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's primitive counts and
# resolutions; the random recipes are this library's choice.

def plain_200(seed: Optional[int] = None):
    """200x200 plain forward render of 5,000 SH-0 Gaussians in a box."""
    seed = SEED_BASE + 0 if seed is None else seed
    return [uniform_box_scene(5000, seed)], [identity_camera()]


def periphery_stereo_05m(n: int = 500_000, seed: Optional[int] = None):
    """Foveated periphery stereo frame: 0.5 M SH-3 Gaussians, 2016x2240 per eye."""
    seed = SEED_BASE + 1 if seed is None else seed
    sc = clustered_room_scene(n, seed)
    return [sc], stereo_eyes(seed + 1000)


def dense_stereo_3m(n: int = 3_000_000, seed: Optional[int] = None, aligned=True):
    """Dense stereo frame of 3 M SH-3 Gaussians plus a 512x512 foveal crop per eye."""
    seed = SEED_BASE + 2 if seed is None else seed
    sc = clustered_room_scene(n, seed, log_scale=(-5.0, 0.7), opacity=(0.5, 1.0))
    eyes = stereo_eyes(seed + 1000)
    crops = [foveal_crop(e, seed + 2000 + i, aligned=aligned) for i, e in enumerate(eyes)]
    return [sc], eyes + crops


def foveal_points_5m(n_points: int = 5_000_000, seed: Optional[int] = None, size: int = 512):
    """Foveal neural-point culling: the periphery scene's left eye, a size x size
    foveal crop at a seeded gaze (the subfrustum), and 5 M neural points on the
    same surfaces as the scene's 0.5 M Gaussians."""
    seed = SEED_BASE + 1 if seed is None else seed
    scenes, eyes = periphery_stereo_05m(seed=seed)
    crop = foveal_crop(eyes[0], seed + 5000, size=size, aligned=False)
    pts = neural_points(n_points, seed + 6000, cluster_seed=seed)
    return scenes, eyes[0], crop, pts


def training_view_1m(n: int = 1_000_000, seed: Optional[int] = None):
    """One 1264x832 training camera over 1 M SH-3 Gaussians, with upstream grads."""
    seed = SEED_BASE + 3 if seed is None else seed
    sc = clustered_room_scene(n, seed)
    rng = _rng(seed + 1000)
    R = _yaw_pitch(rng.uniform(-math.pi, math.pi), rng.normal(0, 0.1))
    cam = Camera(R, np.zeros(3), 1000.0, 1000.0, 632.0, 416.0, 1264, 832)
    return [sc], [cam]


def upstream_grads(cams: List[Camera], seed: int):
    """dL/dRGB [3,H,W] and dL/dDepth [H,W] ~ N(0, 1) per view."""
    rng = _rng(seed)
    out = []
    for c in cams:
        out.append((rng.standard_normal((3, c.height, c.width)).astype(np.float32),
                    rng.standard_normal((c.height, c.width)).astype(np.float32)))
    return out


def batched_multiview(seed: Optional[int] = None, sizes=(100_000, 500_000, 1_000_000, 2_000_000),
                      scale: float = 1.0):
    """Four scenes and 32 views of uneven size for the batched persistent path.

    16 foveal crops of 384..768 px (4 per scene), 12 stereo eyes (pairs 0-1 on
    scene 0, 2-3 on scene 1, 4 on scene 2, 5 on scene 3) and one 1264x832
    training view per scene.  `scale` shrinks the scene sizes for tests.
    """
    seed = SEED_BASE + 4 if seed is None else seed
    scenes = [clustered_room_scene(max(1, int(n * scale)), seed + 10 * i)
              for i, n in enumerate(sizes)]
    rng = _rng(seed + 500)
    views: List[Camera] = []
    pair_scene = [0, 0, 1, 1, 2, 3]
    eyes_by_scene = {s: [] for s in range(4)}
    for p, s in enumerate(pair_scene):
        for e in stereo_eyes(seed + 1000 + p, scene=s):
            views.append(e)
            eyes_by_scene[s].append(e)
    for s in range(4):
        for k in range(4):
            size = int(rng.choice(np.arange(384, 769, 64)))
            base = eyes_by_scene[s][k % len(eyes_by_scene[s])]
            views.append(foveal_crop(base, seed + 3000 + 4 * s + k, size=size))
    for s in range(4):
        R = _yaw_pitch(rng.uniform(-math.pi, math.pi), rng.normal(0, 0.1))
        views.append(Camera(R, np.zeros(3), 1000.0, 1000.0, 632.0, 416.0, 1264, 832,
                            scene=s))
    return scenes, views
