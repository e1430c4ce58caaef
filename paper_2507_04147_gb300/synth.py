"""Seeded synthetic inputs: Gaussian scenes, stereo cameras and gaze trajectories.

This module only draws random numbers and lays out arrays.  It holds none of the
rasterizer's arithmetic (no projection, no colour evaluation, no compositing), so
both the CUDA path and the CPU oracle can take their inputs from it.

Scene recipes (all fp32 structure-of-arrays, NumPy PCG64):

* ``uniform`` -- means ``(ux, uy, 4 + 2 uz)`` with ``u ~ U[-1, 1]^3`` (a cube of
  side 2 centred at depth 4, i.e. depth 2..6 in front of a camera at the origin
  looking down +z), log-scales ``N(-4, 0.5)`` per axis, random unit quaternions
  (normalised 4-D normals, stored ``w, x, y, z``), opacity logits ``N(0, 1.5)``.
  Colour: the view-independent (degree-0) coefficient is set from a drawn base
  colour ``c ~ U(0, 1)`` so that the degree-0 term evaluates to ``c``; higher
  coefficients are ``N(0, 0.2)``.
* ``clustered`` -- 64 isotropic Gaussian clusters of equal weight, centres
  ``U([-1, 1]^2 x [2, 6])``, cluster standard deviation ``U(0.05, 0.3)``;
  log-scales ``N(-4.5, 0.5)`` (log-normal scales), opacities ``Beta(0.5, 0.5)``
  stored as logits, colours as above.

Cameras follow the pinhole convention of the renderer: ``f = W / (2 tan(fov/2))``,
principal point ``((W - 1) / 2, (H - 1) / 2)``, +z forward, +x right, +y down.
Stereo eyes sit at ``-/+ IPD/2`` along the head's x axis with parallel optical axes.

The gaze trajectory follows the oculomotor description of fixations and saccades
(Sec. 2.1): fixations of U(200, 400) ms, saccades of amplitude U(0, 30) degrees in a
uniform direction, eccentricity clamped to 35 degrees, lasting
``min(100, 20 + 2.5 A)`` ms, with linear interpolation during a saccade.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Real spherical-harmonic normalisation of the l = 0 band, 1 / (2 sqrt(pi)).  Only
# used to encode a drawn base colour as a degree-0 coefficient (input preparation).
_Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


@dataclasses.dataclass
class Scene:
    means: np.ndarray           # [N, 3] f32 world position
    log_scales: np.ndarray      # [N, 3] f32 log of per-axis standard deviation
    quats: np.ndarray           # [N, 4] f32 rotation quaternion (w, x, y, z), not necessarily unit
    opacity_logits: np.ndarray  # [N] f32 logit of the opacity
    sh: np.ndarray              # [N, (deg+1)^2, 3] f32 SH coefficients per colour channel
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    world_to_cam: np.ndarray    # [3, 4] f32 row-major [R | t], x_cam = R x_world + t

    def center(self) -> np.ndarray:
        r = self.world_to_cam[:, :3].astype(np.float64)
        t = self.world_to_cam[:, 3].astype(np.float64)
        return -r.T @ t


def _colour_coeffs(rng: np.random.Generator, n: int, degree: int) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), dtype=np.float64)
    base = rng.uniform(0.0, 1.0, size=(n, 3))
    sh[:, 0, :] = (base - 0.5) / _Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, size=(n, k - 1, 3))
    return sh.astype(np.float32)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_scene(n: int, sh_degree: int = 0, seed: int = 0, log_scale_mean: float = -4.0,
                  log_scale_std: float = 0.5) -> Scene:
    """The uniform-cube scene (means uniform in [-1,1]^3 shifted to depth 2..6)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(-1.0, 1.0, size=(n, 3))
    means = np.stack([u[:, 0], u[:, 1], 4.0 + 2.0 * u[:, 2]], axis=1).astype(np.float32)
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity_logits = rng.normal(0.0, 1.5, size=n).astype(np.float32)
    sh = _colour_coeffs(rng, n, sh_degree)
    return Scene(means, log_scales, quats, opacity_logits, sh, sh_degree)


def clustered_scene(n: int, sh_degree: int = 3, seed: int = 0, n_clusters: int = 64) -> Scene:
    """The clustered scene: equal-weight isotropic Gaussian clusters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = np.stack([rng.uniform(-1, 1, n_clusters), rng.uniform(-1, 1, n_clusters),
                        rng.uniform(2, 6, n_clusters)], axis=1)
    sigmas = rng.uniform(0.05, 0.3, n_clusters)
    which = rng.integers(0, n_clusters, size=n)
    means = (centres[which] + rng.normal(size=(n, 3)) * sigmas[which, None]).astype(np.float32)
    log_scales = rng.normal(-4.5, 0.5, size=(n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    op = np.clip(rng.beta(0.5, 0.5, size=n), 1e-6, 1 - 1e-6)
    opacity_logits = np.log(op / (1.0 - op)).astype(np.float32)
    sh = _colour_coeffs(rng, n, sh_degree)
    return Scene(means, log_scales, quats, opacity_logits, sh, sh_degree)


def yaw_matrix(yaw_deg: float) -> np.ndarray:
    """Head-to-world rotation for a yaw about the +y (down) axis."""
    a = math.radians(yaw_deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def pinhole_camera(width: int, height: int, fov_x_deg: float = 90.0, yaw_deg: float = 0.0,
                   eye_offset_x: float = 0.0, znear: float = 0.2) -> Camera:
    """Camera of a head at the origin with the given yaw, eye shifted along head x."""
    f = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    head = yaw_matrix(yaw_deg)                          # head -> world
    centre = head @ np.array([eye_offset_x, 0.0, 0.0])  # eye centre in world
    r = head.T                                          # world -> camera
    t = -r @ centre
    w2c = np.concatenate([r, t[:, None]], axis=1).astype(np.float32)
    f32 = float(np.float32(f))      # the renderer takes fp32 intrinsics
    return Camera(width, height, f32, f32, (width - 1) / 2.0, (height - 1) / 2.0, znear, w2c)


def stereo_cameras(width: int, height: int, yaw_deg: float = 0.0, ipd: float = 0.063,
                   fov_x_deg: float = 90.0):
    return [pinhole_camera(width, height, fov_x_deg, yaw_deg, -ipd / 2.0),
            pinhole_camera(width, height, fov_x_deg, yaw_deg, +ipd / 2.0)]


def gaze_trajectory(n_frames: int, hz: float = 90.0, seed: int = 1, max_amp_deg: float = 30.0,
                    max_ecc_deg: float = 35.0) -> np.ndarray:
    """Gaze angles (deg, [n_frames, 2] as (horizontal, vertical)) sampled at ``hz``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    # Event list: (start_ms, end_ms, start_angle, end_angle)
    t = 0.0
    pos = np.zeros(2)
    events = []
    horizon = n_frames * 1000.0 / hz + 1000.0
    while t < horizon:
        fix = rng.uniform(200.0, 400.0)
        events.append((t, t + fix, pos.copy(), pos.copy()))
        t += fix
        amp = rng.uniform(0.0, max_amp_deg)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        target = pos + amp * np.array([math.cos(ang), math.sin(ang)])
        ecc = float(np.linalg.norm(target))
        if ecc > max_ecc_deg:
            target *= max_ecc_deg / ecc
        dur = min(100.0, 20.0 + 2.5 * float(np.linalg.norm(target - pos)))
        events.append((t, t + dur, pos.copy(), target.copy()))
        t += dur
        pos = target
    out = np.zeros((n_frames, 2))
    k = 0
    for i in range(n_frames):
        ti = i * 1000.0 / hz
        while events[k][1] <= ti:
            k += 1
        t0, t1, a0, a1 = events[k]
        w = (ti - t0) / (t1 - t0) if t1 > t0 else 0.0
        out[i] = a0 + w * (a1 - a0)
    return out


def gaze_pixels(angles_deg: np.ndarray, cam: Camera) -> np.ndarray:
    """Gaze angles (deg) -> pixel position on the image plane of ``cam``."""
    ax = np.radians(np.asarray(angles_deg, dtype=np.float64))
    gx = cam.cx + cam.fx * np.tan(ax[..., 0])
    gy = cam.cy + cam.fy * np.tan(ax[..., 1])
    return np.stack([gx, gy], axis=-1).astype(np.float32)


# --------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    width: int
    height: int
    n_eyes: int
    tile: int
    frames: int
    yaw_step_deg: float
    theta_deg: tuple
    fixed_gaze_px: tuple | None = None   # overrides the trajectory (single-view workload)

    def cameras(self, frame: int):
        yaw = self.yaw_step_deg * frame
        if self.n_eyes == 1:
            return [pinhole_camera(self.width, self.height, 90.0, yaw, 0.0)]
        return stereo_cameras(self.width, self.height, yaw)

    def gaze(self, frame: int, traj: np.ndarray | None = None) -> np.ndarray:
        cams = self.cameras(frame)
        if self.fixed_gaze_px is not None:
            return np.array([self.fixed_gaze_px] * self.n_eyes, dtype=np.float32)
        return np.stack([gaze_pixels(traj[frame], c) for c in cams]).astype(np.float32)


def small_single_view(seed: int = 0) -> Workload:
    """20k Gaussians, SH degree 0, one 256x256 view, 16x16 tiles, gaze at the centre."""
    return Workload("20k-G SH0 256x256 mono, centre gaze",
                    uniform_scene(20000, 0, seed), 256, 256, 1, 16, 1, 0.0, (18.0, 36.0),
                    fixed_gaze_px=(127.5, 127.5))


def stereo_500k(seed: int = 0, frames: int = 240) -> Workload:
    """500k Gaussians, SH degree 3, stereo 1280x1280, 240 frames of gaze at 90 Hz."""
    return Workload("500k-G SH3 stereo 1280x1280, 240-frame gaze trajectory",
                    uniform_scene(500000, 3, seed), 1280, 1280, 2, 16, frames, 0.05, (18.0, 36.0))


def stereo_3m_clustered(seed: int = 0, frames: int = 240) -> Workload:
    """3M clustered Gaussians, SH degree 3, stereo 2064x2208, 240 frames at 90 Hz."""
    return Workload("3M-G clustered SH3 stereo 2064x2208, 240-frame gaze trajectory",
                    clustered_scene(3000000, 3, seed), 2064, 2208, 2, 16, frames, 0.05, (18.0, 36.0))
