"""Independent fp64 NumPy brute force of the 3DGS forward pass, for tiny scenes.

A second, deliberately different restatement used only to pin the C oracle:

* rotations come from ``scipy.spatial.transform.Rotation`` (a library routine), not
  from a hand-written quaternion formula;
* the SH colour uses ``scipy.special.sph_harm_y`` turned into real harmonics with the
  sign convention of the 3DGS renderer (``SH_SIGN`` below);
* the pinhole Jacobian is written directly from d(u, v)/d(t) and checked separately
  against finite differences;
* every pixel gathers its own candidate list (all visible Gaussians whose tile
  rectangle contains the pixel's tile), sorts it by fp64 depth and composites in fp64.

Only the readings of the constants (near 0.2, low-pass 0.3, eigenvalue floor 0.1,
alpha clamp 0.99, skip 1/255, stop 1e-4, +0.5 colour offset, Jacobian clamp 1.3) are
shared with the oracle, because they are the definition being tested.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

# Sign of the 3DGS basis function relative to the real SH built from scipy below,
# coefficient index k = l^2 + l + m.
SH_SIGN = np.array([1, -1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1], dtype=np.float64)


def real_sh(l: int, m: int, d: np.ndarray) -> np.ndarray:
    """Real spherical harmonic of degree l, order m at unit directions d [..., 3]."""
    d = np.asarray(d, dtype=np.float64)
    theta = np.arccos(np.clip(d[..., 2], -1.0, 1.0))      # polar angle from +z
    phi = np.arctan2(d[..., 1], d[..., 0])                # azimuth from +x
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * np.real(y)
    return math.sqrt(2.0) * (-1) ** m * np.imag(y)


def sh_basis64(d: np.ndarray, degree: int) -> np.ndarray:
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            out.append(SH_SIGN[k] * real_sh(l, m, d))
    return np.stack(out, axis=-1)


def project64(scene, cam, tile: int):
    """Per-Gaussian fp64 projection. Returns dict of arrays (invisible -> visible False)."""
    n = scene.n
    W = cam.world_to_cam.astype(np.float64)
    Rc, tc = W[:, :3], W[:, 3]
    mu = scene.means.astype(np.float64)
    t = mu @ Rc.T + tc
    visible = t[:, 2] > cam.znear
    S = np.exp(scene.log_scales.astype(np.float64))
    q = scene.quats.astype(np.float64)
    rot = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    sigma = rot @ (S[:, :, None] ** 2 * np.transpose(rot, (0, 2, 1)))
    tz = np.where(visible, t[:, 2], 1.0)
    limx = 1.3 * (0.5 * cam.width / cam.fx)
    limy = 1.3 * (0.5 * cam.height / cam.fy)
    xc = np.clip(t[:, 0] / tz, -limx, limx) * tz
    yc = np.clip(t[:, 1] / tz, -limy, limy) * tz
    J = np.zeros((n, 2, 3))
    J[:, 0, 0] = cam.fx / tz
    J[:, 0, 2] = -cam.fx * xc / tz ** 2
    J[:, 1, 1] = cam.fy / tz
    J[:, 1, 2] = -cam.fy * yc / tz ** 2
    T = J @ Rc
    cov = T @ sigma @ np.transpose(T, (0, 2, 1))
    cov[:, 0, 0] += 0.3
    cov[:, 1, 1] += 0.3
    a, b, c = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    det = a * c - b * b
    visible &= det > 0
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - det))
    radius = np.ceil(3.0 * np.sqrt(lam))
    u = cam.fx * t[:, 0] / tz + cam.cx
    v = cam.fy * t[:, 1] / tz + cam.cy
    tx_n = (cam.width + tile - 1) // tile
    ty_n = (cam.height + tile - 1) // tile
    x0 = np.clip(np.floor((u - radius) / tile), 0, tx_n)
    x1 = np.clip(np.floor((u + radius) / tile) + 1, 0, tx_n)
    y0 = np.clip(np.floor((v - radius) / tile), 0, ty_n)
    y1 = np.clip(np.floor((v + radius) / tile) + 1, 0, ty_n)
    visible &= (x0 < x1) & (y0 < y1)
    opacity = 1.0 / (1.0 + np.exp(-scene.opacity_logits.astype(np.float64)))
    centre = cam.center()
    d = mu - centre
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    K = (scene.sh_degree + 1) ** 2
    basis = sh_basis64(d, scene.sh_degree)                    # [n, K]
    rgb = np.maximum(0.0, np.einsum("nk,nkc->nc", basis, scene.sh.astype(np.float64)[:, :K]) + 0.5)
    det_s = np.where(det > 0, det, 1.0)
    conic = np.stack([c / det_s, -b / det_s, a / det_s], axis=1)
    return dict(visible=visible, u=u, v=v, conic=conic, opacity=opacity, rgb=rgb, depth=t[:, 2],
                radius=radius, rect=np.stack([x0, y0, x1, y1], axis=1).astype(np.int64),
                cov=np.stack([a, b, c], axis=1))


def render64(scene, cam, tile: int):
    """fp64 image [H, W, 3] and T_final [H, W], each pixel over its own sorted list."""
    p = project64(scene, cam, tile)
    H, W = cam.height, cam.width
    img = np.zeros((H, W, 3))
    tfin = np.ones((H, W))
    n_eval = np.zeros((H, W), np.int64)    # list entries walked (the stopping one included)
    n_blend = np.zeros((H, W), np.int64)   # Gaussians blended
    vis = np.nonzero(p["visible"])[0]
    for y in range(H):
        for x in range(W):
            tx, ty = x // tile, y // tile
            r = p["rect"][vis]
            sel = vis[(r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])]
            order = sel[np.lexsort((sel, p["depth"][sel]))]
            T, C = 1.0, np.zeros(3)
            for g in order:
                n_eval[y, x] += 1
                dx, dy = p["u"][g] - x, p["v"][g] - y
                ca, cb, cc = p["conic"][g]
                power = -0.5 * (ca * dx * dx + cc * dy * dy) - cb * dx * dy
                if power > 0:
                    continue
                alpha = min(0.99, p["opacity"][g] * math.exp(power))
                if alpha < 1.0 / 255.0:
                    continue
                tt = T * (1.0 - alpha)
                if tt < 1e-4:
                    break
                C += p["rgb"][g] * alpha * T
                T = tt
                n_blend[y, x] += 1
            img[y, x] = C
            tfin[y, x] = T
    p["n_eval"], p["n_blend"] = n_eval, n_blend
    return img, tfin, p
