"""fp64 reference forward and gradient of the 3DGS rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the CPU legs of ``bench.py`` use this module.  It restates the forward
pass of 3D Gaussian Splatting (Sec. 2.3: projection, sorting, rasterization) as plain
PyTorch CPU operations in float64, and takes the gradient of a weighted sum of the output
colours with autograd.  That gradient is, by definition, what a backward rasterizer must
return for the loss ``L = sum(dl_drgb * C)``.

Steps, in the order of the forward pass (the constants are the 3DGS conventions the C
oracle uses, see ``a3fr_oracle.c``):

1. activation: ``s = exp(log_scales)``; ``q / |q|`` (w, x, y, z); ``o = sigmoid(logit)``;
   ``Sigma = R(q) diag(s^2) R(q)^T``;
2. camera: ``t = R_c mu + t_c``; ``u = f_x t_x / t_z + c_x`` (same for v);
3. EWA: ``J = [[f_x/t_z, 0, -f_x x'/t_z^2], [0, f_y/t_z, -f_y y'/t_z^2]]`` with
   ``x' = clamp(t_x/t_z, +-1.3 tan(fov_x/2)) t_z`` (same for y'); ``Sigma' = J R_c Sigma
   R_c^T J^T + 0.3 I``; conic = inverse of Sigma';
4. colour: real SH of degree <= 3 (3DGS sign convention) along the unit direction from the
   eye centre ``-R_c^T t_c`` to the mean, ``max(0, . + 0.5)``;
5. per pixel, over ONE list of the visible Gaussians in (depth, index) order, skipping
   Gaussians whose tile rectangle misses the pixel's tile: ``power = -0.5 (a dx^2 + c dy^2)
   - b dx dy`` (skip if > 0), ``alpha = min(0.99, o exp(power))`` (skip if < 1/255), stop
   before the Gaussian that would take T below 1e-4, ``C = sum rgb alpha T``.

Visibility, tile rectangles and the depth order are discrete decisions of the fp32 pass;
they are taken from the C oracle (``oracle.preprocess``) so that the set of Gaussians each
pixel may see is the one the renderer uses.  The alpha / stop decisions are re-made here in
float64; ``margins`` reports, per pixel, how close the nearest such decision came to its
threshold, so tests can exclude pixels where fp32 and fp64 may decide differently.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle

F64 = torch.float64


def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real SH basis [N, (degree+1)^2] at unit directions d [N,3] (3DGS order and signs).

    The normalisations are the closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times
    sqrt 2 for m != 0), multiplied into each polynomial."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    out = [torch.full_like(x, 0.5 * math.sqrt(1.0 / pi))]
    if degree >= 1:
        c1 = math.sqrt(3.0 / (4.0 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if degree >= 2:
        xx, yy, zz = x * x, y * y, z * z
        c2a, c2b, c2c = 0.5 * math.sqrt(15.0 / pi), 0.25 * math.sqrt(5.0 / pi), 0.25 * math.sqrt(15.0 / pi)
        out += [c2a * x * y, -c2a * y * z, c2b * (2 * zz - xx - yy), -c2a * x * z, c2c * (xx - yy)]
    if degree >= 3:
        c3a = 0.25 * math.sqrt(35.0 / (2.0 * pi))
        c3b = 0.5 * math.sqrt(105.0 / pi)
        c3c = 0.25 * math.sqrt(21.0 / (2.0 * pi))
        c3d = 0.25 * math.sqrt(7.0 / pi)
        c3e = 0.25 * math.sqrt(105.0 / pi)
        out += [-c3a * y * (3 * xx - yy), c3b * x * y * z, -c3c * y * (4 * zz - xx - yy),
                c3d * z * (2 * zz - 3 * xx - 3 * yy), -c3c * x * (4 * zz - xx - yy),
                c3e * z * (xx - yy), -c3a * x * (xx - 3 * yy)]
    return torch.stack(out, dim=1)


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """R [N,3,3] of unit quaternions q [N,4] = (w, x, y, z)."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], dim=1)


def project(params: dict, cam, degree: int) -> dict:
    """Steps 1-4 for every Gaussian (float64 tensors, differentiable)."""
    W = torch.as_tensor(np.asarray(cam.world_to_cam, dtype=np.float64).reshape(3, 4), dtype=F64)
    Rc, tc = W[:, :3], W[:, 3]
    mu = params["means"]
    s = torch.exp(params["log_scales"])
    q = params["quats"]
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    R = quat_to_rot(q)
    Sigma = R @ torch.diag_embed(s * s) @ R.transpose(1, 2)
    opacity = torch.sigmoid(params["opacity_logits"])
    t = mu @ Rc.T + tc
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    limx = 1.3 * (0.5 * cam.width / fx)
    limy = 1.3 * (0.5 * cam.height / fy)
    xc = torch.clamp(tx / tz, -limx, limx) * tz
    yc = torch.clamp(ty / tz, -limy, limy) * tz
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * xc / (tz * tz)], -1),
                     torch.stack([zero, fy / tz, -fy * yc / (tz * tz)], -1)], dim=1)
    T = J @ Rc
    cov = T @ Sigma @ T.transpose(1, 2)
    a = cov[:, 0, 0] + 0.3
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + 0.3
    det = a * c - b * b
    u = fx * (tx / tz) + cx
    v = fy * (ty / tz) + cy
    centre = -(Rc.T @ tc)
    d = mu - centre
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    Y = sh_basis(d, degree)
    rgb = torch.clamp(torch.einsum("nk,nkc->nc", Y, params["sh"]) + 0.5, min=0.0)
    return {"u": u, "v": v, "ca": c / det, "cb": -b / det, "cc": a / det, "opacity": opacity,
            "rgb": rgb, "depth": tz}


class Visibility:
    """Discrete decisions of the fp32 pass: visible Gaussians, tile rectangles, depth order."""

    def __init__(self, scene, cam, tile: int):
        rec, rect, _ = oracle.preprocess(scene, cam, tile)
        vis = np.nonzero(rec[:, 11] > 0)[0]
        depth_bits = rec[vis, 9].view(np.uint32)
        self.order = vis[np.lexsort((vis, depth_bits))]   # (depth bits, index)
        self.rect = rect
        self.tile = tile


def composite(proj: dict, vis: Visibility, pixels: np.ndarray, chunk: int = 4096,
              keep_mask: bool = False):
    """Step 5 for the pixels [P,2] (x, y).  Returns (C [P,3] differentiable, info dict);
    with keep_mask, info["contrib"] is the [P, G] mask of contributing Gaussians."""
    # only Gaussians whose rectangle meets the bounding box of the pixels' tiles can reach
    # them (the others fail the membership test for every pixel): drop them up front
    order = vis.order
    tx0, tx1 = pixels[:, 0].min() // vis.tile, pixels[:, 0].max() // vis.tile
    ty0, ty1 = pixels[:, 1].min() // vis.tile, pixels[:, 1].max() // vis.tile
    r = vis.rect[order]
    order = order[(r[:, 0] <= tx1) & (r[:, 2] > tx0) & (r[:, 1] <= ty1) & (r[:, 3] > ty0)]
    g = torch.as_tensor(order, dtype=torch.long)
    u, v = proj["u"][g], proj["v"][g]
    ca, cb, cc = proj["ca"][g], proj["cb"][g], proj["cc"][g]
    op, rgb = proj["opacity"][g], proj["rgb"][g]
    rect = vis.rect[order]
    outs, t_final, n_contrib, margins, masks = [], [], [], [], []
    for p0 in range(0, len(pixels), chunk):
        pix = pixels[p0:p0 + chunk]
        px = torch.as_tensor(pix[:, 0], dtype=F64)[:, None]
        py = torch.as_tensor(pix[:, 1], dtype=F64)[:, None]
        tx = pix[:, 0:1] // vis.tile
        ty = pix[:, 1:2] // vis.tile
        member = torch.as_tensor((rect[None, :, 0] <= tx) & (tx < rect[None, :, 2]) &
                                 (rect[None, :, 1] <= ty) & (ty < rect[None, :, 3]))
        dx = u[None, :] - px
        dy = v[None, :] - py
        power = -0.5 * (ca[None, :] * dx * dx + cc[None, :] * dy * dy) - cb[None, :] * dx * dy
        alpha = torch.clamp(op[None, :] * torch.exp(power), max=0.99)
        with torch.no_grad():
            considered = member & (power <= 0)
            valid = considered & (alpha >= 1.0 / 255.0)
            a_eff = torch.where(valid, alpha, torch.zeros_like(alpha))
            t_incl = torch.cumprod(1.0 - a_eff, dim=1)
            stop = valid & (t_incl < 1e-4)
            G = alpha.shape[1]
            idx = torch.arange(G)[None, :]
            first = torch.where(stop.any(1), stop.int().argmax(1), torch.full((len(pix),), G))
            keep = idx < first[:, None]
            contrib = valid & keep
            # closeness of every decision taken up to the stop to its threshold
            reached = idx <= first[:, None]
            m_alpha = torch.where(considered & reached, (alpha * 255.0 - 1.0).abs(),
                                  torch.full_like(alpha, math.inf))
            m_stop = torch.where(valid & reached, (t_incl / 1e-4 - 1.0).abs(),
                                 torch.full_like(alpha, math.inf))
            margin = torch.minimum(m_alpha.min(1).values, m_stop.min(1).values)
        a_c = torch.where(contrib, alpha, torch.zeros_like(alpha))
        one_m = 1.0 - a_c
        t_excl = torch.cat([torch.ones_like(one_m[:, :1]), torch.cumprod(one_m[:, :-1], dim=1)], 1)
        w = a_c * t_excl
        outs.append(w @ rgb)
        with torch.no_grad():
            t_final.append(torch.prod(one_m, dim=1))
            n_contrib.append(torch.where(contrib, idx + 1, torch.zeros_like(idx)).max(1).values)
            margins.append(margin)
            if keep_mask:
                masks.append(contrib.numpy())
    info = {"t_final": torch.cat(t_final).numpy(), "margin": torch.cat(margins).numpy(),
            "n_contrib_global": torch.cat(n_contrib).numpy()}
    if keep_mask:
        info["contrib"] = np.concatenate(masks)
    return torch.cat(outs), info


def params_f64(scene) -> dict:
    return {k: torch.tensor(np.asarray(getattr(scene, k), dtype=np.float64), dtype=F64)
            for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}


def all_pixels(cam) -> np.ndarray:
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    return np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int64)


def loss(params: dict, scene, cam, tile: int, dl_drgb: np.ndarray, vis: Visibility | None = None,
         pixels: np.ndarray | None = None, keep_mask: bool = False):
    """L = sum(dl_drgb * C) over the pixels (all of them by default); returns (L, C, info)."""
    vis = vis or Visibility(scene, cam, tile)
    pixels = all_pixels(cam) if pixels is None else pixels
    proj = project(params, cam, scene.sh_degree)
    C, info = composite(proj, vis, pixels, keep_mask=keep_mask)
    w = torch.as_tensor(np.asarray(dl_drgb, dtype=np.float64).reshape(-1, 3))
    return (w * C).sum(), C, info


def gradient(scene, cam, tile: int, dl_drgb: np.ndarray, pixels: np.ndarray | None = None) -> dict:
    """dL/d(means, log_scales, quats, opacity_logits, sh) in float64 (NumPy) + 'info'."""
    params = params_f64(scene)
    for t in params.values():
        t.requires_grad_(True)
    L, C, info = loss(params, scene, cam, tile, dl_drgb, pixels=pixels)
    L.backward()
    out = {k: t.grad.numpy().copy() for k, t in params.items()}
    out["info"] = info
    out["rgb"] = C.detach().numpy()
    return out


def finite_difference(scene, cam, tile: int, dl_drgb: np.ndarray, name: str, index, h: float = 1e-4,
                      vis: Visibility | None = None):
    """Central difference (L(p + h) - L(p - h)) / 2h of one parameter element, float64, with
    the discrete decisions of the fp32 pass held fixed; also whether any alpha / stop decision
    of the float64 pass differs between the two sides (then the difference is not a
    derivative)."""
    vis = vis or Visibility(scene, cam, tile)
    vals = []
    masks = []
    for sgn in (1.0, -1.0):
        params = params_f64(scene)
        with torch.no_grad():
            params[name][index] += sgn * h
            L, _, info = loss(params, scene, cam, tile, dl_drgb, vis=vis, keep_mask=True)
        vals.append(float(L))
        masks.append(info["contrib"])
    flipped = not np.array_equal(masks[0], masks[1])
    return (vals[0] - vals[1]) / (2.0 * h), flipped
