"""CPU oracle of the foveated 3DGS forward rasterizer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never calls it and has no CPU fallback.

The arithmetic lives in ``a3fr_oracle.c`` (plain C, fp32 with a fixed operation
order, built with ``-ffp-contract=off``); this module compiles it with gcc and
marshals NumPy arrays through ctypes.  Every function cites the passage it follows
in the C file's comments.

Parity status of each part (pins are the ``-m "not gpu"`` tests in ``tests/``):
  * projection / EWA covariance / conic / radius   -- pinned (closed forms, FD Jacobian,
    scipy rotation, fp64 brute force)
  * SH colour                                       -- pinned (scipy real SH)
  * keys, sort, tile ranges                          -- pinned (brute-force membership,
    Python sorted())
  * compositing                                      -- pinned (single-Gaussian closed
    form, weight-sum and white-colour invariants, input-order invariance, fp64 brute force)
  * threshold margin and the flipped-decision colour -- pinned (a Gaussian at alpha = 1/255
    exactly, a stack whose transmittance lands on 1e-4, closed forms of both margins)
  * foveation level map, live mask, fill             -- pinned (brute-force geometry,
    closed-form disc count)
  * count-based tile levels                          -- pinned (hand-counted cases, ties,
    the k = 0 and k = tiles limits)
  * absolute agreement with the paper's own renderer and its second-layer angle
                                                     -- parity unpinned (the paper prints
    no rendered values and names no second-layer angle)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "a3fr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liba3fr_oracle.so")
_lib = None

REC = 12  # floats per record: u v ca cb cc opacity r g b depth radius visible


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12)]


class Fovea(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("theta_deg", ctypes.c_float * 3),
                ("dtheta_deg", ctypes.c_float), ("level", ctypes.c_int32 * 4)]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.or_exp.argtypes = [ctypes.c_float]
        L.or_exp.restype = ctypes.c_float
        L.or_sh_basis.argtypes = [vp, i32, vp]
        L.or_preprocess.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp]
        L.or_sorted_keys.argtypes = [i32, vp, vp, i32, vp, vp]
        L.or_sorted_keys.restype = i64
        L.or_tile_ranges.argtypes = [i64, vp, i32, vp]
        L.or_layer_radii2.argtypes = [vp, vp, vp]
        L.or_level_map.argtypes = [vp, i32, vp, vp, vp]
        L.or_render.argtypes = [i32, vp, vp, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_render_eye.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, i32,
                                    vp, vp, vp, vp, vp, vp]
        L.or_num_threads.restype = i32
        _lib = L
    return _lib


def camera(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy, c.znear = cam.fx, cam.fy, cam.cx, cam.cy, cam.znear
    w = np.ascontiguousarray(cam.world_to_cam, dtype=np.float32).reshape(12)
    for i in range(12):
        c.world_to_cam[i] = float(w[i])
    return c


def fovea(theta_deg=(18.0, 36.0), dtheta_deg=0.0, levels=(4, 2, 1)) -> Fovea:
    f = Fovea()
    f.n_layers = len(levels)
    for k, t in enumerate(theta_deg):
        f.theta_deg[k] = t
    f.dtheta_deg = dtheta_deg
    for k, lv in enumerate(levels):
        f.level[k] = lv
    return f


def tiles(extent: int, tile: int) -> int:
    return (extent + tile - 1) // tile


def exp32(x: float) -> float:
    return float(np.float32(lib().or_exp(float(x))))


def sh_basis(d, degree: int = 3) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float32)
    out = np.zeros(16, dtype=np.float32)
    lib().or_sh_basis(_p(d), degree, _p(out))
    return out[: (degree + 1) ** 2]


def _scene_arrays(scene):
    return [np.ascontiguousarray(a, dtype=np.float32) for a in
            (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]


def preprocess(scene, cam, tile: int):
    """Per-Gaussian records [N,12], rects [N,4] (x0,y0,x1,y1), tiles touched [N]."""
    n = scene.n
    arrs = _scene_arrays(scene)
    rec = np.zeros((n, REC), dtype=np.float32)
    rect = np.zeros((n, 4), dtype=np.int32)
    touched = np.zeros(n, dtype=np.uint32)
    c = camera(cam)
    lib().or_preprocess(n, scene.sh_degree, *[_p(a) for a in arrs], ctypes.byref(c), tile,
                        _p(rec), _p(rect), _p(touched))
    return rec, rect, touched


def sorted_keys(rec, rect, tiles_x: int):
    n = rec.shape[0]
    total = lib().or_sorted_keys(n, _p(rec), _p(rect), tiles_x, None, None)
    keys = np.zeros(max(total, 1), dtype=np.uint64)
    vals = np.zeros(max(total, 1), dtype=np.uint32)
    lib().or_sorted_keys(n, _p(rec), _p(rect), tiles_x, _p(keys), _p(vals))
    return keys[:total], vals[:total]


def tile_ranges(keys, n_tiles: int):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    ranges = np.zeros((n_tiles, 2), dtype=np.uint32)
    lib().or_tile_ranges(len(keys), _p(keys), n_tiles, _p(ranges))
    return ranges


def layer_radii2(cam, fv: Fovea):
    out = np.zeros(3, dtype=np.float32)
    c = camera(cam)
    lib().or_layer_radii2(ctypes.byref(c), ctypes.byref(fv), _p(out))
    return out


def level_map(cam, tile: int, fv: Fovea, gaze):
    c = camera(cam)
    g = np.ascontiguousarray(gaze, dtype=np.float32)
    out = np.zeros(tiles(cam.width, tile) * tiles(cam.height, tile), dtype=np.uint8)
    lib().or_level_map(ctypes.byref(c), tile, ctypes.byref(fv), _p(g), _p(out))
    return out


def count_levels(level, ranges, count_frac: float):
    """Tile levels by Gaussian count (Sec. 3.6 and 4.6: tiles ordered by how many Gaussians
    they hold, the resolution of the heaviest lowered), the reading taken: with k =
    floor(count_frac * tiles) computed in fp32, tau is the k-th largest instance count of
    the eye's tiles; a tile whose level is 2 or 3 and whose count c satisfies c > 0 and
    c >= tau renders one level lower.  Foveal tiles (level 4) and level 1 keep their level.
    level [tiles] uint8 (one eye), ranges [tiles, 2] uint32; returns a new level array."""
    level = np.array(level, dtype=np.uint8)
    counts = ranges[:, 1].astype(np.int64) - ranges[:, 0].astype(np.int64)
    k = int(np.floor(np.float32(count_frac) * np.float32(len(counts))))
    if k < 1:
        return level
    tau = np.sort(counts)[::-1][min(k, len(counts)) - 1]
    heavy = (counts > 0) & (counts >= tau) & ((level == 2) | (level == 3))
    level[heavy] -= 1
    return level


class Image:
    """Oracle output for a set of pixels (full image or a pixel list)."""

    def __init__(self, count):
        self.rgb = np.zeros((count, 3), dtype=np.float32)
        self.t_final = np.zeros(count, dtype=np.float32)
        self.n_contrib = np.zeros(count, dtype=np.int32)
        self.n_eval = np.zeros(count, dtype=np.int32)    # Gaussians whose rectangle holds the pixel, walked
        self.n_blend = np.zeros(count, dtype=np.int32)   # Gaussians blended into the pixel
        self.margin = np.zeros(count, dtype=np.float32)
        self.rendered = np.zeros(count, dtype=np.uint8)
        self.depth = np.zeros(count, dtype=np.float32)   # expected depth sum(alpha T z)
        # the colour with the pixel's nearest threshold decision (alpha >= 1/255 skip or
        # T >= 1e-4 stop) taken the other way, for pixels whose margin is below 1e-3
        # (equal to rgb elsewhere): what a renderer whose exp differs by an ulp may produce
        self.rgb_alt = np.zeros((count, 3), dtype=np.float32)


def render(rec, rect, cam, tile: int, level=None, pixels=None) -> Image:
    """Composite pixels over the global depth-sorted list (see a3fr_oracle.c)."""
    c = camera(cam)
    n = rec.shape[0]
    if pixels is None:
        count, pix = cam.width * cam.height, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        count = pix.shape[0]
    img = Image(count)
    lv = None if level is None else np.ascontiguousarray(level, dtype=np.uint8)
    lib().or_render(n, _p(np.ascontiguousarray(rec)), _p(np.ascontiguousarray(rect)),
                    ctypes.byref(c), tile, _p(lv), _p(pix), count if pix is not None else 0,
                    _p(img.rgb), _p(img.t_final), _p(img.n_contrib), _p(img.n_eval),
                    _p(img.margin), _p(img.rendered), _p(img.depth), _p(img.rgb_alt),
                    _p(img.n_blend))
    return img


def render_eye(scene, cam, tile: int, fv: Fovea | None, gaze=None, pixels=None) -> Image:
    """Preprocess + (foveated when ``fv`` is given) render of one eye in one call."""
    c = camera(cam)
    arrs = _scene_arrays(scene)
    if pixels is None:
        count, pix = cam.width * cam.height, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        count = pix.shape[0]
    img = Image(count)
    g = None if gaze is None else np.ascontiguousarray(gaze, dtype=np.float32)
    lib().or_render_eye(scene.n, scene.sh_degree, *[_p(a) for a in arrs], ctypes.byref(c), tile,
                        ctypes.byref(fv) if fv is not None else None, _p(g), _p(pix),
                        count if pix is not None else 0, _p(img.rgb), _p(img.t_final),
                        _p(img.n_contrib), _p(img.n_eval), _p(img.margin), _p(img.rendered))
    img.rgb_alt[:] = img.rgb
    return img


def fill_interpolate(img: np.ndarray, rendered: np.ndarray) -> np.ndarray:
    """Interpolating fill of a foveated image (Sec. 3.4: skipped pixels "inherit or
    interpolate"), the reading taken: a skipped pixel becomes the mean of its rendered
    4-neighbours (summed in the order up, down, left, right), else of its rendered diagonal
    neighbours (up-left, up-right, down-left, down-right), else keeps the inherited top-left
    value.  fp32 throughout.  img [H, W, 3] float32, rendered [H, W] bool."""
    H, W, _ = img.shape
    out = img.astype(np.float32).copy()
    for y in range(H):
        for x in range(W):
            if rendered[y, x]:
                continue
            for nbrs in (((0, -1), (0, 1), (-1, 0), (1, 0)), ((-1, -1), (1, -1), (-1, 1), (1, 1))):
                acc = np.zeros(3, dtype=np.float32)
                cnt = 0
                for dx, dy in nbrs:
                    xx, yy = x + dx, y + dy
                    if 0 <= xx < W and 0 <= yy < H and rendered[yy, xx]:
                        acc = (acc + img[yy, xx]).astype(np.float32)
                        cnt += 1
                if cnt:
                    out[y, x] = (acc / np.float32(cnt)).astype(np.float32)
                    break
    return out


def num_threads() -> int:
    return int(lib().or_num_threads())
