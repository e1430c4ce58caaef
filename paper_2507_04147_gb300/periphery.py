"""Learned periphery: the tensor-core CNNs that fill the pixels a foveated render skipped --
a residual network of ten 3x3 convolutions (``RESIDUAL``) and a compact one, a 3x3 convolution
and two per-block layers, whose fill is a single fused kernel (``COMPACT``).

The networks and their kernels live in the CUDA library (``a3fr_cnn_*``, see ``include/a3fr.h``);
this module marshals arguments, initialises parameters, cuts training crops out of the
rasterizer's own renders and computes the image metrics the comparison is reported in.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib, _ptr, _stream_ptr, _torch

RESIDUAL, COMPACT = 0, 1   # A3FR_CNN_RESIDUAL, A3FR_CNN_COMPACT
# (in, out, kernel size) of each layer: ten 3x3 convs; or a 3x3 conv and two per-block layers
ARCH_LAYERS = {RESIDUAL: [(16, 32, 3)] + [(32, 32, 3)] * 8 + [(32, 16, 3)],
               COMPACT: [(16, 32, 3), (32, 32, 1), (32, 16, 1)]}
LAYERS = [(i, o) for i, o, _ in ARCH_LAYERS[RESIDUAL]]


def init_params(seed: int = 0, arch: int = RESIDUAL) -> np.ndarray:
    """He-initialised parameters (flat fp32): input channels 4..15 of layer 0 are zero and the
    last layer is zero, so the initial prediction is its bilinear base exactly (the
    interpolating fill of the periphery) and training only refines it."""
    rng = np.random.default_rng(seed)
    layers = ARCH_LAYERS[arch]
    ws, bs = [], []
    for li, (cin, cout, k) in enumerate(layers):
        fan_in = (4 if li == 0 else cin) * k * k
        w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=(cout, cin, k, k)).astype(np.float32)
        if li == 0:
            w[:, 4:] = 0.0
        if li == len(layers) - 1:
            w[:] = 0.0
        ws.append(w)
        bs.append(np.zeros(cout, dtype=np.float32))
    return pack(ws, bs)


def pack(ws, bs) -> np.ndarray:
    return np.concatenate([np.asarray(w, np.float32).ravel() for w in ws] +
                          [np.asarray(b, np.float32).ravel() for b in bs])


def unpack(flat: np.ndarray, arch: int = RESIDUAL):
    """(weights [out, in, k, k], biases) of a flat parameter vector."""
    ws, bs, o = [], [], 0
    layers = ARCH_LAYERS[arch]
    for cin, cout, k in layers:
        n = cin * cout * k * k
        ws.append(flat[o:o + n].reshape(cout, cin, k, k))
        o += n
    for _, cout, _ in layers:
        bs.append(flat[o:o + cout])
        o += cout
    return ws, bs


class Periphery:
    """A network object of the library (parameters, Adam state and workspaces on the GPU)."""

    def __init__(self, params: np.ndarray | None = None, seed: int = 0, arch: int = RESIDUAL):
        L = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(L.a3fr_cnn_create_arch(ctypes.byref(h), int(arch)), "a3fr_cnn_create_arch")
        self.handle = h.value
        self.arch = int(arch)
        self.n_params = int(L.a3fr_cnn_arch_param_count(self.arch))
        self.set_params(init_params(seed, self.arch) if params is None else params)

    def set_params(self, flat: np.ndarray) -> None:
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {flat.size}")
        _lib.check(_lib.load().a3fr_cnn_set_params(self.handle, flat.ctypes.data, flat.size),
                   "a3fr_cnn_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _lib.check(_lib.load().a3fr_cnn_get_params(self.handle, out.ctypes.data, out.size),
                   "a3fr_cnn_get_params")
        return out

    def forward(self, img, depth, stream=None):
        """Per-block corrections [b, (h+1)//2, (w+1)//2, 16] of images [b, h, w, 3]."""
        torch = _torch()
        b, h, w = img.shape[:3]
        r = torch.empty((b, (h + 1) // 2, (w + 1) // 2, 16), dtype=torch.float32, device=img.device)
        _lib.check(_lib.load().a3fr_cnn_forward(self.handle, _ptr(img), _ptr(depth), b, h, w, _ptr(r),
                                                _stream_ptr(stream)), "a3fr_cnn_forward")
        return r

    def grads(self, img, depth, target, stream=None):
        """(flat fp32 gradient of the mean squared error, loss); synchronous."""
        b, h, w = img.shape[:3]
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _lib.check(_lib.load().a3fr_cnn_grads(self.handle, _ptr(img), _ptr(depth), _ptr(target), b, h, w,
                                              g.ctypes.data, ctypes.byref(loss), _stream_ptr(stream)),
                   "a3fr_cnn_grads")
        return g, float(loss.value)

    def train_step(self, img, depth, target, lr: float, sync: bool = False, stream=None):
        b, h, w = img.shape[:3]
        loss = ctypes.c_float()
        _lib.check(_lib.load().a3fr_cnn_train_step(self.handle, _ptr(img), _ptr(depth), _ptr(target), b, h, w,
                                                   float(lr), ctypes.byref(loss) if sync else None,
                                                   _stream_ptr(stream)), "a3fr_cnn_train_step")
        return float(loss.value) if sync else None

    def fill(self, scene, out, stream=None) -> None:
        """Learned fill of the scene's last foveated render (keep_aux on) in ``out``."""
        handle = scene.handle if hasattr(scene, "handle") else scene
        _lib.check(_lib.load().a3fr_cnn_fill(self.handle, handle, _ptr(out), _stream_ptr(stream)),
                   "a3fr_cnn_fill")

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().a3fr_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------ evaluation
def psnr(a, b, mask=None) -> float:
    """PSNR in dB of images clamped to [0, 1] (MAX = 1), mean over channels and pixels."""
    torch = _torch()
    d = (a.clamp(0, 1) - b.clamp(0, 1)) ** 2
    if mask is not None:
        d = d[mask]
    mse = float(d.mean())
    return math.inf if mse == 0.0 else 10.0 * math.log10(1.0 / mse)


def ssim(a, b) -> float:
    """SSIM (Wang et al. 2004: Gaussian window 11, sigma 1.5, K1 0.01, K2 0.03, L 1) of
    images [n, h, w, 3] clamped to [0, 1], mean over channels and positions."""
    torch = _torch()
    F = torch.nn.functional
    x = a.clamp(0, 1).permute(0, 3, 1, 2).reshape(-1, 1, a.shape[1], a.shape[2]).double()
    y = b.clamp(0, 1).permute(0, 3, 1, 2).reshape(-1, 1, b.shape[1], b.shape[2]).double()
    g = torch.exp(-((torch.arange(11, dtype=torch.float64, device=x.device) - 5.0) ** 2) / (2 * 1.5 ** 2))
    g = g / g.sum()
    win = (g[:, None] * g[None, :])[None, None]
    mu_x, mu_y = F.conv2d(x, win), F.conv2d(y, win)
    sxx = F.conv2d(x * x, win) - mu_x ** 2
    syy = F.conv2d(y * y, win) - mu_y ** 2
    sxy = F.conv2d(x * y, win) - mu_x * mu_y
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mu_x * mu_y + c1) * (2 * sxy + c2)) / ((mu_x ** 2 + mu_y ** 2 + c1) * (sxx + syy + c2))
    return float(s.mean())


def render_crops(scene, cams, crop: int, per_view: int, rng, stream=None):
    """Full-resolution renders of ``scene`` (a Scene with keep_aux on) from each camera, cut
    into ``per_view`` random crop x crop windows (even offsets, so 2x2 blocks stay aligned):
    (images [n, crop, crop, 3], depths [n, crop, crop]) CUDA tensors."""
    torch = _torch()
    from . import BUF_DEPTH
    imgs, deps = [], []
    for cam in cams:
        scene.set_camera(0, cam)
        img = scene.render_full(stream=stream)[0]
        dep = scene.buffer(BUF_DEPTH, torch.float32, stream=stream).reshape(cam.height, cam.width)
        for _ in range(per_view):
            y = int(rng.integers(0, (cam.height - crop) // 2 + 1)) * 2
            x = int(rng.integers(0, (cam.width - crop) // 2 + 1)) * 2
            imgs.append(img[y:y + crop, x:x + crop].clone())
            deps.append(dep[y:y + crop, x:x + crop].clone())
    return torch.stack(imgs), torch.stack(deps)
