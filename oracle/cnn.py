"""Reference of the learned-periphery network -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the CPU legs of ``bench.py`` use this module.  It defines the network
the tensor-core kernels implement, as plain PyTorch CPU operations in float64 (a library
``conv2d`` is one step), with the BF16 storage of the GPU path emulated at the same points:

* input x0 [B, H2, W2, 16]: the quarter-density layer (the top-left pixel of every 2x2 block,
  Sec. 3.4) as (r, g, b, depth / 8) plus 12 zero channels, stored in BF16;
* conv0: 3x3, 16 -> 32, bias, ReLU -> h (BF16);
* four residual blocks: t = ReLU(conv(h) + b) (BF16); h = h + conv(t) + b (BF16);
* conv9: 3x3, 32 -> 16, bias -> r (FP32); channel c * 4 + 2 dy + dx is the residual of colour
  c at sub-pixel (dx, dy) of the block;
* full-resolution prediction: a base from the quarter-density layer + r (2x pixel shuffle).
  The base of sub-pixel (dx, dy) of block (x2, y2) is the bilinear interpolation of the
  top-left pixels a = tl[y2][x2], right = tl[y2][x2 + 1], down = tl[y2 + 1][x2], diag =
  tl[y2 + 1][x2 + 1] (an index past the last block repeats the last block): a at (0, 0),
  (a + right) / 2 at (1, 0), (a + down) / 2 at (0, 1), (((a + right) + down) + diag) / 4 at
  (1, 1) -- where only top-left pixels are rendered this is the interpolating fill of
  Sec. 3.4 ("inherit or interpolate"), so the network learns a correction to it.

The compact network (``forward_compact``) keeps conv0 and replaces the rest by two per-block
layers: t = ReLU(W1 h + b1) (1x1, 32 -> 32, BF16), r = W2 t + b2 (1x1, 32 -> 16, FP32), the
same channel meaning for r -- a prediction from the 3x3-block neighbourhood of each block.

Convolutions use zero padding of one pixel; weights are [out, in, 3, 3] (1x1 layers:
[out, in, 1, 1]) and rounded to BF16.
Gradients are float64 autograd of the same operations with the roundings passed straight
through (the GPU rounds its gradient tensors to BF16 as well, so the two agree to BF16
precision, not bit for bit).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = 32            # hidden channels
IN_CH = 16         # input channels (4 used)
OUT_CH = 16        # output channels (12 used)
N_BLOCKS = 4
N_CONV = 2 + 2 * N_BLOCKS
DEPTH_SCALE = 1.0 / 8.0
LAYERS = [(IN_CH, CH)] + [(CH, CH)] * (2 * N_BLOCKS) + [(CH, OUT_CH)]   # (in, out) per conv


QUANTIZE = True   # emulate the BF16 storage (tests of the definition switch it off)


def bf16(x: torch.Tensor) -> torch.Tensor:
    """Round to BF16 (round to nearest even) and back, gradient passed straight through."""
    if not QUANTIZE:
        return x
    r = x.to(torch.bfloat16).to(x.dtype)
    return x + (r - x).detach()


COMPACT_LAYERS = [(IN_CH, CH, 3), (CH, CH, 1), (CH, OUT_CH, 1)]   # (in, out, kernel size)


def init_params(seed: int = 0):
    """He-initialised weights [out, in, 3, 3] (float32) and zero biases, seeded."""
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for li, (cin, cout) in enumerate(LAYERS):
        fan_in = (4 if li == 0 else cin) * 9
        w = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(cout, cin, 3, 3)).astype(np.float32)
        if li == 0:
            w[:, 4:] = 0.0                      # padding channels of the input
        if li == N_CONV - 1:
            w[:] = 0.0                          # start at the bilinear base exactly
        ws.append(w)
        bs.append(np.zeros(cout, dtype=np.float32))
    return ws, bs


def forward(x0: torch.Tensor, ws, bs) -> torch.Tensor:
    """r [B, H2, W2, 16] (float64) from x0 [B, H2, W2, 16]; ws, bs float64 tensors."""
    h = bf16(x0).permute(0, 3, 1, 2)
    wq = [bf16(w) for w in ws]
    h = bf16(F.relu(F.conv2d(h, wq[0], bs[0], padding=1)))
    for b in range(N_BLOCKS):
        t = bf16(F.relu(F.conv2d(h, wq[1 + 2 * b], bs[1 + 2 * b], padding=1)))
        h = bf16(h + F.conv2d(t, wq[2 + 2 * b], bs[2 + 2 * b], padding=1))
    r = F.conv2d(h, wq[N_CONV - 1], bs[N_CONV - 1], padding=1)
    return r.permute(0, 2, 3, 1)


def init_compact_params(seed: int = 0):
    """He-initialised weights [out, in, k, k] (float32) and zero biases of the compact
    network, seeded; as in the residual network the unused input channels and the last layer
    start at zero, so the initial prediction is the base."""
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for li, (cin, cout, k) in enumerate(COMPACT_LAYERS):
        fan_in = (4 if li == 0 else cin) * k * k
        w = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(cout, cin, k, k)).astype(np.float32)
        if li == 0:
            w[:, 4:] = 0.0
        if li == len(COMPACT_LAYERS) - 1:
            w[:] = 0.0
        ws.append(w)
        bs.append(np.zeros(cout, dtype=np.float32))
    return ws, bs


def forward_compact(x0: torch.Tensor, ws, bs) -> torch.Tensor:
    """r [B, H2, W2, 16] (float64) of the compact network; ws [out, in, k, k], bs float64."""
    h = bf16(x0).permute(0, 3, 1, 2)
    wq = [bf16(w) for w in ws]
    h = bf16(F.relu(F.conv2d(h, wq[0], bs[0], padding=1)))
    t = bf16(F.relu(F.conv2d(h, wq[1], bs[1])))
    r = F.conv2d(t, wq[2], bs[2])
    return r.permute(0, 2, 3, 1)


def base(tl_rgb: torch.Tensor) -> torch.Tensor:
    """Bilinear base [B, H2, W2, 4, 3] of the quarter-density layer tl [B, H2, W2, 3]: entry
    2 dy + dx is the base of sub-pixel (dx, dy) (the last block repeated past the edge)."""
    a = tl_rgb
    right = torch.cat([a[:, :, 1:], a[:, :, -1:]], dim=2)
    down = torch.cat([a[:, 1:], a[:, -1:]], dim=1)
    diag = torch.cat([down[:, :, 1:], down[:, :, -1:]], dim=2)
    return torch.stack([a, (a + right) * 0.5, (a + down) * 0.5, (((a + right) + down) + diag) * 0.25],
                       dim=3)


def shuffle(r: torch.Tensor, tl_rgb: torch.Tensor, H: int, W: int) -> torch.Tensor:
    """Full-resolution prediction [B, H, W, 3]: bilinear base + residual of the sub-pixel."""
    B, H2, W2, _ = r.shape
    bs = base(tl_rgb.to(r.dtype))
    out = torch.empty((B, 2 * H2, 2 * W2, 3), dtype=r.dtype)
    for dy in range(2):
        for dx in range(2):
            out[:, dy::2, dx::2, :] = bs[:, :, :, 2 * dy + dx] + r[..., [c * 4 + 2 * dy + dx for c in range(3)]]
    return out[:, :H, :W]


def make_input(img: np.ndarray, depth: np.ndarray):
    """x0 [B, H2, W2, 16] and the top-left colours [B, H2, W2, 3] of images [B, H, W, 3] and
    depths [B, H, W] (the top-left pixel of every 2x2 block)."""
    tl = img[:, 0::2, 0::2, :]
    z = depth[:, 0::2, 0::2]
    B, H2, W2, _ = tl.shape
    x0 = np.zeros((B, H2, W2, IN_CH), dtype=np.float32)
    x0[..., :3] = tl
    x0[..., 3] = z * DEPTH_SCALE
    return x0, tl


def loss_and_grads(x0: np.ndarray, tl: np.ndarray, target: np.ndarray, ws, bs, net=None):
    """Mean squared error of the prediction over [B, H, W, 3] and its gradients (float64);
    ``net`` is ``forward`` (default) or ``forward_compact``."""
    net = forward if net is None else net
    W_ = [torch.tensor(np.asarray(w, np.float64), requires_grad=True) for w in ws]
    B_ = [torch.tensor(np.asarray(b, np.float64), requires_grad=True) for b in bs]
    H, W = target.shape[1:3]
    r = net(torch.tensor(x0, dtype=torch.float64), W_, B_)
    pred = shuffle(r, torch.tensor(tl, dtype=torch.float64), H, W)
    loss = ((pred - torch.tensor(target, dtype=torch.float64)) ** 2).mean()
    loss.backward()
    return float(loss), [w.grad.numpy() for w in W_], [b.grad.numpy() for b in B_], r.detach().numpy()


def conv3x3_loops(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain-loop 3x3 convolution with zero padding, x [H, W, Cin] -> [H, W, Cout] (float64);
    the definition the library conv2d is checked against."""
    H, W, _ = x.shape
    cout = w.shape[0]
    xp = np.zeros((H + 2, W + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    out = np.zeros((H, W, cout))
    for y in range(H):
        for xx in range(W):
            patch = xp[y:y + 3, xx:xx + 3, :]            # [3, 3, Cin]
            out[y, xx] = np.einsum("kli,okli->o", patch, w.transpose(0, 2, 3, 1)) + b
    return out


def conv1x1_loops(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain-loop per-pixel layer x [H, W, Cin] -> [H, W, Cout] with w [Cout, Cin] (float64)."""
    H, W, cin = x.shape
    cout = w.shape[0]
    out = np.zeros((H, W, cout))
    for y in range(H):
        for xx in range(W):
            for o in range(cout):
                acc = b[o]
                for i in range(cin):
                    acc += w[o, i] * x[y, xx, i]
                out[y, xx, o] = acc
    return out
