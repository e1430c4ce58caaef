"""Backward rasterizer on the GPU (through the C ABI) against the fp64 gradient oracle.

Bar: per parameter group, the largest absolute difference to the oracle gradient is at most
2e-3 of the group's largest oracle magnitude, and the relative L2 difference at most 1e-3.
Derivation: the GPU forward is fp32 with a MUFU ex2 (relative error ~2^-22), the backward
recovers T by division over up to a few hundred contributors and sums per-Gaussian terms
with fp32 atomics (relative rounding ~1e-6 per term, a few hundred to thousands of terms),
so elements are good to ~1e-5 of the group scale; the bound leaves two orders of margin
while a wrong term (a sign, a missing factor, a transposed operand) moves whole groups by
O(1).  Pixels whose oracle decision margin is below 1e-4 get zero upstream gradient, since
fp32 and fp64 may take a different alpha / stop decision there.
"""
import numpy as np
import pytest

import oracle
from oracle import grad as og
import paper_2507_04147_gb300 as a3fr
from paper_2507_04147_gb300 import synth

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_grads(scene_np, cams, dl, fovea=None, gaze=None, tile=16):
    import torch
    s = a3fr.Scene.from_numpy(scene_np, tile=tile)
    for e, c in enumerate(cams):
        s.set_camera(e, c)
    s.keep_aux(True)
    if fovea is None:
        img = s.render_full()
    else:
        s.set_gaze(gaze)
        img = s.render_foveated(fovea)
    g = s.backward(torch.from_numpy(np.ascontiguousarray(dl, dtype=np.float32)).cuda())
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    out["img"] = img.cpu().numpy()
    out["levels"] = s.buffer(a3fr.BUF_LEVELS, torch.uint8).cpu().numpy()
    s.close()
    return out


def compare(gpu, ref, names=NAMES):
    report = {}
    for k in names:
        a, b = gpu[k].ravel(), ref[k].ravel()
        scale = np.abs(b).max()
        assert scale > 0, k
        max_err = np.abs(a - b).max() / scale
        l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
        report[k] = (float(max_err), float(l2))
        assert max_err <= 2e-3 and l2 <= 1e-3, (k, max_err, l2)
    return report


def small_scene(n=64, seed=7):
    return synth.uniform_scene(n, 3, seed=seed, log_scale_mean=-1.8, log_scale_std=0.3)


def masked_weights(scene_np, cam, seed, pixels=None, tile=16):
    rng = np.random.default_rng(seed)
    npx = cam.width * cam.height if pixels is None else len(pixels)
    w = rng.normal(size=(npx, 3))
    _, _, info = og.loss(og.params_f64(scene_np), scene_np, cam, tile, np.zeros((npx, 3)), pixels=pixels)
    w[info["margin"] < 1e-4] = 0.0
    return w


def test_small_scene_matches_oracle_gradient():
    s = small_scene()
    cam = synth.pinhole_camera(32, 32)
    w = masked_weights(s, cam, 1)
    ref = og.gradient(s, cam, 16, w)
    gpu = gpu_grads(s, [cam], w.reshape(1, 32, 32, 3))
    print(compare(gpu, ref))


def test_tile32_stereo_foveated_matches_oracle_gradient():
    """32-pixel tiles: each quadrant of a tile walks the tile's list for its own pixels."""
    s = synth.uniform_scene(500, 3, seed=23, log_scale_mean=-2.5, log_scale_std=0.4)
    cams = synth.stereo_cameras(72, 56, yaw_deg=1.0)
    ws = [masked_weights(s, c, 30 + e, tile=32) for e, c in enumerate(cams)]
    ref = [og.gradient(s, c, 32, w) for c, w in zip(cams, ws)]
    tot = {k: ref[0][k] + ref[1][k] for k in NAMES}
    gpu = gpu_grads(s, cams, np.stack(ws).reshape(2, 56, 72, 3), tile=32)
    print(compare(gpu, tot))


def test_small_scene_matches_central_differences():
    """GPU gradient against fp64 central differences (h = 1e-4) of the oracle forward."""
    s = small_scene(seed=11)
    cam = synth.pinhole_camera(32, 32)
    w = masked_weights(s, cam, 2)
    gpu = gpu_grads(s, [cam], w.reshape(1, 32, 32, 3))
    vis = og.Visibility(s, cam, 16)
    rng = np.random.default_rng(5)
    active = np.nonzero(np.abs(gpu["opacity_logits"]) > 1e-6)[0]
    checked = 0
    for name, idxs in (("means", [(i, k) for i in rng.choice(active, 6, replace=False) for k in range(3)]),
                       ("log_scales", [(i, k) for i in rng.choice(active, 6, replace=False) for k in range(3)]),
                       ("quats", [(i, k) for i in rng.choice(active, 4, replace=False) for k in range(4)]),
                       ("opacity_logits", [(i,) for i in rng.choice(active, 10, replace=False)]),
                       ("sh", [(i, k, c) for i in rng.choice(active, 3, replace=False)
                               for k in (0, 3, 8, 15) for c in (0, 1)])):
        scale = np.abs(gpu[name]).max()
        for idx in idxs:
            fd, flipped = og.finite_difference(s, cam, 16, w, name, idx, h=1e-4, vis=vis)
            if flipped:
                continue
            assert abs(gpu[name][idx] - fd) <= 2e-3 * scale + 1e-3 * abs(fd), (name, idx, gpu[name][idx], fd)
            checked += 1
    assert checked >= 60


def test_stereo_ragged_and_foveated_backward():
    """Two eyes (gradients summed), a ragged image, and a foveated render whose inherited
    pixels pass their gradient to the top-left pixel of their block."""
    s = synth.uniform_scene(600, 3, seed=21, log_scale_mean=-2.5, log_scale_std=0.4)
    cams = synth.stereo_cameras(72, 56, yaw_deg=2.0)
    rng = np.random.default_rng(4)
    ws = [masked_weights(s, c, 10 + e) for e, c in enumerate(cams)]
    # full resolution
    ref = [og.gradient(s, c, 16, w) for c, w in zip(cams, ws)]
    tot = {k: ref[0][k] + ref[1][k] for k in NAMES}
    gpu = gpu_grads(s, cams, np.stack(ws).reshape(2, 56, 72, 3))
    print("full", compare(gpu, tot))
    # foveated: weights folded onto the rendered pixel each output pixel copies
    fv_o = oracle.fovea((18.0, 36.0), 0.0, (4, 2, 1))
    gaze = np.array([[20.0, 30.0], [18.0, 30.0]], np.float32)
    folded, inputs = [], []
    for e, c in enumerate(cams):
        lv = oracle.level_map(c, 16, fv_o, gaze[e])
        img = oracle.render(*oracle.preprocess(s, c, 16)[:2], c, 16, level=lv)
        live = img.rendered.reshape(56, 72).astype(bool)
        _, _, info = og.loss(og.params_f64(s), s, c, 16, np.zeros((56 * 72, 3)))
        near = (info["margin"] < 1e-4).reshape(56, 72)
        w = ws[e].reshape(56, 72, 3).copy()
        ys, xs = np.nonzero(~live)
        # an inherited pixel copies its block's top-left pixel: its weight counts there
        w[ys[near[ys & ~1, xs & ~1]], xs[near[ys & ~1, xs & ~1]]] = 0.0
        f = np.where(live[..., None], w, 0.0)
        np.add.at(f, (ys & ~1, xs & ~1), w[ys, xs])
        folded.append(f.reshape(-1, 3))
        inputs.append(w)
    ref = [og.gradient(s, c, 16, f) for c, f in zip(cams, folded)]
    tot = {k: ref[0][k] + ref[1][k] for k in NAMES}
    gpu = gpu_grads(s, cams, np.stack(inputs), fovea=a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1)),
                    gaze=gaze)
    print("foveated", compare(gpu, tot))


def test_backward_requires_an_aux_render():
    import torch
    s = a3fr.Scene.from_numpy(small_scene())
    s.set_camera(0, synth.pinhole_camera(32, 32))
    s.render_full()                     # keep_aux off: nothing to walk back from
    with pytest.raises(a3fr.A3FRError, match="NOT_READY"):
        s.backward(torch.zeros((1, 32, 32, 3), device="cuda"))
    s.close()


def test_autograd_training_reduces_the_loss():
    import torch
    from paper_2507_04147_gb300.autograd import GaussianRasterizer, render
    target_np = synth.uniform_scene(400, 1, seed=31, log_scale_mean=-2.6, log_scale_std=0.3)
    cam = synth.pinhole_camera(64, 64)
    tgt = a3fr.Scene.from_numpy(target_np)
    tgt.set_camera(0, cam)
    target = tgt.render_full().clone()
    rng = np.random.default_rng(0)
    f = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda", requires_grad=True)
    params = [f(target_np.means + rng.normal(0, 0.02, target_np.means.shape)),
              f(target_np.log_scales), f(target_np.quats),
              f(target_np.opacity_logits + rng.normal(0, 0.5, 400)),
              f(target_np.sh + rng.normal(0, 0.2, target_np.sh.shape))]
    rast = GaussianRasterizer(*params)
    rast.set_camera(0, cam)
    opt = torch.optim.Adam(params, lr=5e-3)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        img = render(rast)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert all(p.grad is not None and torch.isfinite(p.grad).all() for p in params)
    assert losses[-1] < 0.5 * losses[0], losses


def test_one_million_gaussians_1024_sampled_gradients():
    """1M Gaussians, SH3, 1024x1024: gradients of sampled Gaussians against the oracle
    restricted to the tiles each one touches (its gradient depends on no other pixel)."""
    import torch
    s = synth.uniform_scene(1_000_000, 3, seed=5)
    cam = synth.pinhole_camera(1024, 1024)
    rng = np.random.default_rng(9)
    w = rng.normal(size=(1024 * 1024, 3)).astype(np.float32)
    rec, rect, touched = oracle.preprocess(s, cam, 16)
    cand = np.nonzero((touched >= 1) & (touched <= 2) & (rec[:, 5] > 0.3))[0]
    picks = rng.choice(cand, 12, replace=False)
    # pixels of each pick's tiles; zero the weights of near-threshold pixels there
    pix_sets = []
    for g in picks:
        x0, y0, x1, y1 = rect[g]
        ys, xs = np.mgrid[y0 * 16:y1 * 16, x0 * 16:x1 * 16]
        pix_sets.append(np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int64))
    params = og.params_f64(s)
    proj = og.project(params, cam, 3)
    vis = og.Visibility(s, cam, 16)
    for pix in pix_sets:
        _, info = og.composite(proj, vis, pix)
        lin = pix[:, 1] * 1024 + pix[:, 0]
        w[lin[info["margin"] < 1e-4]] = 0.0
    gpu = gpu_grads(s, [cam], w.reshape(1, 1024, 1024, 3))
    for g, pix in zip(picks, pix_sets):
        lin = pix[:, 1] * 1024 + pix[:, 0]
        ref = og.gradient(s, cam, 16, w[lin].astype(np.float64), pixels=pix)
        for k in NAMES:
            a, b = gpu[k][g].ravel(), ref[k][g].ravel()
            scale = max(np.abs(b).max(), 1e-6)
            assert np.abs(a - b).max() <= 2e-3 * scale + 1e-7, (k, g, a, b)
