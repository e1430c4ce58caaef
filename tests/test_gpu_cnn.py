"""Learned periphery on the tensor cores: kernels against the CPU oracle of the network."""
import math

import numpy as np
import pytest

import paper_2507_04147_gb300 as a3fr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("n,k", [(32, 16), (32, 64), (16, 48)])
def test_tensor_core_tile_gemm(n, k):
    import torch
    g = torch.Generator().manual_seed(n * 100 + k)
    A = torch.randn(128, k, generator=g).to(torch.bfloat16)
    B = torch.randn(n, k, generator=g).to(torch.bfloat16)
    D = torch.empty(128, n, device="cuda")
    a3fr.tc_tile_gemm(A.cuda(), B.cuda(), D, variant=0)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    err = (D.cpu().double() - ref).abs().max().item()
    assert err < 1e-4 * max(1.0, ref.abs().max().item()), err


# ------------------------------------------------------------------ the network
import torch as _t                                            # noqa: E402

from oracle import cnn as ocnn                                # noqa: E402
from paper_2507_04147_gb300 import periphery, synth           # noqa: E402


def random_params(seed, arch=periphery.RESIDUAL):
    rng = np.random.default_rng(seed)
    flat = periphery.init_params(seed, arch)
    ws, bs = periphery.unpack(flat.copy(), arch)
    for li, w in enumerate(ws):
        w += rng.normal(0, 0.02, w.shape).astype(np.float32)
        if li == 0:
            w[:, 4:] = 0.0
    for b in bs:
        b += rng.normal(0, 0.05, b.shape).astype(np.float32)
    return periphery.pack(ws, bs)


def random_images(seed, b=2, h=40, w=56):
    rng = np.random.default_rng(seed)
    img = rng.uniform(0, 1, size=(b, h, w, 3)).astype(np.float32)
    depth = rng.uniform(0, 6, size=(b, h, w)).astype(np.float32)
    return img, depth


ORACLE_NET = {periphery.RESIDUAL: ocnn.forward, periphery.COMPACT: ocnn.forward_compact}


@pytest.mark.parametrize("arch", [periphery.RESIDUAL, periphery.COMPACT])
def test_network_forward_matches_reference(arch):
    flat = random_params(1, arch)
    img, depth = random_images(2)
    net = periphery.Periphery(flat, arch=arch)
    r = net.forward(_t.from_numpy(img).cuda(), _t.from_numpy(depth).cuda()).cpu().numpy()
    net.close()
    ws, bs = periphery.unpack(flat, arch)
    x0, _ = ocnn.make_input(img, depth)
    ref = ORACLE_NET[arch](_t.tensor(x0, dtype=_t.float64), [_t.tensor(w, dtype=_t.float64) for w in ws],
                           [_t.tensor(b, dtype=_t.float64) for b in bs]).numpy()
    scale = np.abs(ref).max()
    err = np.abs(r - ref)
    print("forward max", err.max() / scale, "mean", err.mean() / scale)
    assert err.max() <= 3e-2 * scale and err.mean() <= 2e-3 * scale


@pytest.mark.parametrize("arch", [periphery.RESIDUAL, periphery.COMPACT])
def test_network_gradients_match_reference(arch):
    flat = random_params(3, arch)
    img, depth = random_images(4)
    rng = np.random.default_rng(5)
    target = np.clip(img + rng.normal(0, 0.1, img.shape), 0, 1).astype(np.float32)
    net = periphery.Periphery(flat, arch=arch)
    g, loss = net.grads(_t.from_numpy(img).cuda(), _t.from_numpy(depth).cuda(), _t.from_numpy(target).cuda())
    net.close()
    ws, bs = periphery.unpack(flat, arch)
    x0, tl = ocnn.make_input(img, depth)
    ref_loss, gw, gb, _ = ocnn.loss_and_grads(x0, tl, target, ws, bs, net=ORACLE_NET[arch])
    assert loss == pytest.approx(ref_loss, rel=2e-3)
    gws, gbs = periphery.unpack(g, arch)
    for li in range(len(gw)):
        for got, ref, kind in ((gws[li], gw[li], "w"), (gbs[li], gb[li], "b")):
            rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-12)
            print(li, kind, rel)
            assert rel <= 5e-2, (li, kind, rel)


@pytest.mark.parametrize("arch,lr0,min_gain_itp", [(periphery.RESIDUAL, 3e-5, 1.0), (periphery.COMPACT, 1e-3, 0.5)])
def test_learned_fill_beats_inherit_and_interpolating_fills(arch, lr0, min_gain_itp):
    """Trained on the rasterizer's own renders, the network's fill of a foveated render is
    closer to the full-resolution render than the inherit fill (by several dB: it starts from
    the bilinear base) and than the interpolating fill, on views it never saw."""
    import paper_2507_04147_gb300 as a3fr
    scene_np = synth.uniform_scene(200_000, 1, seed=3, log_scale_mean=-3.6)
    scene = a3fr.Scene.from_numpy(scene_np)
    scene.keep_aux(True)
    rng = np.random.default_rng(0)
    train_cams = [synth.pinhole_camera(384, 384, yaw_deg=float(y)) for y in rng.uniform(-20, 20, 24)]
    imgs, deps = periphery.render_crops(scene, train_cams, 96, 8, rng)
    net = periphery.Periphery(seed=0, arch=arch)
    probe = (imgs[:16].contiguous(), deps[:16].contiguous(), imgs[:16].contiguous())
    first = net.grads(*probe)[1]
    for step in range(300):
        idx = _t.from_numpy(rng.choice(len(imgs), 16, replace=False)).cuda()
        lr = lr0 * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * step / 300)))
        net.train_step(imgs[idx].contiguous(), deps[idx].contiguous(), imgs[idx].contiguous(), lr)
    last = net.grads(*probe)[1]
    assert last < first
    fv = a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1))
    gains = []
    for yaw in (27.0, -27.0, 33.0):
        cam = synth.pinhole_camera(384, 384, yaw_deg=yaw)
        scene.set_camera(0, cam)
        full = scene.render_full().clone()
        scene.set_gaze([[40.0, 40.0]])
        inh = scene.render_foveated(fv).clone()
        lv = scene.buffer(a3fr.BUF_LEVELS, _t.uint8).reshape(24, 24)
        itp = scene.render_foveated(a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1),
                                               fill=a3fr.FILL_INTERPOLATE)).clone()
        learned = inh.clone()
        scene.render_foveated(fv, out=learned)
        net.fill(scene, learned)
        _t.cuda.synchronize()
        per = (lv == 1).repeat_interleave(16, 0).repeat_interleave(16, 1)[None]
        p_inh = periphery.psnr(inh, full, per)
        p_itp = periphery.psnr(itp, full, per)
        p_cnn = periphery.psnr(learned, full, per)
        print(yaw, "periphery PSNR inherit", p_inh, "interpolate", p_itp, "learned", p_cnn)
        gains.append((p_cnn - p_inh, p_cnn - p_itp))
    net.close()
    scene.close()
    assert min(g[0] for g in gains) > 3.0, gains
    assert min(g[1] for g in gains) > min_gain_itp, gains


@pytest.mark.parametrize("arch", [periphery.RESIDUAL, periphery.COMPACT])
@pytest.mark.parametrize("tile,width,height,eyes", [(16, 201, 137, 1), (32, 256, 192, 1), (32, 203, 141, 2)])
def test_fused_fill_equals_forward_plus_compose(tile, width, height, eyes, arch):
    """The fill runs its first convolution on the render directly and composes in the last
    one's epilogue (the compact network: all three layers in one kernel); its image equals
    the training forward's residuals composed here: rendered pixels kept, each skipped
    sub-pixel = bilinear base of the top-left pixels (last block repeated past the edge) + its
    residual, bit for bit.  Ragged blocks at odd sizes; a stereo frame whose second eye starts
    4 bytes off an 8-byte boundary (odd pixel count).  The compact network's training forward
    runs its per-block layers as 3x3 convolutions whose other taps are zero (18 MMAs where the
    fused kernel issues 2): the zero products leave every accumulator unchanged."""
    import paper_2507_04147_gb300 as a3fr
    scene_np = synth.uniform_scene(20000, 1, seed=5, log_scale_mean=-3.6)
    scene = a3fr.Scene.from_numpy(scene_np, tile=tile)
    scene.keep_aux(True)
    cams = [synth.pinhole_camera(width, height)] if eyes == 1 else synth.stereo_cameras(width, height, yaw_deg=4.0)
    for e, cam in enumerate(cams):
        scene.set_camera(e, cam)
    scene.set_gaze([[0.3 * width, 0.4 * height], [0.6 * width, 0.5 * height]][:eyes])
    fv = a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1))
    got = _t.empty((eyes, height, width, 3), dtype=_t.float32, device="cuda")
    scene.render_foveated(fv, out=got)
    img = got.clone()
    depth = scene.buffer(a3fr.BUF_DEPTH, _t.float32).reshape(eyes, height, width)
    tx = (width + tile - 1) // tile
    ty = (height + tile - 1) // tile
    levels_all = scene.buffer(a3fr.BUF_LEVELS, _t.uint8).reshape(eyes, ty, tx).long()
    net = periphery.Periphery(random_params(11, arch), arch=arch)
    r = net.forward(img, depth)                      # [eyes, H2, W2, 16]
    net.fill(scene, got)
    _t.cuda.synchronize()
    net.close()
    scene.close()
    # compose the reference from img and r (fp32, the kernel's order of operations)
    H2, W2 = (height + 1) // 2, (width + 1) // 2
    xr = _t.clamp(_t.arange(W2, device="cuda") + 1, max=W2 - 1)
    yd = _t.clamp(_t.arange(H2, device="cuda") + 1, max=H2 - 1)
    ys, xs = _t.meshgrid(_t.arange(H2, device="cuda"), _t.arange(W2, device="cuda"), indexing="ij")
    for e in range(eyes):
        levels = levels_all[e]
        tl = img[e, 0::2, 0::2]                       # [H2, W2, 3]
        a, right, down, diag = tl, tl[:, xr], tl[yd], tl[yd][:, xr]
        lv = levels[(2 * ys) // tile, (2 * xs) // tile][..., None]
        res = r[e]
        ref = img.clone()[e]
        bt = (a + right) * 0.5
        bb = (a + down) * 0.5
        bd = (((a + right) + down) + diag) * 0.25
        for dy, dx, base, need in ((0, 1, bt, 2), (1, 0, bb, 3), (1, 1, bd, 1)):
            val = base + res[..., [4 * c + 2 * dy + dx for c in range(3)]]
            sel = (lv <= need).expand_as(val)
            ry, rx = 2 * ys + dy, 2 * xs + dx
            ok = ((ry < height) & (rx < width))[..., None].expand_as(val) & sel
            cur = ref[ry.clamp(max=height - 1), rx.clamp(max=width - 1)]
            ref[ry[ok[..., 0]], rx[ok[..., 0]]] = _t.where(ok, val, cur)[ok[..., 0]]
        assert bool((levels < 4).any()) and bool((levels == 4).any())
        diff = (got[e] - ref).abs().max().item()
        assert _t.equal(got[e], ref), (e, diff)
