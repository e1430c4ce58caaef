"""Pins of the learned-periphery reference network (oracle/cnn.py) -- CPU only."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import cnn


def test_library_conv_equals_loop_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(7, 9, 5))
    w = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    ref = cnn.conv3x3_loops(x, w, b)
    got = F.conv2d(torch.tensor(x).permute(2, 0, 1)[None], torch.tensor(w), torch.tensor(b),
                   padding=1)[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_shuffle_places_each_subpixel():
    B, H2, W2 = 1, 2, 3
    r = torch.arange(B * H2 * W2 * 16, dtype=torch.float64).reshape(B, H2, W2, 16)
    tl = torch.full((B, H2, W2, 3), 1000.0, dtype=torch.float64)
    out = cnn.shuffle(r, tl, 4, 5)                 # ragged: the last column is cut
    assert out.shape == (1, 4, 5, 3)
    for y in range(4):
        for x in range(5):
            for c in range(3):
                k = c * 4 + 2 * (y % 2) + (x % 2)
                assert out[0, y, x, c] == 1000.0 + r[0, y // 2, x // 2, k]


def test_gradients_equal_central_differences():
    cnn.QUANTIZE = False
    try:
        rng = np.random.default_rng(1)
        ws, bs = cnn.init_params(3)
        ws = [w + rng.normal(0, 0.05, w.shape).astype(np.float32) for w in ws]
        bs = [b + rng.normal(0, 0.05, b.shape).astype(np.float32) for b in bs]
        img = rng.uniform(size=(1, 10, 12, 3))
        depth = rng.uniform(2, 6, size=(1, 10, 12))
        x0, tl = cnn.make_input(img, depth)
        target = img + rng.normal(0, 0.05, img.shape)
        loss, gw, gb, _ = cnn.loss_and_grads(x0, tl, target, ws, bs)

        def L(ws_, bs_):
            r = cnn.forward(torch.tensor(x0, dtype=torch.float64),
                            [torch.tensor(np.asarray(w, np.float64)) for w in ws_],
                            [torch.tensor(np.asarray(b, np.float64)) for b in bs_])
            pred = cnn.shuffle(r, torch.tensor(tl, dtype=torch.float64), 10, 12)
            return float(((pred - torch.tensor(target)) ** 2).mean())

        h = 1e-6
        for li, idx in [(0, (3, 1, 0, 2)), (4, (7, 30, 1, 1)), (9, (5, 12, 2, 0)), (9, (11, 0, 1, 1))]:
            wp = [np.asarray(w, np.float64).copy() for w in ws]
            wm = [np.asarray(w, np.float64).copy() for w in ws]
            wp[li][idx] += h
            wm[li][idx] -= h
            fd = (L(wp, bs) - L(wm, bs)) / (2 * h)
            assert abs(fd - gw[li][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, gw[li][idx])
        for li, k in [(2, 5), (9, 7)]:
            bp = [np.asarray(b, np.float64).copy() for b in bs]
            bm = [np.asarray(b, np.float64).copy() for b in bs]
            bp[li][k] += h
            bm[li][k] -= h
            fd = (L(ws, bp) - L(ws, bm)) / (2 * h)
            assert abs(fd - gb[li][k]) <= 1e-6 * max(1.0, abs(fd))
    finally:
        cnn.QUANTIZE = True


def test_base_is_bilinear_on_a_ramp_and_repeats_at_the_edge():
    """The base reproduces a linear ramp exactly inside the layer (bilinear interpolation at
    the sub-pixel positions) and repeats the last block past the right and bottom edges."""
    H2, W2 = 4, 5
    yy, xx = np.meshgrid(np.arange(H2), np.arange(W2), indexing="ij")
    ramp = lambda y, x: 0.25 + 0.5 * x - 0.125 * y        # value at pixel (2x2 + x, 2y2 + y) / 2
    tl = np.stack([ramp(yy, xx)] * 3, -1)[None]
    b = cnn.base(torch.tensor(tl, dtype=torch.float64)).numpy()[0]
    for dy in range(2):
        for dx in range(2):
            want = ramp(yy + 0.5 * dy, xx + 0.5 * dx)
            inner = (xx + dx < W2) & (yy + dy < H2)
            np.testing.assert_allclose(b[..., 2 * dy + dx, 0][inner], want[inner], rtol=0, atol=1e-15)
    # past the right edge the (1, 0) base is the last block itself
    np.testing.assert_array_equal(b[:, -1, 1, 0], tl[0, :, -1, 0])
    np.testing.assert_array_equal(b[-1, :, 2, 0], tl[0, -1, :, 0])


def test_initial_network_is_near_the_base():
    rng = np.random.default_rng(2)
    ws, bs = cnn.init_params(0)
    img = rng.uniform(size=(1, 32, 32, 3))
    x0, tl = cnn.make_input(img, rng.uniform(2, 6, size=(1, 32, 32)))
    r = cnn.forward(torch.tensor(x0, dtype=torch.float64), [torch.tensor(np.asarray(w, np.float64)) for w in ws],
                    [torch.tensor(np.asarray(b, np.float64)) for b in bs])
    assert r.abs().max() == 0.0                    # zero last layer: the prediction is the base


# ------------------------------------------------------------------ the compact network
def test_library_1x1_equals_loop_definition():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(5, 6, 7))
    w = rng.normal(size=(3, 7))
    b = rng.normal(size=3)
    ref = cnn.conv1x1_loops(x, w, b)
    got = F.conv2d(torch.tensor(x).permute(2, 0, 1)[None], torch.tensor(w)[:, :, None, None],
                   torch.tensor(b))[0].permute(1, 2, 0).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_compact_forward_equals_plain_loops():
    """Unquantised, the compact network is 3x3 conv + ReLU, per-block layer + ReLU, per-block
    layer, composed from the plain-loop definitions (a misplaced ReLU, bias or padding fails)."""
    cnn.QUANTIZE = False
    try:
        rng = np.random.default_rng(5)
        ws, bs = cnn.init_compact_params(1)
        ws = [w + rng.normal(0, 0.1, w.shape).astype(np.float32) for w in ws]
        bs = [b + rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
        x0 = rng.normal(size=(1, 5, 6, 16))
        r = cnn.forward_compact(torch.tensor(x0), [torch.tensor(np.asarray(w, np.float64)) for w in ws],
                                [torch.tensor(np.asarray(b, np.float64)) for b in bs]).numpy()[0]
        h = np.maximum(cnn.conv3x3_loops(x0[0], ws[0].astype(np.float64), bs[0]), 0.0)
        t = np.maximum(cnn.conv1x1_loops(h, ws[1][:, :, 0, 0].astype(np.float64), bs[1]), 0.0)
        ref = cnn.conv1x1_loops(t, ws[2][:, :, 0, 0].astype(np.float64), bs[2])
        np.testing.assert_allclose(r, ref, rtol=1e-10, atol=1e-10)
        assert (h == 0).any() and (t == 0).any() and (ref < 0).any()   # both ReLUs and a sign in play
    finally:
        cnn.QUANTIZE = True


def test_compact_gradients_equal_central_differences():
    cnn.QUANTIZE = False
    try:
        rng = np.random.default_rng(6)
        ws, bs = cnn.init_compact_params(2)
        ws = [w + rng.normal(0, 0.05, w.shape).astype(np.float32) for w in ws]
        bs = [b + rng.normal(0, 0.05, b.shape).astype(np.float32) for b in bs]
        img = rng.uniform(size=(1, 10, 12, 3))
        depth = rng.uniform(2, 6, size=(1, 10, 12))
        x0, tl = cnn.make_input(img, depth)
        target = img + rng.normal(0, 0.05, img.shape)
        loss, gw, gb, _ = cnn.loss_and_grads(x0, tl, target, ws, bs, net=cnn.forward_compact)

        def L(ws_, bs_):
            r = cnn.forward_compact(torch.tensor(x0, dtype=torch.float64),
                                    [torch.tensor(np.asarray(w, np.float64)) for w in ws_],
                                    [torch.tensor(np.asarray(b, np.float64)) for b in bs_])
            pred = cnn.shuffle(r, torch.tensor(tl, dtype=torch.float64), 10, 12)
            return float(((pred - torch.tensor(target)) ** 2).mean())

        h = 1e-6
        for li, idx in [(0, (3, 1, 0, 2)), (0, (30, 3, 2, 2)), (1, (7, 30, 0, 0)), (2, (5, 12, 0, 0)),
                        (2, (11, 0, 0, 0))]:
            wp = [np.asarray(w, np.float64).copy() for w in ws]
            wm = [np.asarray(w, np.float64).copy() for w in ws]
            wp[li][idx] += h
            wm[li][idx] -= h
            fd = (L(wp, bs) - L(wm, bs)) / (2 * h)
            assert abs(fd - gw[li][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, gw[li][idx])
        for li, k in [(0, 5), (1, 9), (2, 7)]:
            bp = [np.asarray(b, np.float64).copy() for b in bs]
            bm = [np.asarray(b, np.float64).copy() for b in bs]
            bp[li][k] += h
            bm[li][k] -= h
            fd = (L(ws, bp) - L(ws, bm)) / (2 * h)
            assert abs(fd - gb[li][k]) <= 1e-6 * max(1.0, abs(fd))
    finally:
        cnn.QUANTIZE = True


def test_initial_compact_network_is_the_base():
    rng = np.random.default_rng(7)
    ws, bs = cnn.init_compact_params(0)
    assert [w.shape for w in ws] == [(32, 16, 3, 3), (32, 32, 1, 1), (16, 32, 1, 1)]
    img = rng.uniform(size=(1, 16, 20, 3))
    x0, tl = cnn.make_input(img, rng.uniform(2, 6, size=(1, 16, 20)))
    r = cnn.forward_compact(torch.tensor(x0, dtype=torch.float64),
                            [torch.tensor(np.asarray(w, np.float64)) for w in ws],
                            [torch.tensor(np.asarray(b, np.float64)) for b in bs])
    assert r.abs().max() == 0.0
