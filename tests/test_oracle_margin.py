"""Pins of the oracle's threshold margin and of its flipped-decision colour (no GPU).

The GPU parity tests accept a pixel when it matches the oracle within 2e-4, or, where the
oracle's margin to the alpha >= 1/255 skip or to the T >= 1e-4 stop (Sec. 2.3
"Rasterization") is below 1e-5, when it matches the oracle's colour with that nearest
decision taken the other way.  Both the margin and that colour are therefore checked here
against closed forms on hand-built records: a Gaussian whose alpha is 1/255 at known
pixels, and a two-Gaussian stack whose transmittance lands on 1e-4.  A margin taken
against the wrong threshold, without its 255 or 10^4 scale, or with the stop decision
dropped, fails one of them; so does a flipped colour that flips the wrong decision.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_04147_gb300 import synth


def _record(u, v, a, b, c, opacity, rgb, depth):
    r = np.zeros(12, np.float32)
    r[:12] = [u, v, a, b, c, opacity, rgb[0], rgb[1], rgb[2], depth, 20.0, 1.0]
    return r


def _render(recs, width=64, height=64, tile=16):
    rec = np.stack(recs).astype(np.float32)
    tx, ty = oracle.tiles(width, tile), oracle.tiles(height, tile)
    rect = np.tile(np.int32([0, 0, tx, ty]), (len(recs), 1))
    cam = synth.pinhole_camera(width, height)
    return oracle.render(rec, rect, cam, tile), width, height


def test_alpha_skip_margin_and_flip_closed_form():
    """One Gaussian with alpha = 1/255 (to fp32 rounding) at the four pixels 3 px from its
    centre along the axes.  Closed form of the margin at every pixel: |255 raw - 1| with
    raw = o exp(-0.5 A d^2) (the stop decision, ~10^2 or more away, never wins)."""
    o = 0.5
    A = np.float32(math.log(255.0 * o) / 4.5)        # o exp(-0.5 A 9) = 1/255
    colour = (0.8, 0.6, 0.4)
    img, W, H = _render([_record(20.0, 30.0, A, 0.0, A, o, colour, 3.0)])
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs - 20.0) ** 2 + (ys - 30.0) ** 2
    raw = o * np.exp(-0.5 * float(A) * d2)
    alpha = np.minimum(0.99, raw)
    m_skip = np.abs(255.0 * raw - 1.0)
    m_stop = np.where(alpha >= 1 / 255, np.abs(1e4 * (1.0 - alpha) - 1.0), np.inf)
    margin = np.minimum(m_skip, m_stop).reshape(-1)
    np.testing.assert_allclose(img.margin, margin, rtol=1e-5, atol=2e-6)
    near = np.flatnonzero(img.margin < 1e-5)
    assert sorted(near.tolist()) == sorted([30 * W + 17, 30 * W + 23, 27 * W + 20, 33 * W + 20])
    for p in near:
        # flipping the skip adds or removes exactly this Gaussian's weight raw * T (T = 1)
        diff = np.abs(img.rgb[p].astype(np.float64) - img.rgb_alt[p])
        np.testing.assert_allclose(diff, np.array(colour) * raw.reshape(-1)[p], rtol=1e-5)
        assert min(np.abs(img.rgb[p]).max(), np.abs(img.rgb_alt[p]).max()) == 0.0
    far = img.margin >= 1e-3
    assert far.sum() == W * H - 4 - (img.margin[~far] >= 1e-5).sum()
    assert np.array_equal(img.rgb[far], img.rgb_alt[far])


@pytest.mark.parametrize("o2", [np.float32(0.99), np.nextafter(np.float32(0.99), np.float32(0.0))])
def test_stop_margin_and_flip_closed_form(o2):
    """Two coincident Gaussians at the pixel centre (power 0): the front one at the 0.99
    clamp leaves T1 = 1 - 0.99; the back one, of opacity o2, would leave T' = T1 (1 - o2),
    which lands on 1e-4 within a few fp32 ulps (below with o2 = 0.99: the pixel stops
    before it; above with the next smaller o2: it blends).  Margin |10^4 T' - 1|; the
    flipped colour adds or removes the back Gaussian's weight o2 T1."""
    c1, c2 = (0.9, 0.2, 0.1), (0.1, 0.3, 0.7)
    tiny = np.float32(1e-6)
    img, W, H = _render([_record(10.0, 10.0, tiny, 0.0, tiny, 1.0, c1, 2.0),
                         _record(10.0, 10.0, tiny, 0.0, tiny, o2, c2, 3.0)])
    p = 10 * W + 10
    a1 = float(np.float32(0.99))
    t1 = float(np.float32(1.0) - np.float32(a1))
    t2 = t1 * (1.0 - float(o2))
    assert img.margin[p] < 1e-5
    assert abs(img.margin[p] - abs(1e4 * t2 - 1.0)) < 1e-6
    front = np.array(c1) * a1
    back = np.array(c2) * float(o2) * t1
    stops = t2 < 1e-4
    main, alt = (front, front + back) if stops else (front + back, front)
    np.testing.assert_allclose(img.rgb[p], main, rtol=1e-5)
    np.testing.assert_allclose(img.rgb_alt[p], alt, rtol=1e-5)
    assert img.n_contrib[p] == (1 if stops else 2)


def test_margin_is_the_smallest_over_the_decisions():
    """The stop pixel of the stack above plus, behind it, a Gaussian whose alpha at that
    pixel is 1/255 (1.0001/255, so it passes): the stop decision is nearer (|10^4 T' - 1|
    ~ 2e-6 against 1e-4), so the margin and the flip are the stop's -- and the pixel never
    reaches the third Gaussian, so its decision does not count."""
    tiny = np.float32(1e-6)
    img, W, H = _render([_record(10.0, 10.0, tiny, 0.0, tiny, 1.0, (0.9, 0.2, 0.1), 2.0),
                         _record(10.0, 10.0, tiny, 0.0, tiny, 0.99, (0.1, 0.3, 0.7), 3.0),
                         _record(10.0, 10.0, tiny, 0.0, tiny, 1.0001 / 255, (1.0, 1.0, 1.0), 4.0)])
    p = 10 * W + 10
    t1 = float(np.float32(1.0) - np.float32(0.99))
    assert abs(img.margin[p] - abs(1e4 * t1 * (1.0 - float(np.float32(0.99))) - 1.0)) < 1e-6
    # flipped: the second Gaussian blends, then the third (alpha 1.0001/255) stops the pixel
    # since T would fall below 1e-4 again
    np.testing.assert_allclose(img.rgb_alt[p].astype(np.float64) - img.rgb[p],
                               np.array([0.1, 0.3, 0.7]) * float(np.float32(0.99)) * t1, atol=1e-7)
