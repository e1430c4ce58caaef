"""Pins of the fp64 gradient oracle (oracle/grad.py) -- CPU only.

* its forward equals the C oracle's fp32 image (same decisions, fp64 arithmetic);
* its autograd gradient equals fp64 central finite differences (h = 1e-4) of its own
  forward for every parameter group, on 64 Gaussians at 32x32;
* a single Gaussian's gradients equal their closed forms.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import grad as og
from paper_2507_04147_gb300 import synth


def small_scene(n=64, seed=7, degree=3):
    s = synth.uniform_scene(n, degree, seed=seed, log_scale_mean=-1.8, log_scale_std=0.3)
    return s


def test_forward_matches_c_oracle():
    s = small_scene()
    cam = synth.pinhole_camera(32, 32)
    ref = oracle.render(*oracle.preprocess(s, cam, 16)[:2], cam, 16)
    L, C, info = og.loss(og.params_f64(s), s, cam, 16, np.zeros((32 * 32, 3)))
    ok = (ref.margin >= 1e-5) & (info["margin"] >= 1e-4)
    assert ok.mean() > 0.95
    err = np.abs(C.detach().numpy() - ref.rgb.astype(np.float64)).max(axis=1)
    assert err[ok].max() < 2e-5, err[ok].max()
    assert np.abs(info["t_final"] - ref.t_final)[ok].max() < 2e-5


def test_autograd_matches_central_differences():
    s = small_scene()
    cam = synth.pinhole_camera(32, 32)
    rng = np.random.default_rng(3)
    w = rng.normal(size=(32 * 32, 3))
    g = og.gradient(s, cam, 16, w)
    vis = og.Visibility(s, cam, 16)
    # Gaussians that reach some pixel: the ones with a non-zero opacity gradient
    active = np.nonzero(np.abs(g["opacity_logits"]) > 1e-8)[0]
    assert len(active) > 20
    picks = rng.choice(active, size=8, replace=False)
    checked = 0
    for name, comps in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 0),
                        ("sh", None)):
        for i in picks:
            idxs = [(i,)] if comps == 0 else ([(i, k) for k in range(comps)] if comps else
                                              [(i, k, c) for k in (0, 1, 5, 15) for c in (0, 2)])
            for idx in idxs:
                fd, flipped = og.finite_difference(s, cam, 16, w, name, idx, h=1e-4, vis=vis)
                if flipped:
                    continue
                ad = g[name][idx]
                scale = max(1e-3, np.abs(g[name]).max())
                assert abs(ad - fd) <= 1e-5 * scale + 1e-4 * abs(fd), (name, idx, ad, fd)
                checked += 1
    assert checked > 100


def test_single_gaussian_closed_forms():
    s = synth.uniform_scene(1, 0, seed=2, log_scale_mean=-1.5, log_scale_std=0.0)
    s.means[0] = [0.05, -0.03, 3.0]
    s.opacity_logits[0] = 0.3
    cam = synth.pinhole_camera(16, 16)
    pix = np.array([[8, 7]])
    w = np.array([[1.0, 0.0, 0.0]])
    g = og.gradient(s, cam, 16, w, pixels=pix)
    params = og.params_f64(s)
    proj = og.project(params, cam, 0)
    dx = float(proj["u"][0]) - 8.0
    dy = float(proj["v"][0]) - 7.0
    power = -0.5 * (float(proj["ca"][0]) * dx * dx + float(proj["cc"][0]) * dy * dy) \
        - float(proj["cb"][0]) * dx * dy
    o = 1.0 / (1.0 + math.exp(-float(s.opacity_logits[0])))
    alpha = o * math.exp(power)
    assert 1 / 255 < alpha < 0.99
    red = float(proj["rgb"][0, 0])
    assert g["rgb"][0, 0] == pytest.approx(red * alpha, rel=1e-12)
    # dC/dlogit = rgb exp(power) o (1 - o); dC/d(DC coefficient) = Y_00 alpha
    assert g["opacity_logits"][0] == pytest.approx(red * math.exp(power) * o * (1 - o), rel=1e-10)
    assert g["sh"][0, 0, 0] == pytest.approx(0.5 * math.sqrt(1 / math.pi) * alpha, rel=1e-10)
    assert g["sh"][0, 0, 1] == 0.0
