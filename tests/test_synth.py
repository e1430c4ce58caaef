"""Seeded input generators: determinism, shapes and the stated distributions."""
import math

import numpy as np

from paper_2507_04147_gb300 import synth


def test_uniform_scene_recipe():
    a = synth.uniform_scene(20000, 0, seed=0)
    b = synth.uniform_scene(20000, 0, seed=0)
    assert np.array_equal(a.means, b.means) and np.array_equal(a.sh, b.sh)
    assert a.means.dtype == np.float32 and a.sh.shape == (20000, 1, 3)
    assert a.means[:, :2].min() >= -1 and a.means[:, :2].max() <= 1
    assert a.means[:, 2].min() >= 2 and a.means[:, 2].max() <= 6
    assert abs(a.log_scales.mean() + 4) < 0.02 and abs(a.log_scales.std() - 0.5) < 0.02
    assert abs(a.opacity_logits.std() - 1.5) < 0.05
    np.testing.assert_allclose(np.linalg.norm(a.quats, axis=1), 1, atol=1e-6)
    base = a.sh[:, 0, :] * (0.5 / math.sqrt(math.pi)) + 0.5
    assert base.min() >= -1e-6 and base.max() <= 1 + 1e-6
    c = synth.uniform_scene(1000, 3, seed=1)
    assert c.sh.shape == (1000, 16, 3) and abs(c.sh[:, 1:].std() - 0.2) < 0.01


def test_clustered_scene_recipe():
    s = synth.clustered_scene(50000, 3, seed=0)
    assert s.n == 50000 and s.sh.shape == (50000, 16, 3)
    op = 1 / (1 + np.exp(-s.opacity_logits.astype(np.float64)))
    assert abs(op.mean() - 0.5) < 0.01 and ((op < 0.1) | (op > 0.9)).mean() > 0.35   # Beta(0.5, 0.5)


def test_stereo_cameras_and_gaze():
    cams = synth.stereo_cameras(1280, 1280, yaw_deg=1.0)
    np.testing.assert_allclose(np.linalg.norm(cams[0].center() - cams[1].center()), 0.063, rtol=1e-6)
    assert cams[0].fx == 640.0 and cams[0].cx == 639.5
    traj = synth.gaze_trajectory(240)
    assert traj.shape == (240, 2)
    assert np.linalg.norm(traj, axis=1).max() <= 35.0 + 1e-9
    steps = np.linalg.norm(np.diff(traj, axis=0), axis=1)
    assert (steps == 0).mean() > 0.5          # fixations dominate
    assert steps.max() * 90 > 100             # saccades exceed 100 deg/s
    g = synth.gaze_pixels(np.zeros(2), cams[0])
    np.testing.assert_allclose(g, [639.5, 639.5])
