"""Incremental-rendering rounds: pins of the schedule oracle (Eq. 3, Eq. 3', Eq. 4) and of
the offline profiling, without a GPU."""
import json
import math
import os

import numpy as np

import oracle
from oracle import rounds as orounds
from paper_2507_04147_gb300 import rounds as prounds
from paper_2507_04147_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_table2_constants_match_the_golden_fixture():
    g = json.load(open(GOLDEN))
    np.testing.assert_allclose(np.array(prounds.TABLE2_SIGMA_DEG), np.array(g["vit_exit_sigma_deg"]["value"]))
    np.testing.assert_allclose(prounds.TABLE2_CUM_LATENCY_MS, g["vit_exit_latency_ms"]["cumulative"][1:])


def test_eq3_radius_keeps_the_early_region_inside_the_final_one():
    rng = np.random.default_rng(0)
    for _ in range(200):
        u_i, u_n = rng.uniform(0, 500, 2), rng.uniform(0, 500, 2)
        r_n = rng.uniform(10, 300)
        r_i = max(0.0, r_n - np.linalg.norm(u_i - u_n))            # Eq. 3 at equality
        if r_i == 0.0:
            continue                                               # an empty region
        ang = rng.uniform(0, 2 * np.pi, 500)
        rad = r_i * np.sqrt(rng.uniform(0, 1, 500))
        pts = u_i + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
        assert np.all(np.linalg.norm(pts - u_n, axis=1) <= r_n + 1e-9)


def test_eq4_max_radius_covers_the_final_region():
    rng = np.random.default_rng(1)
    for _ in range(200):
        u_j, u_n = rng.uniform(0, 500, 2), rng.uniform(0, 500, 2)
        r_n = rng.uniform(10, 300)
        r_max = r_n + np.linalg.norm(u_j - u_n)                    # Eq. 4
        ang = rng.uniform(0, 2 * np.pi, 500)
        rad = r_n * np.sqrt(rng.uniform(0, 1, 500))
        pts = u_n + np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
        assert np.all(np.linalg.norm(pts - u_j, axis=1) <= r_max + 1e-9)


def test_expected_distance_closed_form_and_monte_carlo():
    # isotropic errors: the difference is isotropic with variance s_i^2 + s_n^2 per axis and
    # its mean norm is the Rayleigh mean sqrt(pi/2) * sqrt(s_i^2 + s_n^2)
    e = orounds.expected_distance_gaussian((3.0, 3.0), (4.0, 4.0))
    assert abs(e - math.sqrt(math.pi / 2) * 5.0) < 1e-6
    f = 640.0
    mc = prounds.profile_expected_distances(f_px=f, samples=400_000)
    sig = [[f * math.tan(math.radians(s)) for s in pair] for pair in prounds.TABLE2_SIGMA_DEG]
    for i in range(5):
        ref = orounds.expected_distance_gaussian(sig[i], sig[-1])
        assert abs(mc[i] - ref) / ref < 0.01, (i, mc[i], ref)
    assert mc[-1] == 0.0
    assert np.all(np.diff(mc) < 0)           # later exits are closer to the final prediction


def test_schedule_oracle_sir_growth_and_completion():
    cam = synth.pinhole_camera(256, 256)
    fv = oracle.fovea()
    expected = [40.0, 20.0, 0.0]
    fr = orounds.FrameRounds(cam, 16, fv, expected, sir=True, step_px=8.0)
    rf = orounds.final_radii(cam, fv)
    assert np.all(fr.level == 1)
    fr.round(1, (100.0, 120.0))
    np.testing.assert_array_equal(fr.r, np.maximum(np.float32(0), rf - np.float32(40.0)))
    prev = fr.r.copy()
    for _ in range(20):                      # no new prediction: SIR grows up to rf + E_1
        fr.round(0, (0.0, 0.0))
        assert np.all(fr.r >= prev)
        assert np.all(fr.r <= rf + np.float32(40.0))
        prev = fr.r.copy()
    np.testing.assert_array_equal(fr.r, (rf + np.float32(40.0)).astype(np.float32))
    assert not fr.complete
    fr.round(3, (110.0, 118.0))
    np.testing.assert_array_equal(fr.r, rf)          # E_N = 0: the final radii
    assert fr.complete
    # the frame's levels cover the plain foveated levels of the final gaze
    plain = oracle.level_map(cam, 16, fv, (110.0, 118.0))
    assert np.all(fr.level >= plain)


def test_schedule_without_sir_renders_nothing_between_predictions():
    cam = synth.pinhole_camera(128, 128)
    fr = orounds.FrameRounds(cam, 16, oracle.fovea(), [10.0, 0.0], sir=False, step_px=8.0)
    fr.round(1, (64.0, 64.0))
    lv = fr.level.copy()
    r = fr.r.copy()
    fr.round(0, (0.0, 0.0))
    assert np.array_equal(fr.level, lv) and np.array_equal(fr.r, r) and fr.rounds == 1


def test_synthetic_predictions_follow_the_exit_errors():
    p = prounds.synthetic_predictions([[640.0, 640.0], [640.0, 640.0]], seed=3)
    assert p.shape == (6, 2, 2)
    assert np.array_equal(p[:, 0], p[:, 1])          # same angular error for both eyes
