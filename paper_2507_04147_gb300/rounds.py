"""Host side of incremental rendering (Sec. 3.3, Algorithm 1).

* ``profile_expected_distances`` is the offline profiling step of Eq. 3': the expected
  distance between an early prediction u_i and the final one u_N, estimated by Monte Carlo
  over a tracker error model (the paper averages over OpenEDS; here the per-exit error
  spread of Table 2 stands in for the data).
* ``run_frame`` drives one frame the way Algorithm 1's two processes interleave: a tracker
  thread posts u_1..u_N into the scene's mailbox at their (scaled) exit times while the host
  keeps launching rounds; each round reads the newest prediction when it runs on the GPU.
  Without speculative rounds the host waits for the next prediction before each round.

Every step of a round runs in the CUDA library (``a3fr_render_round``); this module only
schedules calls and measures time.
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

# Table 2, A3FR-ViT without pruning: gaze error (sigma_x, sigma_y) in degrees per exit and
# cumulative latency in ms per exit (the embedding's 1.00 ms precedes exit 1).
TABLE2_SIGMA_DEG = ((8.40, 9.33), (6.08, 7.05), (4.50, 4.46), (3.58, 3.38), (2.97, 2.85),
                    (2.05, 2.16))
TABLE2_CUM_LATENCY_MS = (5.11, 9.45, 13.91, 18.31, 22.21, 26.28)
# Table 1: 3DGS rendering latency at 1080p on the paper's edge GPU (the time scale the
# tracker latencies are compared with).
TABLE1_RENDER_1080P_MS = 37.78


def profile_expected_distances(sigma_deg=TABLE2_SIGMA_DEG, f_px: float = 640.0,
                               samples: int = 200_000, seed: int = 0) -> np.ndarray:
    """E[dist(u_i, u_N)] in pixels per exit i (Eq. 3'), last entry 0.

    Errors of the exits are modelled as independent zero-mean Gaussians with per-axis
    standard deviations sigma_deg (degrees), mapped to pixels at the image centre
    (f tan(sigma)); the expectation is a Monte Carlo mean.
    """
    rng = np.random.default_rng(seed)
    sig = np.array([[f_px * math.tan(math.radians(s)) for s in pair] for pair in sigma_deg])
    n = len(sig)
    err = rng.normal(size=(n, samples, 2)) * sig[:, None, :]
    out = np.linalg.norm(err - err[-1][None], axis=2).mean(axis=1)
    out[-1] = 0.0
    return out.astype(np.float32)


def synthetic_predictions(true_gaze_px, sigma_deg=TABLE2_SIGMA_DEG, f_px: float = 640.0,
                          seed: int = 0) -> np.ndarray:
    """Early-exit predictions u_i = g + e_i (pixels, [N, eyes, 2]) for the true gaze g."""
    rng = np.random.default_rng(seed)
    g = np.asarray(true_gaze_px, dtype=np.float64).reshape(-1, 2)
    sig = np.array([[f_px * math.tan(math.radians(s)) for s in pair] for pair in sigma_deg])
    e = rng.normal(size=(len(sig), 2)) * sig          # the same angular error for both eyes
    return (g[None, :, :] + e[:, None, :]).astype(np.float32)


def _busy_wait_until(t: float):
    while True:
        d = t - time.perf_counter()
        if d <= 0:
            return
        if d > 2e-4:
            time.sleep(d - 1e-4)


def run_frame(scene, fovea, rounds, out, predictions, exit_times_s, stream, sir: bool = True,
              max_rounds: int = 64, load=None) -> dict:
    """Render one frame in rounds while a tracker thread posts ``predictions``.

    exit_times_s[i] is when prediction i+1 becomes available, relative to the frame start;
    ``load(t)`` (optional) returns a slow-down factor for the tracker at time t (CPU load
    injection).  Returns the frame latency (start -> completion of the round that used the
    final prediction), the rounds run and the exits each round consumed.
    """
    import torch

    n = len(predictions)
    posted = threading.Event()
    t0 = time.perf_counter()

    def tracker():
        t_prev, t_now = 0.0, t0
        for i in range(n):
            dt = exit_times_s[i] - t_prev
            t_prev = exit_times_s[i]
            if load is not None:
                dt *= load(t_now - t0)
            t_now += dt
            _busy_wait_until(t_now)
            scene.post_prediction(i + 1, predictions[i])
            posted.set()

    scene.begin_frame(fovea, rounds, out=out, stream=stream)
    th = threading.Thread(target=tracker, daemon=True)
    th.start()
    consumed = []
    t_done = None
    for _ in range(max_rounds):
        if not sir:
            # without speculative rounds the GPU waits for the next prediction
            last = consumed[-1] if consumed else 0
            while scene.round_status()["exit_consumed"] == last and not _newer_posted(posted):
                time.sleep(0)
            posted.clear()
        scene.render_round(out, stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        ev.synchronize()
        st = scene.round_status()
        consumed.append(st["exit_consumed"])
        if st["complete"]:
            t_done = time.perf_counter()
            break
    th.join()
    return {"latency_s": (t_done - t0) if t_done else None, "rounds": len(consumed),
            "exits": consumed}


def _newer_posted(ev: threading.Event) -> bool:
    return ev.is_set()
