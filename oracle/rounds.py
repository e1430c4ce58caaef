"""Oracle of the incremental rendering rounds (Sec. 3.3, Algorithm 1) -- TEST INFRASTRUCTURE.

Only tests, the smoke check and the benchmark's CPU legs use this module.  It restates,
in fp32 NumPy, what each round of a frame renders:

* round 1 renders every tile at the peripheral level (the outermost layer's level);
* a round that sees a new prediction u_i (exit i) uses the layer radii
  ``r_{k,i} = max(0, r_{k,N} - E_i)`` around u_i                                (Eq. 3');
* a round that sees no new prediction grows the radii around the last prediction u_j by a
  step, up to ``r^max_{k,j} = r_{k,N} + E_j``                                  (Eq. 4), when
  speculative incremental rendering (SIR) is on, and renders nothing otherwise;
* every tile ends at the highest level any round gave it (labels are nested, so rendering
  a higher level only adds pixels).

``r_{k,N}`` is the fp32 square root of the fp32 square of ``f tan(theta_k + dtheta)`` -- the
same radius the oracle's level map uses -- and every radius update is an fp32 operation, so
the level decisions can be compared bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

import oracle


def final_radii(cam, fv) -> np.ndarray:
    """r_{k,N} for k = 0..2 (fp32): sqrt of the squared layer radius of Eq. 1."""
    return np.sqrt(oracle.layer_radii2(cam, fv)).astype(np.float32)


def level_map_r2(cam, tile: int, levels, r2, gaze) -> np.ndarray:
    """Tile levels for explicit squared radii (fp32 decisions as in or_level_map)."""
    tx_n, ty_n = oracle.tiles(cam.width, tile), oracle.tiles(cam.height, tile)
    out = np.zeros(tx_n * ty_n, dtype=np.uint8)
    g0, g1 = np.float32(gaze[0]), np.float32(gaze[1])
    n_layers = len(levels)
    for ty in range(ty_n):
        for tx in range(tx_n):
            x0, y0 = np.float32(tx * tile), np.float32(ty * tile)
            x1 = np.float32(min((tx + 1) * tile, cam.width) - 1)
            y1 = np.float32(min((ty + 1) * tile, cam.height) - 1)
            dx = max(max(x0 - g0, g0 - x1), np.float32(0.0))
            dy = max(max(y0 - g1, g1 - y1), np.float32(0.0))
            d2 = np.float32(dx * dx) + np.float32(dy * dy)
            layer = n_layers - 1
            for k in range(n_layers - 1):
                if d2 <= np.float32(r2[k]):
                    layer = k
                    break
            out[ty * tx_n + tx] = levels[layer]
    return out


class FrameRounds:
    """Replays the device round logic for one eye."""

    def __init__(self, cam, tile: int, fv, expected_px, sir: bool, step_px: float):
        self.cam, self.tile = cam, tile
        self.levels = [int(fv.level[k]) for k in range(fv.n_layers)]
        self.rf = final_radii(cam, fv)
        self.expected = np.asarray(expected_px, dtype=np.float32)
        self.n_exits = len(expected_px)
        self.sir, self.step = sir, np.float32(step_px)
        n_tiles = oracle.tiles(cam.width, tile) * oracle.tiles(cam.height, tile)
        self.level = np.full(n_tiles, self.levels[-1], dtype=np.uint8)   # round 1
        self.last_exit = 0
        self.gaze = np.zeros(2, dtype=np.float32)
        self.r = np.zeros(3, dtype=np.float32)
        self.complete = False
        self.rounds = 0

    def round(self, exit_index: int, gaze) -> np.ndarray:
        """One round that finds prediction (exit_index, gaze) in the mailbox (exit 0: none)."""
        active = False
        if 0 < exit_index <= self.n_exits and exit_index > self.last_exit:
            self.last_exit = exit_index
            self.gaze = np.asarray(gaze, dtype=np.float32)
            e = self.expected[exit_index - 1]
            self.r = np.maximum(np.float32(0.0), self.rf - e).astype(np.float32)      # Eq. 3'
            active = True
        elif self.sir and self.last_exit > 0 and not self.complete:
            e = self.expected[self.last_exit - 1]
            self.r = np.minimum(self.r + self.step, self.rf + e).astype(np.float32)   # Eq. 4
            active = True
        if active:
            r2 = (self.r * self.r).astype(np.float32)
            target = level_map_r2(self.cam, self.tile, self.levels, r2, self.gaze)
            self.level = np.maximum(self.level, target)
            self.rounds += 1
        if self.last_exit == self.n_exits:
            self.complete = True
        return self.level


def expected_distance_gaussian(sigma_i, sigma_n) -> float:
    """E[dist(u_i, u_N)] for independent zero-mean Gaussian errors of std sigma_i, sigma_n
    per axis (any unit): the mean norm of a 2-D Gaussian with per-axis variance
    sigma_i^2 + sigma_n^2, by numerical integration of the Rayleigh-type density."""
    sx = math.hypot(sigma_i[0], sigma_n[0])
    sy = math.hypot(sigma_i[1], sigma_n[1])
    if sx == 0 and sy == 0:
        return 0.0
    # E|X| for X ~ N(0, diag(sx^2, sy^2)) = integral over angle of the radial mean
    th = np.linspace(0.0, 2.0 * math.pi, 20001)[:-1]
    s2 = 1.0 / (np.cos(th) ** 2 / sx ** 2 + np.sin(th) ** 2 / sy ** 2)
    # radial part: int_0^inf r^2 exp(-r^2 / (2 s2)) dr / (2 pi sx sy) = sqrt(pi/2) s2^1.5 / (2 pi sx sy)
    return float(np.mean(np.sqrt(np.pi / 2.0) * s2 ** 1.5 / (sx * sy)))
