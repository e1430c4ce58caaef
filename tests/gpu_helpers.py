"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and read
back every intermediate buffer, and compare images with the oracle's margin rule."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2507_04147_gb300 as a3fr

# Pixel tolerance and threshold-margin exemption.  A pixel whose oracle margin to the
# alpha >= 1/255 or T >= 1e-4 decision is below DELTA can legitimately flip between an
# fp32 libm exp and the GPU's ex2.approx (relative error ~2^-22 per evaluation,
# accumulated over a few hundred blends), so it is counted instead of bounded.
TOL = 2e-4
DELTA = 1e-5
MAX_EXEMPT_FRACTION = 2e-3


def run(scene_np, cams, gaze=None, fovea=None, full=False, capacity=0, keep_aux=True,
        out=None, tile=16, batch_mult=1, binning=a3fr.BINNING_AUTO):
    import torch
    s = a3fr.Scene.from_numpy(scene_np, instance_capacity=capacity, tile=tile)
    s.set_batch(batch_mult)
    s.set_binning(binning)
    for e, c in enumerate(cams):
        s.set_camera(e, c)
    s.keep_aux(keep_aux)
    if full:
        img = s.render_full(out=out)
    else:
        s.set_gaze(np.asarray(gaze, np.float32).reshape(len(cams), 2))
        img = s.render_foveated(fovea if fovea is not None else a3fr.Fovea(), out=out)
    torch.cuda.synchronize()
    eyes, n = len(cams), scene_np.n
    H, W = cams[0].height, cams[0].width
    r = dict(scene=s, img=img.cpu().numpy())
    r["rec"] = s.buffer(a3fr.BUF_RECORDS, torch.float32).cpu().numpy().reshape(eyes, n, 12)
    r["rect"] = s.buffer(a3fr.BUF_RECTS, torch.int16).cpu().numpy().view(np.uint16).reshape(eyes, n, 4)
    r["keys"] = s.buffer(a3fr.BUF_KEYS, torch.int64).cpu().numpy().view(np.uint64)
    r["vals"] = s.buffer(a3fr.BUF_VALUES, torch.int32).cpu().numpy().view(np.uint32)
    r["ranges"] = s.buffer(a3fr.BUF_RANGES, torch.int32).cpu().numpy().view(np.uint32).reshape(-1, 2)
    r["levels"] = s.buffer(a3fr.BUF_LEVELS, torch.uint8).cpu().numpy()
    if keep_aux:
        r["t_final"] = s.buffer(a3fr.BUF_T_FINAL, torch.float32).cpu().numpy().reshape(eyes, H, W)
        r["n_contrib"] = s.buffer(a3fr.BUF_N_CONTRIB, torch.int32).cpu().numpy().reshape(eyes, H, W)
        r["depth"] = s.buffer(a3fr.BUF_DEPTH, torch.float32).cpu().numpy().reshape(eyes, H, W)
    r["stats"] = s.stats()
    return r


def oracle_eye(scene_np, cam, tile=16):
    rec, rect, touched = oracle.preprocess(scene_np, cam, tile)
    keys, vals = oracle.sorted_keys(rec, rect, oracle.tiles(cam.width, tile))
    return rec, rect, touched, keys, vals


def strip_eye(keys, eye, n_tiles):
    return keys - np.uint64(eye * n_tiles << 32) if eye else keys


def compare_pixels(gpu_rgb, ref, tol=TOL, delta=DELTA):
    """gpu_rgb [P,3] vs oracle Image ref over the same P pixels."""
    err = np.abs(gpu_rgb.reshape(-1, 3).astype(np.float64) - ref.rgb.astype(np.float64)).max(axis=1)
    exempt = ref.margin < delta
    bad = (err > tol) & ~exempt
    info = dict(max_err=float(err[~exempt].max()) if (~exempt).any() else 0.0,
                exempt=int(exempt.sum()), pixels=int(err.size), bad=int(bad.sum()))
    assert not bad.any(), info
    assert exempt.mean() <= MAX_EXEMPT_FRACTION, info
    return info
