"""A3FR foveated 3D Gaussian Splatting forward rasterizer for GB300 (sm_103a).

Python binding of libA3FR.so.  The functions below carry the names of the C ABI
(``include/a3fr.h``) and only marshal arguments: PyTorch supplies device memory and
streams, every step of a render runs in the library's CUDA kernels.

    scene = Scene(means, log_scales, quats, opacity_logits, sh)   # CUDA fp32 tensors
    scene.set_camera(0, cam_left); scene.set_camera(1, cam_right)
    scene.set_gaze([[gx0, gy0], [gx1, gy1]], side_stream)
    img = scene.render_foveated(Fovea())     # [eyes, H, W, 3] on the current stream
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import A3FRError, BUF_DEPTH, BUF_KEYS, BUF_LEVELS, BUF_N_CONTRIB, BUF_RANGES, BUF_RECORDS, \
    BUF_RECTS, BUF_T_FINAL, BUF_VALUES, STATUS_CAPACITY, STATUS_TIMEOUT

__all__ = ["Scene", "Fovea", "A3FRError", "camera_struct", "create_scene", "destroy_scene",
           "set_camera", "set_gaze", "render_foveated", "render_full", "get_stats",
           "set_keep_aux", "set_graph_mode", "set_stage_timing", "get_stage_times", "copy_buffer", "sort_pairs", "sort_pairs_workspace_bytes",
           "sort_pairs_noalloc", "Rounds", "begin_frame", "post_prediction", "render_round", "stall_mailbox",
           "get_round_status", "run_frame",
           "error_string"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return t.data_ptr()


FILL_INHERIT, FILL_INTERPOLATE = 0, 1
BINNING_AUTO, BINNING_DIRECT, BINNING_SORTED = 0, 1, 2


def Fovea(theta_deg=(18.0, 36.0), dtheta_deg: float = 0.0, levels=(4, 2, 1),
          fill: int = FILL_INHERIT, count_frac: float = 0.0) -> _lib.Fovea:
    """Foveation layers (Eq. 1 radii from eccentricity angles; Sec. 3.4 levels and fill;
    Sec. 3.6 count-based tile levels when count_frac > 0)."""
    f = _lib.Fovea()
    f.n_layers = len(levels)
    for k, t in enumerate(theta_deg):
        f.theta_deg[k] = float(t)
    f.dtheta_deg = float(dtheta_deg)
    for k, lv in enumerate(levels):
        f.level[k] = int(lv)
    f.fill = int(fill)
    f.count_frac = float(count_frac)
    return f


def camera_struct(cam) -> _lib.Camera:
    """Camera (any object with width/height/fx/fy/cx/cy/znear/world_to_cam) -> C struct."""
    c = _lib.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy, c.znear = (float(cam.fx), float(cam.fy), float(cam.cx),
                                       float(cam.cy), float(cam.znear))
    w = np.ascontiguousarray(cam.world_to_cam, dtype=np.float32).reshape(12)
    for i in range(12):
        c.world_to_cam[i] = float(w[i])
    return c


# ------------------------------------------------------------ C-ABI names
def create_scene(desc: _lib.SceneDesc, instance_capacity: int = 0) -> int:
    lib = _lib.load()
    out = ctypes.c_void_p()
    _lib.check(lib.a3fr_create_scene(ctypes.byref(desc), instance_capacity, ctypes.byref(out)),
               "a3fr_create_scene")
    return out.value


def destroy_scene(handle: int) -> None:
    _lib.check(_lib.load().a3fr_destroy_scene(handle), "a3fr_destroy_scene")


def set_camera(handle: int, eye: int, cam: _lib.Camera) -> None:
    _lib.check(_lib.load().a3fr_set_camera(handle, eye, ctypes.byref(cam)), "a3fr_set_camera")


def set_gaze(handle: int, gaze_px, side_stream=None) -> None:
    g = np.ascontiguousarray(np.asarray(gaze_px, dtype=np.float32).reshape(-1))
    _lib.check(_lib.load().a3fr_set_gaze(handle, g.ctypes.data, _stream_ptr(side_stream)),
               "a3fr_set_gaze")


def render_foveated(handle: int, fovea: _lib.Fovea, out_rgb, stream=None) -> None:
    _lib.check(_lib.load().a3fr_render_foveated(handle, ctypes.byref(fovea), _ptr(out_rgb),
                                                _stream_ptr(stream)), "a3fr_render_foveated")


def render_full(handle: int, out_rgb, stream=None) -> None:
    _lib.check(_lib.load().a3fr_render_full(handle, _ptr(out_rgb), _stream_ptr(stream)),
               "a3fr_render_full")


def backward(handle: int, dl_drgb, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh,
             stream=None) -> None:
    """Gradients of sum(dl_drgb * image) of the last render (keep_aux on) into the d_* CUDA
    tensors (overwritten; layouts of the scene arrays)."""
    g = _lib.Grads()
    g.means, g.log_scales, g.quats = _ptr(d_means), _ptr(d_log_scales), _ptr(d_quats)
    g.opacity_logits, g.sh = _ptr(d_opacity_logits), _ptr(d_sh)
    _lib.check(_lib.load().a3fr_backward(handle, _ptr(dl_drgb), ctypes.byref(g), _stream_ptr(stream)),
               "a3fr_backward")


def tc_tile_gemm(a_bf16, b_bf16, d, variant: int = 0, stream=None) -> None:
    """D[128][n] = A[128][k] B[n][k]^T on the tensor cores (bf16 tensors in, fp32 out)."""
    _lib.check(_lib.load().a3fr_tc_tile_gemm(_ptr(a_bf16), _ptr(b_bf16), _ptr(d), b_bf16.shape[0],
                                             a_bf16.shape[1], variant, _stream_ptr(stream)),
               "a3fr_tc_tile_gemm")


def get_stats(handle: int, reset: bool = False) -> dict:
    st = _lib.Stats()
    _lib.check(_lib.load().a3fr_get_stats(handle, ctypes.byref(st), int(reset)), "a3fr_get_stats")
    return {"status": st.status, "n_eyes": st.n_eyes, "instances": st.instances,
            "instances_eye": [st.instances_eye[0], st.instances_eye[1]],
            "capacity": st.capacity, "evaluations": st.evaluations,
            "records_staged": st.records_staged, "renders": st.renders,
            "kernel_launches": st.kernel_launches, "contributions": st.contributions}


def set_stage_timing(handle: int, ring: int) -> None:
    _lib.check(_lib.load().a3fr_set_stage_timing(handle, ring), "a3fr_set_stage_timing")


def get_stage_times(handle: int, max_renders: int) -> np.ndarray:
    """Stage durations (ms) of the last timed renders, [k, 6] oldest first."""
    ms = np.zeros((max_renders, len(_lib.STAGES)), dtype=np.float32)
    k = ctypes.c_int(0)
    _lib.check(_lib.load().a3fr_get_stage_times(handle, max_renders, ms.ctypes.data,
                                                ctypes.byref(k)), "a3fr_get_stage_times")
    return ms[:k.value]


def set_graph_mode(handle: int, on: bool) -> None:
    _lib.check(_lib.load().a3fr_set_graph_mode(handle, int(on)), "a3fr_set_graph_mode")


def set_keep_aux(handle: int, keep: bool) -> None:
    _lib.check(_lib.load().a3fr_set_keep_aux(handle, int(keep)), "a3fr_set_keep_aux")


def copy_buffer(handle: int, which: int, dst=None, stream=None) -> int:
    """Copy an internal buffer into the CUDA tensor dst; returns the buffer size in bytes."""
    lib = _lib.load()
    needed = ctypes.c_size_t(0)
    if dst is None:
        _lib.check(lib.a3fr_copy_buffer(handle, which, None, 0, ctypes.byref(needed), None),
                   "a3fr_copy_buffer")
        return needed.value
    nbytes = dst.numel() * dst.element_size()
    _lib.check(lib.a3fr_copy_buffer(handle, which, _ptr(dst), nbytes, ctypes.byref(needed),
                                    _stream_ptr(stream)), "a3fr_copy_buffer")
    return needed.value


def sort_pairs_workspace_bytes(n: int) -> int:
    return int(_lib.load().a3fr_sort_pairs_workspace_bytes(n))


def sort_pairs(keys, vals, keys_alt, vals_alt, key_bits: int, workspace, stream=None) -> None:
    """Stable radix sort of (uint64 key, uint32 value) CUDA tensors by the low key_bits bits."""
    n = keys.numel()
    _lib.check(_lib.load().a3fr_sort_pairs(_ptr(keys), _ptr(vals), _ptr(keys_alt), _ptr(vals_alt),
                                           n, key_bits, _ptr(workspace), workspace.numel(),
                                           _stream_ptr(stream)), "a3fr_sort_pairs")


def sort_pairs_noalloc(keys, vals, key_bits: int, stream=None) -> None:
    """The same sort for callers that cannot allocate: scratch comes from a fixed device
    array inside the library (at most NOALLOC_MAX_PAIRS pairs; overlapping calls race)."""
    _lib.check(_lib.load().a3fr_sort_pairs_noalloc(_ptr(keys), _ptr(vals), keys.numel(), key_bits,
                                                   _stream_ptr(stream)), "a3fr_sort_pairs_noalloc")


def Rounds(expected_dist_px, sir: bool = True, sir_step_px: float = 8.0) -> _lib.Rounds:
    """Round schedule: E[dist(u_i, u_N)] per exit (pixels, last = 0), SIR on/off and step."""
    r = _lib.Rounds()
    r.n_exits = len(expected_dist_px)
    r.sir = int(bool(sir))
    for i, e in enumerate(expected_dist_px):
        r.expected_dist_px[i] = float(e)
    r.sir_step_px = float(sir_step_px)
    return r


def begin_frame(handle: int, fovea: _lib.Fovea, rounds: _lib.Rounds, out_rgb, stream=None) -> None:
    _lib.check(_lib.load().a3fr_begin_frame(handle, ctypes.byref(fovea), ctypes.byref(rounds),
                                            _ptr(out_rgb), _stream_ptr(stream)), "a3fr_begin_frame")


def post_prediction(handle: int, exit_index: int, gaze_px) -> None:
    g = np.ascontiguousarray(np.asarray(gaze_px, dtype=np.float32).reshape(-1))
    _lib.check(_lib.load().a3fr_post_prediction(handle, exit_index, g.ctypes.data),
               "a3fr_post_prediction")


def render_round(handle: int, out_rgb, stream=None) -> None:
    _lib.check(_lib.load().a3fr_render_round(handle, _ptr(out_rgb), _stream_ptr(stream)),
               "a3fr_render_round")


def stall_mailbox(handle: int, stall: bool) -> None:
    _lib.check(_lib.load().a3fr_stall_mailbox(handle, int(bool(stall))), "a3fr_stall_mailbox")


def get_round_status(handle: int) -> dict:
    st = _lib.RoundStatus()
    _lib.check(_lib.load().a3fr_get_round_status(handle, ctypes.byref(st)), "a3fr_get_round_status")
    return {"exit_consumed": st.exit_consumed, "complete": st.complete, "rounds": st.rounds,
            "radius_px": [st.radius_px[0], st.radius_px[1], st.radius_px[2]]}


def run_frame(handle: int, fovea, rounds, predictions, exit_time_us, out_rgb, mode: int = 0,
              load_period_us: float = 0.0, load_factor: float = 1.0, max_rounds: int = 64,
              stream=None) -> dict:
    """One frame of Algorithm 1 in native code (see a3fr_run_frame)."""
    pred = np.ascontiguousarray(np.asarray(predictions, dtype=np.float32))
    times = np.ascontiguousarray(np.asarray(exit_time_us, dtype=np.float64))
    d = _lib.FrameDriver()
    d.mode, d.n_exits = int(mode), int(len(times))
    d.predictions, d.exit_time_us = pred.ctypes.data, times.ctypes.data
    d.load_period_us, d.load_factor, d.max_rounds = float(load_period_us), float(load_factor), int(max_rounds)
    r = _lib.FrameResult()
    _lib.check(_lib.load().a3fr_run_frame(handle, ctypes.byref(fovea), ctypes.byref(rounds),
                                          ctypes.byref(d), _ptr(out_rgb), _stream_ptr(stream),
                                          ctypes.byref(r)), "a3fr_run_frame")
    k = min(r.rounds, 16)
    return {"latency_us": r.latency_us, "tracker_end_us": r.tracker_end_us, "rounds": r.rounds,
            "exits": list(r.exit_per_round[:k]), "round_end_us": list(r.round_end_us[:k])}


def error_string(code: int) -> str:
    return _lib.load().a3fr_error_string(code).decode()


# ------------------------------------------------------------ convenience object
class Scene:
    """Owns a library scene over CUDA fp32 tensors (kept alive by this object)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, sh_degree: int | None = None,
                 instance_capacity: int = 0, tile: int = 16):
        torch = _torch()
        ts = [means, log_scales, quats, opacity_logits, sh]
        for t in ts:
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("scene tensors must be contiguous CUDA float32")
        self._tensors = ts
        n = means.shape[0]
        if sh_degree is None:
            sh_degree = int(round((sh.shape[1]) ** 0.5)) - 1
        self.n, self.sh_degree = n, sh_degree
        d = _lib.SceneDesc()
        d.n, d.sh_degree, d.tile, d.reserved = n, sh_degree, tile, 0
        d.means, d.log_scales, d.quats = _ptr(means), _ptr(log_scales), _ptr(quats)
        d.opacity_logits, d.sh = _ptr(opacity_logits), _ptr(sh)
        self.handle = create_scene(d, instance_capacity)
        self.cams = {}
        self.tile = tile

    @classmethod
    def from_numpy(cls, scene, device="cuda", **kw) -> "Scene":
        torch = _torch()
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        return cls(f(scene.means), f(scene.log_scales), f(scene.quats), f(scene.opacity_logits),
                   f(scene.sh), scene.sh_degree, **kw)

    def close(self):
        if getattr(self, "handle", None):
            destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_eyes(self) -> int:
        return 2 if 1 in self.cams else 1

    def set_camera(self, eye: int, cam):
        self.cams[eye] = cam
        set_camera(self.handle, eye, camera_struct(cam))

    def set_gaze(self, gaze_px, side_stream=None):
        set_gaze(self.handle, gaze_px, side_stream)

    def _out(self, out):
        if out is not None:
            return out
        c = self.cams[0]
        return _torch().empty((self.n_eyes, c.height, c.width, 3), device="cuda",
                              dtype=_torch().float32)

    def render_foveated(self, fovea=None, out=None, stream=None):
        out = self._out(out)
        render_foveated(self.handle, fovea if fovea is not None else Fovea(), out, stream)
        return out

    def render_full(self, out=None, stream=None):
        out = self._out(out)
        render_full(self.handle, out, stream)
        return out

    def begin_frame(self, fovea, rounds, out=None, stream=None):
        out = self._out(out)
        begin_frame(self.handle, fovea, rounds, out, stream)
        return out

    def post_prediction(self, exit_index: int, gaze_px):
        post_prediction(self.handle, exit_index, gaze_px)

    def render_round(self, out, stream=None):
        render_round(self.handle, out, stream)
        return out

    def round_status(self) -> dict:
        return get_round_status(self.handle)

    def stall_mailbox(self, stall: bool = True):
        stall_mailbox(self.handle, stall)

    def stats(self, reset: bool = False) -> dict:
        return get_stats(self.handle, reset)

    def stage_timing(self, ring: int):
        set_stage_timing(self.handle, ring)

    def stage_times(self, max_renders: int) -> np.ndarray:
        return get_stage_times(self.handle, max_renders)

    def graph_mode(self, on: bool = True):
        set_graph_mode(self.handle, on)

    def set_tile(self, tile: int):
        _lib.check(_lib.load().a3fr_set_tile(self.handle, int(tile)), "a3fr_set_tile")
        self.tile = int(tile)

    def set_batch(self, batch_mult: int):
        _lib.check(_lib.load().a3fr_set_batch(self.handle, int(batch_mult)), "a3fr_set_batch")

    def set_binning(self, mode: int):
        """BINNING_AUTO, BINNING_DIRECT or BINNING_SORTED (the same tile lists either way)."""
        _lib.check(_lib.load().a3fr_set_binning(self.handle, int(mode)), "a3fr_set_binning")

    def autotune(self, fovea=None, out=None, timed_renders: int = 5, stream=None) -> dict:
        """Times every (tile, batch) configuration on the current view and keeps the fastest."""
        out = self._out(out)
        r = _lib.TuneResult()
        _lib.check(_lib.load().a3fr_autotune(self.handle, ctypes.byref(fovea if fovea is not None else Fovea()),
                                             _ptr(out), int(timed_renders), _stream_ptr(stream),
                                             ctypes.byref(r)), "a3fr_autotune")
        self.tile = int(r.tile)
        return {"tile": r.tile, "batch_mult": r.batch_mult,
                "ms": {(t, m): r.ms[i][j] for i, t in enumerate((16, 32)) for j, m in enumerate((1, 2))}}

    def backward(self, dl_drgb, stream=None) -> dict:
        """Gradients of sum(dl_drgb * image) of the last render (needs keep_aux) as new
        CUDA tensors shaped like the scene arrays."""
        torch = _torch()
        if not (dl_drgb.is_cuda and dl_drgb.dtype == torch.float32 and dl_drgb.is_contiguous()):
            raise ValueError("dl_drgb must be a contiguous CUDA float32 tensor")
        names = ("means", "log_scales", "quats", "opacity_logits", "sh")
        grads = {k: torch.empty_like(t) for k, t in zip(names, self._tensors)}
        backward(self.handle, dl_drgb, *[grads[k] for k in names], stream=stream)
        return grads

    def keep_aux(self, keep: bool = True):
        set_keep_aux(self.handle, keep)

    def buffer(self, which: int, dtype, shape=None, stream=None):
        """Copy of an internal buffer of the last render as a CUDA tensor."""
        torch = _torch()
        nbytes = copy_buffer(self.handle, which)
        itemsize = torch.empty((), dtype=dtype).element_size()
        t = torch.empty(nbytes // itemsize, dtype=dtype, device="cuda")
        if nbytes:
            copy_buffer(self.handle, which, t, stream)
        return t.reshape(shape) if shape is not None else t
