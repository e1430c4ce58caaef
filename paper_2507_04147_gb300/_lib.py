"""ctypes binding of libA3FR.so: the C structs of include/a3fr.h and the raw entry points.

Argument marshalling only.  Every step of a render runs in the CUDA library; if the
library is missing or fails to load this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libA3FR.so")

A3FR_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "CAPACITY", -5: "TIMEOUT", -6: "NOT_READY"}
STATUS_CAPACITY = 1
STATUS_TIMEOUT = 2

NOALLOC_MAX_PAIRS = 262144

STAGES = ("preprocess", "depth_sort", "bin", "emit", "composite")

BUF_RECORDS, BUF_RECTS, BUF_KEYS, BUF_VALUES, BUF_RANGES, BUF_LEVELS, BUF_T_FINAL, BUF_N_CONTRIB, BUF_DEPTH = range(1, 10)


class SceneDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("sh_degree", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("means", ctypes.c_void_p),
                ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12)]


class Fovea(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("theta_deg", ctypes.c_float * 3),
                ("dtheta_deg", ctypes.c_float), ("level", ctypes.c_int32 * 4), ("fill", ctypes.c_int32),
                ("count_frac", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("n_eyes", ctypes.c_int32),
                ("instances", ctypes.c_int64), ("instances_eye", ctypes.c_int64 * 2),
                ("capacity", ctypes.c_int64), ("evaluations", ctypes.c_uint64),
                ("records_staged", ctypes.c_uint64), ("renders", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("contributions", ctypes.c_uint64)]


MAX_EXITS = 8


class Rounds(ctypes.Structure):
    _fields_ = [("n_exits", ctypes.c_int32), ("sir", ctypes.c_int32),
                ("expected_dist_px", ctypes.c_float * MAX_EXITS), ("sir_step_px", ctypes.c_float)]


class RoundStatus(ctypes.Structure):
    _fields_ = [("exit_consumed", ctypes.c_int32), ("complete", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("radius_px", ctypes.c_float * 3)]


DRIVE_A3FR, DRIVE_SFR, DRIVE_FRR = 0, 1, 2


class FrameDriver(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_exits", ctypes.c_int32),
                ("predictions", ctypes.c_void_p), ("exit_time_us", ctypes.c_void_p),
                ("load_period_us", ctypes.c_double), ("load_factor", ctypes.c_double),
                ("max_rounds", ctypes.c_int32)]


class FrameResult(ctypes.Structure):
    _fields_ = [("latency_us", ctypes.c_double), ("tracker_end_us", ctypes.c_double),
                ("rounds", ctypes.c_int32), ("exit_per_round", ctypes.c_int32 * 16),
                ("round_end_us", ctypes.c_double * 16)]


class TuneResult(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("batch_mult", ctypes.c_int32), ("ms", (ctypes.c_float * 2) * 2)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class A3FRError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where} failed: A3FR_ERR_{ERRORS.get(code, code)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lib = None

# name -> (argtypes, restype)
_SIGS = {
    "a3fr_create_scene": ([ctypes.POINTER(SceneDesc), ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "a3fr_destroy_scene": ([ctypes.c_void_p], ctypes.c_int),
    "a3fr_set_camera": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Camera)], ctypes.c_int),
    "a3fr_set_gaze": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_render_foveated": ([ctypes.c_void_p, ctypes.POINTER(Fovea), ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_render_full": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_get_stats": ([ctypes.c_void_p, ctypes.POINTER(Stats), ctypes.c_int], ctypes.c_int),
    "a3fr_set_keep_aux": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_set_graph_mode": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_set_tile": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_set_batch": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_set_binning": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_autotune": ([ctypes.c_void_p, ctypes.POINTER(Fovea), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                       ctypes.POINTER(TuneResult)], ctypes.c_int),
    "a3fr_tc_tile_gemm": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "a3fr_cnn_param_count": ([], ctypes.c_size_t),
    "a3fr_cnn_create": ([ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "a3fr_cnn_arch_param_count": ([ctypes.c_int], ctypes.c_size_t),
    "a3fr_cnn_create_arch": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int], ctypes.c_int),
    "a3fr_cnn_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "a3fr_cnn_set_params": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "a3fr_cnn_get_params": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "a3fr_cnn_forward": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_cnn_grads": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                        ctypes.c_void_p], ctypes.c_int),
    "a3fr_cnn_train_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                             ctypes.c_void_p], ctypes.c_int),
    "a3fr_cnn_fill": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_backward": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Grads), ctypes.c_void_p],
                      ctypes.c_int),
    "a3fr_copy_buffer": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                          ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p], ctypes.c_int),
    "a3fr_sort_pairs_workspace_bytes": ([ctypes.c_size_t], ctypes.c_size_t),
    "a3fr_sort_pairs": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                         ctypes.c_void_p], ctypes.c_int),
    "a3fr_sort_pairs_noalloc": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                 ctypes.c_void_p], ctypes.c_int),
    "a3fr_begin_frame": ([ctypes.c_void_p, ctypes.POINTER(Fovea), ctypes.POINTER(Rounds),
                          ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_post_prediction": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "a3fr_render_round": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "a3fr_stall_mailbox": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_get_round_status": ([ctypes.c_void_p, ctypes.POINTER(RoundStatus)], ctypes.c_int),
    "a3fr_run_frame": ([ctypes.c_void_p, ctypes.POINTER(Fovea), ctypes.POINTER(Rounds),
                        ctypes.POINTER(FrameDriver), ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.POINTER(FrameResult)], ctypes.c_int),
    "a3fr_set_stage_timing": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "a3fr_get_stage_times": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "a3fr_error_string": ([ctypes.c_int], ctypes.c_char_p),
    "a3fr_last_error_detail": ([], ctypes.c_char_p),
}


def load(path: str = LIB_PATH):
    """Load libA3FR.so (built by ``paper_2507_04147_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libA3FR.so is not built ({path}); run __graft_entry__.build() "
                           "or python -m paper_2507_04147_gb300.build -- there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(code: int, where: str):
    if code != A3FR_OK:
        detail = ""
        if code == -2 and _lib is not None:
            detail = (_lib.a3fr_last_error_detail() or b"").decode()
        raise A3FRError(code, where, detail)
