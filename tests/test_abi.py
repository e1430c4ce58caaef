"""The C-ABI library builds, loads and exports every symbol include/a3fr.h declares.

No GPU is needed: these tests make no compute call, only argument checks that fail
before any CUDA work.
"""
import ctypes
import os
import re

import pytest

import paper_2507_04147_gb300 as a3fr
from paper_2507_04147_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "a3fr.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(a3fr_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("a3fr_create_scene", "a3fr_destroy_scene", "a3fr_set_camera",
                     "a3fr_set_gaze", "a3fr_render_foveated", "a3fr_render_full",
                     "a3fr_get_stats", "a3fr_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the Python binding wraps every one of them
    assert set(declared_functions()) <= set(_lib._SIGS)


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(_lib.Camera) == 4 * 19
    assert ctypes.sizeof(_lib.Fovea) == 4 * 11
    assert ctypes.sizeof(_lib.SceneDesc) == 16 + 5 * 8
    assert ctypes.sizeof(_lib.Stats) == 8 + 8 + 16 + 8 + 40


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert a3fr.error_string(code).startswith("A3FR_")
    assert "unknown" in a3fr.error_string(-99)


def test_invalid_arguments_rejected_before_cuda(lib):
    out = ctypes.c_void_p()
    assert lib.a3fr_create_scene(None, 0, ctypes.byref(out)) == -1
    d = _lib.SceneDesc()
    d.n, d.sh_degree, d.tile = 10, 5, 16          # degree out of range
    assert lib.a3fr_create_scene(ctypes.byref(d), 0, ctypes.byref(out)) == -1
    d.sh_degree, d.tile = 0, 12                    # unsupported tile
    assert lib.a3fr_create_scene(ctypes.byref(d), 0, ctypes.byref(out)) == -1
    d.tile = 16                                    # null arrays with n > 0
    assert lib.a3fr_create_scene(ctypes.byref(d), 0, ctypes.byref(out)) == -1
    d.means = 8                                    # misaligned
    assert lib.a3fr_create_scene(ctypes.byref(d), 0, ctypes.byref(out)) == -1
    assert lib.a3fr_destroy_scene(None) == -1
    assert lib.a3fr_set_camera(None, 0, None) == -1
    assert lib.a3fr_set_gaze(None, None, None) == -1
    assert lib.a3fr_render_full(None, None, None) == -1
    assert lib.a3fr_render_foveated(None, None, None, None) == -1
    assert lib.a3fr_get_stats(None, None, 0) == -1
    assert lib.a3fr_sort_pairs(None, None, None, None, 0, 40, None, 0, None) == 0   # n = 0: no-op
    assert lib.a3fr_sort_pairs(None, None, None, None, 5, 40, None, 0, None) == -1
    assert lib.a3fr_sort_pairs_workspace_bytes(10**6) > 0


def test_periphery_parameter_counts_match_the_layer_tables(lib):
    """Host-only arithmetic of the library: the flat parameter count of each network equals
    the Python layer tables' (weights [out][in][k][k], then biases); unknown ones are 0 and
    cannot be created."""
    from paper_2507_04147_gb300 import periphery
    for arch, layers in periphery.ARCH_LAYERS.items():
        want = sum(i * o * k * k + o for i, o, k in layers)
        assert lib.a3fr_cnn_arch_param_count(arch) == want
    assert lib.a3fr_cnn_param_count() == lib.a3fr_cnn_arch_param_count(periphery.RESIDUAL)
    assert lib.a3fr_cnn_arch_param_count(7) == 0
    out = ctypes.c_void_p()
    assert lib.a3fr_cnn_create_arch(ctypes.byref(out), 7) == -1
    assert lib.a3fr_cnn_create_arch(None, periphery.COMPACT) == -1


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(_lib.load, "__wrapped__") \
            else _missing_load(str(tmp_path / "nope.so"))


def _missing_load(path):
    saved = _lib._lib
    _lib._lib = None
    try:
        return _lib.load(path)
    finally:
        _lib._lib = saved
