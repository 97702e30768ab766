"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads
without a GPU, and exports every function include/gmr.h declares; the ctypes
structures match the header's layouts."""

import ctypes
import os
import re

import numpy as np

import gmr_inputs as gi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gmr.h")).read()
    return sorted(set(re.findall(r"^GMR_API [^(]*?\b(gmr_\w+)\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2602_14493_b300 import build, _lib

    build.build()
    L = ctypes.CDLL(build.LIB)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(_lib.EXPORTS) == declared
    _lib.load()


def test_struct_layouts_match_header():
    from paper_2602_14493_b300 import _lib

    assert ctypes.sizeof(_lib.GmrCamera) == 76 == gi.CAMERA_DTYPE.itemsize
    assert ctypes.sizeof(_lib.GmrConfig) == 48
    assert ctypes.sizeof(_lib.GmrStats) == 80
    cam = gi.look_at((0.0, -3.0, 1.0), 32, 16)
    arr = np.array([cam], dtype=gi.CAMERA_DTYPE)
    from paper_2602_14493_b300.render import camera_array

    ca = camera_array(arr)
    assert ca[0].width == 32 and ca[0].height == 16
    np.testing.assert_array_equal(np.array(ca[0].R[:]), arr[0]["R"])


def test_host_only_entry_points_without_gpu():
    """Host-side entry points that touch no device: defaults, status names,
    image offsets, argument checks on a null context."""
    from paper_2602_14493_b300 import _lib

    L = _lib.load()
    cfg = _lib.GmrConfig()
    assert L.gmr_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.tile, cfg.threads, cfg.threads_bwd, cfg.batch, cfg.cov_mode, cfg.color_mode, cfg.flags) == (
        16, 128, 128, 256, 0, 0, 1)
    assert L.gmr_status_string(4) == b"GMR_ERR_CAPACITY"
    cams = (_lib.GmrCamera * 3)()
    for i, (w, h) in enumerate([(10, 7), (3, 3), (256, 1)]):
        cams[i].width, cams[i].height = w, h
    off = (ctypes.c_int64 * 4)()
    assert L.gmr_image_offsets(cams, 3, off) == 0
    assert list(off) == [0, 70, 79, 335]
    assert L.gmr_render_fwd(None, None, 0, None, 0, None, None, None, 1, None, None, None) == 1
    assert L.gmr_render_bwd(None, None, None, None, None, 0, None) == 1
    assert L.gmr_destroy(None) == 1
