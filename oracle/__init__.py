"""FP64 CPU oracle for the Gaussian Mesh Renderer (test infrastructure).

A thin ctypes wrapper around ``libgmr_oracle.so`` (built from
``gmr_oracle.cpp``). Only the tests, the smoke check and the benchmark's CPU
baseline use it; the CUDA library never does, and this package imports
nothing from the CUDA package.

Inputs are the FP32 arrays of ``gmr_inputs.Scene``; the oracle widens them to
FP64 exactly and evaluates conversion (Sec. 2.2, Eq. 3-16), EWA projection
and brute-force compositing (Sec. 2.1) in FP64, plus the FP32 binning
specification (depth key, tile rectangle) evaluated with IEEE single
operations in a fixed order.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

FLAG_ALPHA_SKIP = 1
FLAG_TERMINATE = 2
FLAG_ALPHA_CLAMP = 4

DEFAULT_BANDS = (2e-5, 2e-4)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int, ctypes.c_longlong, ctypes.c_float
        L.gmr_oracle_convert.argtypes = [i32, P, i32, P, i32, P, P, P, P]
        L.gmr_oracle_project.argtypes = [i32, P, P, i32, P, P, P, P, P, P]
        L.gmr_oracle_bins.argtypes = [i32, P, i32, P, i32, P, P, i32, P, P, P, P]
        L.gmr_oracle_count_pairs.argtypes = [i32, P, i32, P, i32, P, P, i32]
        L.gmr_oracle_count_pairs.restype = i64
        L.gmr_oracle_sorted_pairs.argtypes = [i32, P, i32, P, i32, P, P, i32, i64, P, P, P]
        L.gmr_oracle_sorted_pairs.restype = i64
        L.gmr_oracle_render.argtypes = [i32, P, i32, P, P, i32, P, f32, i32, i32, P, P, P, i32, i64, P,
                                        P, P, P, P, P, P, i32]
        L.gmr_oracle_backward.argtypes = [i32, P, i32, P, P, i32, P, f32, i32, i32, P, P, P, i32, i64, P,
                                          P, P, P, P, P, P, i32]
        L.gmr_oracle_jvp.argtypes = [i32, P, i32, P, P, i32, P, f32, i32, i32, P, P, P, i32, i64, P, P,
                                     P, P, P, P, P, i32]
        L.gmr_oracle_sh_basis.argtypes = [i32, i64, P, P]
        L.gmr_oracle_set_threads.argtypes = [i32]
        L.gmr_oracle_set_threads.restype = i32
        L.gmr_oracle_set_binned.argtypes = [i32]
        L.gmr_oracle_set_binned.restype = i32
        _LIB = L
    return _LIB


def set_threads(n):
    """Host threads of the oracle's parallel loops (n < 1: every core).
    Returns the count in use. Results are bit-identical for every count."""
    return int(lib().gmr_oracle_set_threads(int(n)))


_BINNED = False
# The binned mode's grid lists every face whose o G can reach (1 - 1e-3)/255
# at a pixel of the cell, which covers the flag bands up to this width.
BINNED_MAX_ALPHA_BAND = 1e-3


def set_binned(on):
    """Binned compositing (each pixel walks the faces a 16 x 16-pixel grid
    cell lists, built from each face's FP64 support, instead of every
    visible face) for the calls that follow. Same decisions, order and
    results as the brute force (tested); returns the previous setting."""
    global _BINNED
    prev = bool(lib().gmr_oracle_set_binned(1 if on else 0))
    _BINNED = bool(on)
    return prev


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def cam_arrays(cams):
    """Flatten a CAMERA_DTYPE array to (float32 [C,17], int32 [C,2])."""
    C = len(cams)
    cf = np.zeros((C, 17), dtype=np.float32)
    ci = np.zeros((C, 2), dtype=np.int32)
    for c in range(C):
        cf[c, 0:9] = cams[c]["R"]
        cf[c, 9:12] = cams[c]["t"]
        cf[c, 12] = cams[c]["fx"]
        cf[c, 13] = cams[c]["fy"]
        cf[c, 14] = cams[c]["cx"]
        cf[c, 15] = cams[c]["cy"]
        cf[c, 16] = cams[c]["znear"]
        ci[c, 0] = cams[c]["width"]
        ci[c, 1] = cams[c]["height"]
    return np.ascontiguousarray(cf), np.ascontiguousarray(ci)


def all_pixels(cams):
    """(view, x, y) of every pixel, in the packed image order (view-major,
    then row-major)."""
    out = []
    for c, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        out.append(np.stack([np.full(W * H, c), xx.ravel(), yy.ravel()], 1))
    if not out:
        return np.zeros((0, 3), dtype=np.int32)
    return np.ascontiguousarray(np.concatenate(out, 0).astype(np.int32))


def pixel_offsets(cams):
    off = [0]
    for cam in cams:
        off.append(off[-1] + int(cam["width"]) * int(cam["height"]))
    return np.array(off, dtype=np.int64)


def convert(verts, faces, cov_mode=0):
    """Sec. 2.2 conversion in FP64. Returns dict with means [F,3], cov
    [F,3,3], aux [F,8] = (sxx, sxy, syy, lam1, lam2, kappa, area, degenerate)
    and frame [F,3,3] (rows xa, ya, n)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    F = len(f)
    means = np.zeros((F, 3))
    cov = np.zeros((F, 9))
    aux = np.zeros((F, 8))
    frame = np.zeros((F, 9))
    rc = lib().gmr_oracle_convert(len(v), _p(v), F, _p(f), cov_mode, _p(means), _p(cov), _p(aux), _p(frame))
    if rc != 0:
        raise ValueError(f"oracle convert failed ({rc})")
    return {"means": means, "cov": cov.reshape(F, 3, 3), "aux": aux, "frame": frame.reshape(F, 3, 3)}


def project(means, cov, cams):
    """EWA projection of FP64 Gaussians into every camera (view-major)."""
    m = np.ascontiguousarray(means, dtype=np.float64)
    cv = np.ascontiguousarray(np.asarray(cov, dtype=np.float64).reshape(-1, 9))
    F = len(m)
    cf, ci = cam_arrays(cams)
    C = len(cams)
    u = np.zeros((C * F, 2))
    sig = np.zeros((C * F, 3))
    conic = np.zeros((C * F, 3))
    tcam = np.zeros((C * F, 3))
    lib().gmr_oracle_project(F, _p(m), _p(cv), C, _p(cf), _p(ci), _p(u), _p(sig), _p(conic), _p(tcam))
    return {"u": u, "sigma": sig, "conic": conic, "tcam": tcam}


def bins(verts, faces, cams, tile=16):
    v = np.ascontiguousarray(verts, dtype=np.float32)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    F, C = len(f), len(cams)
    cf, ci = cam_arrays(cams)
    vis = np.zeros(C * F, dtype=np.uint8)
    db = np.zeros(C * F, dtype=np.uint32)
    rect = np.zeros((C * F, 4), dtype=np.int32)
    uxyr = np.zeros((C * F, 4), dtype=np.float32)
    rc = lib().gmr_oracle_bins(len(v), _p(v), F, _p(f), C, _p(cf), _p(ci), tile, _p(vis), _p(db), _p(rect),
                               _p(uxyr))
    if rc != 0:
        raise ValueError(f"oracle bins failed ({rc})")
    return {"visible": vis.astype(bool), "depth_bits": db, "rect": rect, "uxyr": uxyr}


def tile_counts(cams, tile):
    tx = [(int(c["width"]) + tile - 1) // tile for c in cams]
    ty = [(int(c["height"]) + tile - 1) // tile for c in cams]
    return tx, ty


def sorted_pairs(verts, faces, cams, tile=16):
    """(tile_ids, face_ids, ranges[total_tiles, 2]) in (tile, depth, index)
    order."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    f = np.ascontiguousarray(faces, dtype=np.int32)
    F, C = len(f), len(cams)
    cf, ci = cam_arrays(cams)
    L = lib()
    n = L.gmr_oracle_count_pairs(len(v), _p(v), F, _p(f), C, _p(cf), _p(ci), tile)
    tx, ty = tile_counts(cams, tile)
    total = int(sum(a * b for a, b in zip(tx, ty)))
    tiles = np.zeros(max(n, 1), dtype=np.uint32)
    fids = np.zeros(max(n, 1), dtype=np.uint32)
    ranges = np.zeros((max(total, 1), 2), dtype=np.uint32)
    m = L.gmr_oracle_sorted_pairs(len(v), _p(v), F, _p(f), C, _p(cf), _p(ci), tile, max(n, 1), _p(tiles),
                                  _p(fids), _p(ranges))
    assert m == n
    return tiles[:n], fids[:n], ranges[:total]


def _scene_args(scene, cov_mode, color_mode, bg, rgb=None):
    v = np.ascontiguousarray(scene.verts, dtype=np.float32)
    f = np.ascontiguousarray(scene.faces, dtype=np.int32)
    c = np.ascontiguousarray(scene.rgb if rgb is None else rgb, dtype=np.float32)
    o = None if scene.opacity is None else np.ascontiguousarray(scene.opacity, dtype=np.float32)
    cf, ci = cam_arrays(scene.cams)
    b = np.ascontiguousarray(np.asarray(bg if bg is not None else (0.0, 0.0, 0.0), dtype=np.float64))
    return v, f, c, o, cf, ci, b


def render(scene, pixels=None, cov_mode=0, color_mode=0, bg=None, tile=16, bands=DEFAULT_BANDS,
           opacity_scalar=1.0, sh_degree=0):
    """FP64 render of the given pixels (default: every pixel), by brute
    force over every visible face, or binned (set_binned).
    color_mode 0: per-face rgb [F,3]; 1: per-vertex rgb [V,3] (Eq. 16);
    2: spherical-harmonic coefficients [F,(sh_degree+1)^2,3]."""
    if pixels is None:
        pixels = all_pixels(scene.cams)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    v, f, c, o, cf, ci, b = _scene_args(scene, cov_mode, color_mode, bg)
    n = len(pix)
    out = np.zeros((n, 3))
    T = np.zeros(n)
    last = np.zeros(n, dtype=np.int32)
    nc = np.zeros(n, dtype=np.int32)
    fl = np.zeros(n, dtype=np.int32)
    bd = np.ascontiguousarray(np.asarray(bands, dtype=np.float64)) if bands is not None else None
    if _BINNED and bd is not None and bd[0] > BINNED_MAX_ALPHA_BAND:
        raise ValueError(f"binned mode covers alpha bands up to {BINNED_MAX_ALPHA_BAND}")
    rc = lib().gmr_oracle_render(len(v), _p(v), len(f), _p(f), _p(c), color_mode, _p(o), opacity_scalar,
                                 cov_mode, len(scene.cams), _p(cf), _p(ci), _p(b), tile, n, _p(pix), _p(out),
                                 _p(T), _p(last), _p(nc), _p(fl), _p(bd), sh_degree)
    if rc != 0:
        raise ValueError(f"oracle render failed ({rc})")
    return {"rgb": out, "T": T, "last_face": last, "n_contrib": nc, "flags": fl}


def backward(scene, dLdI, pixels=None, cov_mode=0, color_mode=0, bg=None, tile=16, opacity_scalar=1.0, dLdT=None,
             sh_degree=0):
    """Reverse-mode FP64 gradients for dL/dI (and optionally dL/dT_final)
    given at ``pixels``."""
    if pixels is None:
        pixels = all_pixels(scene.cams)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    g = np.ascontiguousarray(np.asarray(dLdI, dtype=np.float64).reshape(-1, 3))
    assert len(g) == len(pix)
    v, f, c, o, cf, ci, b = _scene_args(scene, cov_mode, color_mode, bg)
    V, F, C = len(v), len(f), len(scene.cams)
    dV = np.zeros((V, 3))
    drgb = np.zeros(c.shape)
    dop = np.zeros(F)
    rec = np.zeros((C * F, 9))
    gT = None if dLdT is None else np.ascontiguousarray(np.asarray(dLdT, dtype=np.float64).reshape(-1))
    assert gT is None or len(gT) == len(pix)
    rc = lib().gmr_oracle_backward(V, _p(v), F, _p(f), _p(c), color_mode, _p(o), opacity_scalar, cov_mode, C,
                                   _p(cf), _p(ci), _p(b), tile, len(pix), _p(pix), _p(g), _p(dV), _p(drgb),
                                   _p(dop), _p(rec), _p(gT), sh_degree)
    if rc != 0:
        raise ValueError(f"oracle backward failed ({rc})")
    return {"dverts": dV, "drgb": drgb, "dopacity": dop, "rec": rec}


def sh_basis(degree, dirs):
    """Real spherical harmonics of degree <= ``degree`` (colour mode 2) at
    unit directions dirs [n,3]: [n,(degree+1)^2]."""
    d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((len(d), (degree + 1) ** 2))
    if lib().gmr_oracle_sh_basis(int(degree), len(d), _p(d), _p(out)) != 0:
        raise ValueError("degree must be 0..3")
    return out


def jvp(scene, w, dverts=None, drgb=None, dop=None, pixels=None, cov_mode=0, color_mode=0, bg=None, tile=16,
        opacity_scalar=1.0, wT=None, sh_degree=0):
    """Forward-mode d/de (sum <w, I(x + e dir)> + sum wT T_final) with dual
    numbers."""
    if pixels is None:
        pixels = all_pixels(scene.cams)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    ww = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1, 3))
    v, f, c, o, cf, ci, b = _scene_args(scene, cov_mode, color_mode, bg)

    def arr(a):
        return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))

    dv, dc, do = arr(dverts), arr(drgb), arr(dop)
    out = np.zeros(1)
    rc = lib().gmr_oracle_jvp(len(v), _p(v), len(f), _p(f), _p(c), color_mode, _p(o), opacity_scalar, cov_mode,
                              len(scene.cams), _p(cf), _p(ci), _p(b), tile, len(pix), _p(pix), _p(ww), _p(dv),
                              _p(dc), _p(do), _p(out),
                              _p(None if wT is None else np.ascontiguousarray(np.asarray(wT, dtype=np.float64))),
                              sh_degree)
    if rc != 0:
        raise ValueError(f"oracle jvp failed ({rc})")
    return float(out[0])
