"""Python front end of the Gaussian Mesh Renderer CUDA library.

``Renderer`` owns one library context (workspace + forward state) and marshals
torch CUDA tensors into the C ABI of include/gmr.h; ``GMRRender`` is the
``torch.autograd.Function`` whose forward and backward are the library's
``gmr_render_fwd`` / ``gmr_render_bwd``. PyTorch only provides device memory
and streams here.
"""

from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib

_COV = {"area": _lib.GMR_COV_AREA, "embed_raw": _lib.GMR_COV_EMBED_RAW}
_COLOR = {"face": _lib.GMR_COLOR_PER_FACE, "vertex": _lib.GMR_COLOR_PER_VERTEX, "sh": _lib.GMR_COLOR_SH}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_dev(t: torch.Tensor, name: str, dtype):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def camera_array(cams) -> ctypes.Array:
    """CAMERA_DTYPE numpy array -> ctypes array of gmr_camera (same bytes)."""
    a = np.ascontiguousarray(cams)
    if a.dtype.itemsize != ctypes.sizeof(_lib.GmrCamera):
        raise ValueError("camera records must be 76 bytes (gmr_inputs.CAMERA_DTYPE)")
    arr = (_lib.GmrCamera * len(a))()
    ctypes.memmove(arr, a.ctypes.data, a.nbytes)
    return arr


def pixel_offsets(cams) -> np.ndarray:
    off = [0]
    for c in cams:
        off.append(off[-1] + int(c["width"]) * int(c["height"]))
    return np.array(off, dtype=np.int64)


def _stage_mask(profile):
    """profile: False / True (every stage) / stage names to time."""
    if isinstance(profile, (bool, int)) or profile is None:
        return 0
    return sum(1 << _lib.STAGES.index(name) for name in profile)


def _default_threads(tile):
    return {8: 64, 32: 256}.get(tile, 128)


class Renderer:
    """One library context on the current CUDA device.

    tile: 8, 16 or 32; threads / threads_bwd: threads per tile in the forward
    / backward (32/64 for 8x8 tiles, 64/128/256 for 16x16, 256 for 32x32;
    None: 64, 128 and 256 respectively); batch: Gaussians per shared-memory
    batch (64/128/256);
    cov_mode: "area" (Eq. 13) or "embed_raw" (Eq. 15 literally);
    color_mode: "face" (F x 3 colours), "vertex" (V x 3, Eq. 16) or "sh"
    (view-dependent: F x (sh_degree + 1)^2 x 3 spherical-harmonic
    coefficients, sh_degree 0..3);
    sync_check: read the pair count back once per forward and grow buffers
    (False: never synchronise; pre-size with ``reserve`` for graph capture).
    profile: time the stages with CUDA events (True: all of them; or a list
    of stage names from ``STAGES``).
    persistent: run the compositing kernels as persistent grids (resident
    CTAs taking tiles from a counter) instead of one CTA per tile.
    half_fwd / half_bwd: the half-warp layout in the forward / backward
    compositing kernel (16-lane halves with their own 4x4-pixel units and
    lists; 16x16 tiles with 128 or 256 threads, or 8x8 tiles).
    warp_fwd / warp_bwd: the warp-staged layout (each warp stages the
    tile's list itself, no block-wide barrier inside a tile).
    deterministic: every gradient sum of the backward in a fixed order
    (bit-identical gradients for identical inputs and launch shape; the
    backward runs block-staged with at most 128 Gaussians per batch, so not
    with half_bwd or warp_bwd).
    """

    def __init__(self, tile=16, batch=256, cov_mode="area", color_mode="face", bg=(0.0, 0.0, 0.0),
                 sync_check=True, profile=False, threads=None, debug_counts=False, threads_bwd=None,
                 persistent=False, sh_degree=0, half_fwd=False, half_bwd=False, warp_fwd=False,
                 warp_bwd=False, deterministic=False):
        if not torch.cuda.is_available():
            raise _lib.GmrError("the Gaussian Mesh Renderer needs a CUDA device")
        torch.cuda.init()
        self._L = _lib.load()
        self.cfg = _lib.GmrConfig()
        self._L.gmr_config_default(ctypes.byref(self.cfg))
        self.cfg.tile = tile
        self.cfg.threads = threads or _default_threads(tile)
        self.cfg.threads_bwd = threads_bwd or _default_threads(tile)
        self.cfg.batch = batch
        self.cfg.cov_mode = _COV[cov_mode]
        self.cfg.color_mode = _COLOR[color_mode]
        self.cfg.sh_degree = int(sh_degree)
        self.cfg.bg[:] = [float(x) for x in bg]
        self.cfg.flags = ((_lib.GMR_FLAG_SYNC_CHECK if sync_check else 0) | (_lib.GMR_FLAG_PROFILE if profile else 0)
                          | (_lib.GMR_FLAG_DEBUG_COUNTS if debug_counts else 0)
                          | (_lib.GMR_FLAG_PERSISTENT if persistent else 0)
                          | (_lib.GMR_FLAG_HALF_WARP_FWD if half_fwd else 0)
                          | (_lib.GMR_FLAG_HALF_WARP_BWD if half_bwd else 0)
                          | (_lib.GMR_FLAG_WARP_STAGE_FWD if warp_fwd else 0)
                          | (_lib.GMR_FLAG_WARP_STAGE_BWD if warp_bwd else 0)
                          | (_lib.GMR_FLAG_DETERMINISTIC if deterministic else 0))
        self.cfg.profile_stages = _stage_mask(profile)
        self.color_mode = color_mode
        self._ctx = ctypes.c_void_p()
        self._check(self._L.gmr_create(ctypes.byref(self.cfg), ctypes.byref(self._ctx)), "gmr_create")
        self.fwd_token = 0
        self._saved = None

    # -- plumbing
    def _check(self, status, what):
        if status != _lib.GMR_OK:
            msg = self._L.gmr_last_error(self._ctx).decode() if self._ctx else ""
            raise _lib.GmrError(f"{what} failed: {_lib.STATUS_NAMES.get(status, status)} {msg}")

    def close(self):
        if self._ctx:
            torch.cuda.synchronize()
            self._L.gmr_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._ctx:
                self._L.gmr_destroy(self._ctx)
        except Exception:
            pass

    def set_config(self, **kw):
        """Changes configuration fields; a new tile size without thread
        counts takes that size's default thread counts. A refused change
        (GmrError) leaves the configuration as it was."""
        saved_cfg = type(self.cfg).from_buffer_copy(self.cfg)
        saved_color_mode = self.color_mode
        if "tile" in kw:
            kw.setdefault("threads", _default_threads(kw["tile"]))
            kw.setdefault("threads_bwd", _default_threads(kw["tile"]))
        for k, v in kw.items():
            if k == "cov_mode":
                v = _COV[v]
            if k == "color_mode":
                self.color_mode = v
                v = _COLOR[v]
            if k == "bg":
                self.cfg.bg[:] = [float(x) for x in v]
                continue
            if k == "sync_check":
                self.cfg.flags = (self.cfg.flags & ~_lib.GMR_FLAG_SYNC_CHECK) | (_lib.GMR_FLAG_SYNC_CHECK if v else 0)
                continue
            flag = {"persistent": _lib.GMR_FLAG_PERSISTENT, "half_fwd": _lib.GMR_FLAG_HALF_WARP_FWD,
                    "half_bwd": _lib.GMR_FLAG_HALF_WARP_BWD, "warp_fwd": _lib.GMR_FLAG_WARP_STAGE_FWD,
                    "warp_bwd": _lib.GMR_FLAG_WARP_STAGE_BWD, "deterministic": _lib.GMR_FLAG_DETERMINISTIC}.get(k)
            if flag is not None:
                self.cfg.flags = (self.cfg.flags & ~flag) | (flag if v else 0)
                continue
            if k == "profile":
                self.cfg.flags = (self.cfg.flags & ~_lib.GMR_FLAG_PROFILE) | (_lib.GMR_FLAG_PROFILE if v else 0)
                self.cfg.profile_stages = _stage_mask(v)
                continue
            setattr(self.cfg, k, v)
        try:
            self._check(self._L.gmr_set_config(self._ctx, ctypes.byref(self.cfg)), "gmr_set_config")
        except _lib.GmrError:
            self.cfg = saved_cfg
            self.color_mode = saved_color_mode
            raise

    def set_workspace_limit(self, max_bytes):
        """Caps the device bytes of the workspace (0: no cap); a call that
        would grow it beyond the cap raises GmrError (GMR_ERR_OOM)."""
        self._check(self._L.gmr_set_workspace_limit(self._ctx, int(max_bytes)), "gmr_set_workspace_limit")

    def reserve(self, max_faces, max_views, max_pixels, max_pairs):
        self._check(self._L.gmr_reserve(self._ctx, int(max_faces), int(max_views), int(max_pixels), int(max_pairs)),
                    "gmr_reserve")

    def _remember(self, verts, faces, rgb, opacity):
        """Keeps the forward's inputs (the backward reads them again) with
        their version counters, which torch bumps on every in-place change."""
        self.fwd_token += 1
        inputs = (verts, faces, rgb, opacity)
        self._saved = inputs
        self._saved_versions = tuple(None if t is None else t._version for t in inputs)

    def _saved_inputs(self):
        """The last forward's inputs; raises when one of them was modified in
        place since (the backward would mix new values with the forward's
        compositing state)."""
        if self._saved is None:
            raise _lib.GmrError("backward without a forward")
        for t, ver, name in zip(self._saved, self._saved_versions, ("verts", "faces", "rgb", "opacity")):
            if t is not None and t._version != ver:
                raise _lib.GmrError(f"{name} was modified in place between the forward and the backward")
        return self._saved

    # -- entry points
    def convert(self, verts, faces, rgb=None, opacity=None, stream=None):
        _check_dev(verts, "verts", torch.float32)
        _check_dev(faces, "faces", torch.int32)
        F = faces.shape[0]
        dev = verts.device
        means = torch.empty((F, 3), device=dev, dtype=torch.float32)
        cov = torch.empty((F, 6), device=dev, dtype=torch.float32)
        face_rgb = torch.empty((F, 3), device=dev, dtype=torch.float32) if rgb is not None else None
        face_o = torch.empty((F,), device=dev, dtype=torch.float32)
        self._check(self._L.gmr_convert(self._ctx, _ptr(verts), verts.shape[0], _ptr(faces), F, _ptr(rgb),
                                        _ptr(opacity), _ptr(means), _ptr(cov), _ptr(face_rgb), _ptr(face_o),
                                        _stream(stream)), "gmr_convert")
        return {"means": means, "cov": cov, "rgb": face_rgb, "opacity": face_o}

    def forward(self, verts, faces, rgb, opacity, cams, images=None, t_final=None, stream=None, want_t=True):
        """Render all views; returns (images [Npix, 3], t_final [Npix] or None)."""
        _check_dev(verts, "verts", torch.float32)
        _check_dev(faces, "faces", torch.int32)
        _check_dev(rgb, "rgb", torch.float32)
        if opacity is not None:
            _check_dev(opacity, "opacity", torch.float32)
        cam_arr = cams if isinstance(cams, ctypes.Array) else camera_array(cams)
        npix = sum(int(c.width) * int(c.height) for c in cam_arr)
        dev = verts.device
        if images is None:
            images = torch.empty((npix, 3), device=dev, dtype=torch.float32)
        if t_final is None and want_t:
            t_final = torch.empty((npix,), device=dev, dtype=torch.float32)
        self._check(self._L.gmr_render_fwd(self._ctx, _ptr(verts), verts.shape[0], _ptr(faces), faces.shape[0],
                                           _ptr(rgb), _ptr(opacity), cam_arr, len(cam_arr), _ptr(images),
                                           _ptr(t_final), _stream(stream)), "gmr_render_fwd")
        self._remember(verts, faces, rgb, opacity)
        return images, t_final

    def forward_l2(self, verts, faces, rgb, opacity, cams, target, images=None, grad=None, loss=None, stream=None):
        """Render all views and the squared-error loss against ``target`` in
        one pass (gmr_render_fwd_l2); returns (images, dL/dimages, loss)."""
        for t, name in ((verts, "verts"), (rgb, "rgb"), (target, "target")):
            _check_dev(t, name, torch.float32)
        _check_dev(faces, "faces", torch.int32)
        if opacity is not None:
            _check_dev(opacity, "opacity", torch.float32)
        cam_arr = cams if isinstance(cams, ctypes.Array) else camera_array(cams)
        npix = sum(int(c.width) * int(c.height) for c in cam_arr)
        if tuple(target.shape) != (npix, 3):
            raise _lib.GmrError(f"target must be [{npix}, 3]")
        dev = verts.device
        if images is None:
            images = torch.empty((npix, 3), device=dev, dtype=torch.float32)
        if grad is None:
            grad = torch.empty((npix, 3), device=dev, dtype=torch.float32)
        if loss is None:
            loss = torch.empty((), device=dev, dtype=torch.float64)
        self._check(self._L.gmr_render_fwd_l2(self._ctx, _ptr(verts), verts.shape[0], _ptr(faces), faces.shape[0],
                                              _ptr(rgb), _ptr(opacity), cam_arr, len(cam_arr), _ptr(images), None,
                                              _ptr(target), _ptr(grad), _ptr(loss), _stream(stream)),
                    "gmr_render_fwd_l2")
        self._remember(verts, faces, rgb, opacity)
        return images, grad, loss

    def backward(self, dL_dimages, dverts=None, drgb=None, dopacity=None, accumulate=False, stream=None,
                 dL_dtfinal=None):
        """Gradients of the last forward from dL/dimages and/or dL/dT_final
        (either may be None, not both)."""
        if dL_dimages is not None:
            _check_dev(dL_dimages, "dL_dimages", torch.float32)
        if dL_dtfinal is not None:
            _check_dev(dL_dtfinal, "dL_dtfinal", torch.float32)
        verts, faces, rgb, opacity = self._saved_inputs()
        if dverts is None:
            dverts = torch.empty_like(verts)
        if drgb is None:
            drgb = torch.empty_like(rgb)
        if dopacity is None and opacity is not None:
            dopacity = torch.empty_like(opacity)
        self._check(self._L.gmr_render_bwd_ex(self._ctx, _ptr(dL_dimages), _ptr(dL_dtfinal), _ptr(dverts),
                                              _ptr(drgb), _ptr(dopacity), 1 if accumulate else 0, _stream(stream)),
                    "gmr_render_bwd_ex")
        return dverts, drgb, dopacity

    def backward_l2(self, images, target, loss=None, dverts=None, drgb=None, dopacity=None, accumulate=False,
                    stream=None, dL_dtfinal=None):
        """Backward of the squared-error loss sum((images - target)^2) of the
        last forward, the loss formed inside the compositing backward
        (gmr_render_bwd_l2): returns (loss, dverts, drgb, dopacity)."""
        _check_dev(images, "images", torch.float32)
        _check_dev(target, "target", torch.float32)
        if tuple(target.shape) != tuple(images.shape):
            raise _lib.GmrError("target must have the shape of images")
        if dL_dtfinal is not None:
            _check_dev(dL_dtfinal, "dL_dtfinal", torch.float32)
        verts, faces, rgb, opacity = self._saved_inputs()
        if loss is None:
            loss = torch.empty((), device=verts.device, dtype=torch.float64)
        if dverts is None:
            dverts = torch.empty_like(verts)
        if drgb is None:
            drgb = torch.empty_like(rgb)
        if dopacity is None and opacity is not None:
            dopacity = torch.empty_like(opacity)
        self._check(self._L.gmr_render_bwd_l2(self._ctx, _ptr(images), _ptr(target), _ptr(loss), _ptr(dL_dtfinal),
                                              _ptr(dverts), _ptr(drgb), _ptr(dopacity), 1 if accumulate else 0,
                                              _stream(stream)), "gmr_render_bwd_l2")
        return loss, dverts, drgb, dopacity

    def silhouette_bce(self, t_final, mask, grad=None, loss=None, weight=1.0, stream=None):
        """weight x the binary cross-entropy of the rendered mask 1 - t_final
        against mask (mean over pixels); returns (loss, dL/dt_final)."""
        _check_dev(t_final, "t_final", torch.float32)
        _check_dev(mask, "mask", torch.float32)
        if grad is None:
            grad = torch.empty_like(t_final)
        if loss is None:
            loss = torch.empty((), device=t_final.device, dtype=torch.float64)
        self._check(self._L.gmr_silhouette_bce(self._ctx, _ptr(t_final), _ptr(mask), t_final.numel(),
                                               float(weight), _ptr(grad), _ptr(loss), _stream(stream)),
                    "gmr_silhouette_bce")
        return loss, grad

    def l2_loss(self, img, target, grad=None, loss=None, stream=None):
        _check_dev(img, "img", torch.float32)
        _check_dev(target, "target", torch.float32)
        if grad is None:
            grad = torch.empty_like(img)
        if loss is None:
            loss = torch.empty((), device=img.device, dtype=torch.float64)
        self._check(self._L.gmr_l2_loss(self._ctx, _ptr(img), _ptr(target), img.numel(), _ptr(grad), _ptr(loss),
                                        _stream(stream)), "gmr_l2_loss")
        return loss, grad

    def adam_step(self, params, grads, m, v, lr, step, group=1, betas=(0.9, 0.999), eps=1e-8, stream=None):
        """In-place Adam (group=1) or VectorAdam (group=3, per 3-vector
        second moment; v has params.numel() / 3 entries) step; step >= 1."""
        for t, name in ((params, "params"), (grads, "grads"), (m, "m"), (v, "v")):
            _check_dev(t, name, torch.float32)
        n = params.numel()
        if grads.numel() != n or m.numel() != n or v.numel() * group != n:
            raise ValueError("adam_step: params, grads, m and v sizes do not match")
        self._check(self._L.gmr_adam_step(self._ctx, _ptr(params), _ptr(grads), _ptr(m), _ptr(v), n, group,
                                          float(lr), float(betas[0]), float(betas[1]), float(eps), int(step),
                                          _stream(stream)), "gmr_adam_step")

    def mesh_regularizers(self, verts, faces, w_edge=1.0, w_lap=1.0, dverts=None, losses=None, stream=None):
        """Edge-length and Laplacian regularisers: returns a device tensor of
        the two (unweighted) losses; adds w_edge and w_lap times their vertex
        gradients to dverts when it is given."""
        _check_dev(verts, "verts", torch.float32)
        _check_dev(faces, "faces", torch.int32)
        if dverts is not None:
            _check_dev(dverts, "dverts", torch.float32)
        if losses is None:
            losses = torch.empty(2, device=verts.device, dtype=torch.float64)
        self._check(self._L.gmr_mesh_regularizers(self._ctx, _ptr(verts), verts.shape[0], _ptr(faces),
                                                  faces.shape[0], float(w_edge), float(w_lap), _ptr(dverts),
                                                  _ptr(losses), _stream(stream)), "gmr_mesh_regularizers")
        return losses

    def chamfer(self, a, b, out=None, stream=None):
        """Chamfer distance between point sets a [na, 3] and b [nb, 3]:
        a device tensor of 2 doubles (mean a->b and b->a squared nearest
        distances; CD = their sum)."""
        _check_dev(a, "a", torch.float32)
        _check_dev(b, "b", torch.float32)
        if out is None:
            out = torch.empty(2, device=a.device, dtype=torch.float64)
        self._check(self._L.gmr_chamfer(self._ctx, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(out),
                                        _stream(stream)), "gmr_chamfer")
        return out

    def device_status(self, stream=None) -> int:
        st = ctypes.c_uint32()
        self._check(self._L.gmr_get_device_status(self._ctx, _stream(stream), ctypes.byref(st)),
                    "gmr_get_device_status")
        return int(st.value)

    def stats(self, stream=None) -> dict:
        s = _lib.GmrStats()
        self._check(self._L.gmr_get_stats(self._ctx, _stream(stream), ctypes.byref(s)), "gmr_get_stats")
        return {k: int(getattr(s, k)) for k, _ in _lib.GmrStats._fields_}

    def stage_times(self, stream=None) -> dict:
        """Milliseconds of each stage's last profiled run (None if not run)."""
        ms = (ctypes.c_float * len(_lib.STAGES))()
        self._check(self._L.gmr_get_stage_times(self._ctx, _stream(stream), ms), "gmr_get_stage_times")
        return {k: (float(ms[i]) if ms[i] >= 0 else None) for i, k in enumerate(_lib.STAGES)}

    def debug_state(self, n_views, n_faces, n_tiles, n_pixels, stream=None):
        """Copies of the last forward's binning data (for tests)."""
        dev = torch.device("cuda")
        R = n_views * n_faces
        depth = torch.empty(R, dtype=torch.int32, device=dev)
        rects = torch.empty((R, 4), dtype=torch.int32, device=dev)
        rec_u = torch.empty((R, 4), dtype=torch.float32, device=dev)
        conic = torch.empty((R, 4), dtype=torch.float32, device=dev)
        ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=dev)
        n_last = torch.empty(n_pixels, dtype=torch.int32, device=dev)
        npairs = ctypes.c_int64()
        self._check(self._L.gmr_debug_forward_state(self._ctx, _ptr(depth), _ptr(rects), None, None, 0, _ptr(ranges),
                                                    _ptr(rec_u), _ptr(conic), _ptr(n_last), None,
                                                    ctypes.byref(npairs), _stream(stream)), "gmr_debug_forward_state")
        P = int(npairs.value)
        tiles = torch.empty(max(P, 1), dtype=torch.int32, device=dev)
        fids = torch.empty(max(P, 1), dtype=torch.int32, device=dev)
        self._check(self._L.gmr_debug_forward_state(self._ctx, None, None, _ptr(tiles), _ptr(fids), max(P, 1), None,
                                                    None, None, None, None, ctypes.byref(npairs), _stream(stream)),
                    "gmr_debug_forward_state")
        torch.cuda.synchronize()
        u32 = lambda t: t.cpu().numpy().view(np.uint32)
        return {"depth_bits": u32(depth), "rects": rects.cpu().numpy(), "rec_u": rec_u.cpu().numpy(),
                "conic": conic.cpu().numpy()[:, :3], "ranges": u32(ranges), "n_last": u32(n_last),
                "tile_ids": u32(tiles)[:P], "face_ids": u32(fids)[:P], "n_pairs": P}


    def contributor_counts(self, n_pixels, stream=None) -> torch.Tensor:
        """Per-pixel contributor counts of the last forward, then per-pixel
        hashes of the ordered contributor lists (debug_counts)."""
        out = torch.empty(2 * n_pixels, dtype=torch.int32, device="cuda")
        npairs = ctypes.c_int64()
        self._check(self._L.gmr_debug_forward_state(self._ctx, None, None, None, None, 0, None, None, None, None,
                                                    _ptr(out), ctypes.byref(npairs), _stream(stream)),
                    "gmr_debug_forward_state")
        return out


class GMRRender(torch.autograd.Function):
    """images = GMRRender.apply(verts, rgb, opacity, faces, cams, renderer)

    Differentiable w.r.t. verts (V x 3), rgb and opacity (per face). The
    backward runs gmr_render_bwd on the renderer's stored forward state, so a
    renderer serves one outstanding forward at a time.
    """

    @staticmethod
    def forward(ctx, verts, rgb, opacity, faces, cams, renderer: Renderer):
        images, _ = renderer.forward(verts, faces, rgb, opacity, cams, want_t=False)
        ctx.renderer = renderer
        ctx.token = renderer.fwd_token
        ctx.has_opacity = opacity is not None
        return images

    @staticmethod
    def backward(ctx, dimg):
        r: Renderer = ctx.renderer
        if r.fwd_token != ctx.token:
            raise _lib.GmrError("the renderer ran another forward before this backward")
        dverts, drgb, dop = r.backward(dimg.contiguous())
        return dverts, drgb, (dop if ctx.has_opacity else None), None, None, None


class GMRRenderWithT(torch.autograd.Function):
    """images, t_final = GMRRenderWithT.apply(verts, rgb, opacity, faces,
    cams, renderer): as GMRRender, with the final transmittance (1 - the
    rendered silhouette) as a second differentiable output."""

    @staticmethod
    def forward(ctx, verts, rgb, opacity, faces, cams, renderer: Renderer):
        images, t_final = renderer.forward(verts, faces, rgb, opacity, cams, want_t=True)
        ctx.renderer = renderer
        ctx.token = renderer.fwd_token
        ctx.has_opacity = opacity is not None
        return images, t_final

    @staticmethod
    def backward(ctx, dimg, dt):
        r: Renderer = ctx.renderer
        if r.fwd_token != ctx.token:
            raise _lib.GmrError("the renderer ran another forward before this backward")
        if dimg is None and dt is None:
            return None, None, None, None, None, None
        dverts, drgb, dop = r.backward(None if dimg is None else dimg.contiguous(),
                                       dL_dtfinal=None if dt is None else dt.contiguous())
        return dverts, drgb, (dop if ctx.has_opacity else None), None, None, None


def copy_h2d(dst: torch.Tensor, src: torch.Tensor, stream=None) -> torch.Tensor:
    """dst (device) <- src (page-locked host tensor, e.g. from pin_memory()),
    copied by a kernel that reads the host buffer over the bus
    (gmr_copy_h2d); asynchronous on the stream. Returns dst."""
    if not dst.is_cuda or src.is_cuda or not src.is_pinned():
        raise _lib.GmrError("copy_h2d: dst must be a CUDA tensor and src a pinned host tensor")
    if not dst.is_contiguous() or not src.is_contiguous():
        raise _lib.GmrError("copy_h2d: tensors must be contiguous")
    n = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != n:
        raise _lib.GmrError("copy_h2d: sizes differ")
    L = _lib.load()
    st = L.gmr_copy_h2d(ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()), n, _stream(stream))
    if st != 0:
        raise _lib.GmrError(f"gmr_copy_h2d failed ({st})")
    return dst


def render(verts, faces, rgb, opacity, cams, renderer: Renderer):
    """Differentiable batched render of all views (packed [Npix, 3])."""
    return GMRRender.apply(verts, rgb, opacity, faces, cams, renderer)
