"""The fitting loop around the renderer (Sec. 3.1): a mesh's vertex
positions and face colours are optimised so that its renders match target
images, here with the squared-error image loss and Adam or VectorAdam
(`gmr_adam_step`), and the result is scored by the chamfer distance to the
target vertices (`gmr_chamfer`).

Each step renders a batch of views, either in one call for all views (the
batched form) or one call per view (the per-view form), computes the loss,
runs the backward and updates the parameters; all of it on the GPU through
the C ABI. Target images are rendered beforehand by the same renderer from
the target mesh.
"""

from __future__ import annotations

import numpy as np
import torch

from .render import Renderer, camera_array


def render_targets(renderer: Renderer, target_verts, faces, target_rgb, opacity, view_sets):
    """Target images of every step's views, rendered from the target mesh:
    a list of [pixels, 3] device tensors."""
    out = []
    for cams in view_sets:
        img, _ = renderer.forward(target_verts, faces, target_rgb, opacity, camera_array(cams), want_t=False)
        out.append(img.clone())
    return out


def fit(scene, steps=None, lr=1e-3, form="batched", optimizer="adam", renderer=None, targets=None,
        betas=(0.9, 0.999), eps=1e-8, between_steps=None):
    """Optimise scene.verts and scene.rgb against renders of
    scene.extra["target_verts"] / ["target_rgb"] from scene.extra["view_sets"].

    form: "batched" (one call for all views of a step) or "per_view";
    optimizer: "adam" (per element) or "vectoradam" (vertex second moments
    per 3-vector). Returns a dict with the per-step losses and times (ms,
    CUDA events around each whole step), the fitted vertices and colours,
    and the chamfer distances to the target vertices before and after.
    between_steps, if given, is called after each step's closing event (so
    outside the timed region), e.g. to flush the L2 cache."""
    if form not in ("batched", "per_view"):
        raise ValueError("form must be 'batched' or 'per_view'")
    if optimizer not in ("adam", "vectoradam"):
        raise ValueError("optimizer must be 'adam' or 'vectoradam'")
    dev = torch.device("cuda")
    r = renderer or Renderer()
    view_sets = scene.extra["view_sets"]
    steps = len(view_sets) if steps is None else steps
    view_sets = view_sets[:steps]
    faces = torch.from_numpy(np.ascontiguousarray(scene.faces)).to(dev)
    verts = torch.from_numpy(np.ascontiguousarray(scene.verts)).to(dev).clone()
    rgb = torch.from_numpy(np.ascontiguousarray(scene.rgb)).to(dev).clone()
    opacity = torch.from_numpy(np.ascontiguousarray(scene.opacity)).to(dev)
    tverts = torch.from_numpy(np.ascontiguousarray(scene.extra["target_verts"])).to(dev)
    trgb = torch.from_numpy(np.ascontiguousarray(scene.extra["target_rgb"])).to(dev)
    if targets is None:
        targets = render_targets(r, tverts, faces, trgb, opacity, view_sets)

    gv = 3 if optimizer == "vectoradam" else 1
    m_v, v_v = torch.zeros_like(verts), torch.zeros(verts.numel() // gv, device=dev)
    m_c, v_c = torch.zeros_like(rgb), torch.zeros(rgb.numel(), device=dev)
    dv, dc, dop = torch.empty_like(verts), torch.empty_like(rgb), torch.empty_like(opacity)
    cd0 = r.chamfer(verts, tverts).sum()

    cam_arrays = [camera_array(cams) for cams in view_sets]
    n_views = len(view_sets[0])
    per_view_cams = [[camera_array(cams[k:k + 1]) for k in range(len(cams))] for cams in view_sets]
    npix = targets[0].shape[0]
    img = torch.empty((npix, 3), device=dev)
    grad = torch.empty_like(img)
    losses = torch.zeros(steps, n_views if form == "per_view" else 1, dtype=torch.float64, device=dev)
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]

    for t in range(steps):
        events[t][0].record()
        if form == "batched":
            r.forward(verts, faces, rgb, opacity, cam_arrays[t], images=img, want_t=False)
            r.l2_loss(img, targets[t], grad, losses[t, 0])
            r.backward(grad, dv, dc, dop)
        else:
            off = 0
            for k, cam in enumerate(per_view_cams[t]):
                n = int(cam[0].width) * int(cam[0].height)
                sl = slice(off, off + n)
                r.forward(verts, faces, rgb, opacity, cam, images=img[sl], want_t=False)
                r.l2_loss(img[sl], targets[t][sl], grad[sl], losses[t, k])
                r.backward(grad[sl], dv, dc, dop, accumulate=k > 0)
                off += n
        r.adam_step(verts, dv, m_v, v_v, lr, t + 1, group=gv, betas=betas, eps=eps)
        r.adam_step(rgb, dc, m_c, v_c, lr, t + 1, group=1, betas=betas, eps=eps)
        events[t][1].record()
        if between_steps is not None:
            between_steps()
    cd1 = r.chamfer(verts, tverts).sum()
    torch.cuda.synchronize()
    return {
        "loss": losses.sum(1).cpu().numpy(),
        "ms": np.array([a.elapsed_time(b) for a, b in events]),
        "verts": verts,
        "rgb": rgb,
        "chamfer_initial": float(cd0),
        "chamfer_final": float(cd1),
        "pixels_per_step": npix,
        "status": r.device_status(),
    }
