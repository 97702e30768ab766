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


def render_targets(renderer: Renderer, target_verts, faces, target_rgb, opacity, view_sets, masks=False):
    """Target images of every step's views, rendered from the target mesh:
    a list of [pixels, 3] device tensors (with masks=True also the target
    silhouettes 1 - T_final, a list of [pixels] tensors)."""
    out, sil = [], []
    for cams in view_sets:
        img, T = renderer.forward(target_verts, faces, target_rgb, opacity, camera_array(cams), want_t=masks)
        out.append(img.clone())
        if masks:
            sil.append((1.0 - T).clone())
    return (out, sil) if masks else out


def fit(scene, steps=None, lr=1e-3, form="batched", optimizer="adam", renderer=None, targets=None,
        betas=(0.9, 0.999), eps=1e-8, between_steps=None, w_silhouette=0.0, w_edge=0.0, w_laplacian=0.0):
    """Optimise scene.verts and scene.rgb against renders of
    scene.extra["target_verts"] / ["target_rgb"] from scene.extra["view_sets"].

    form: "batched" (one call for all views of a step) or "per_view";
    optimizer: "adam" (per element) or "vectoradam" (vertex second moments
    per 3-vector). Returns a dict with the per-step losses and times (ms,
    CUDA events around each whole step), the fitted vertices and colours,
    and the chamfer distances to the target vertices before and after.
    between_steps, if given, is called after each step's closing event (so
    outside the timed region), e.g. to flush the L2 cache. w_silhouette,
    w_edge and w_laplacian add the other losses of the paper's fitting loop
    (silhouette cross-entropy against the target's silhouettes, edge-length
    and Laplacian regularisers); all 0 by default (image loss only)."""
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
    use_sil = w_silhouette != 0.0
    use_reg = w_edge != 0.0 or w_laplacian != 0.0
    masks = None
    if targets is None or use_sil:
        rendered = render_targets(r, tverts, faces, trgb, opacity, view_sets, masks=use_sil)
        targets, masks = rendered if use_sil else (rendered, None)

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
    tfin = torch.empty(npix, device=dev) if use_sil else None
    gradT = torch.empty_like(tfin) if use_sil else None
    losses = torch.zeros(steps, n_views if form == "per_view" else 1, dtype=torch.float64, device=dev)
    sil_losses = torch.zeros(steps, n_views if form == "per_view" else 1, dtype=torch.float64, device=dev)
    reg_losses = torch.zeros(steps, 2, dtype=torch.float64, device=dev)
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]

    for t in range(steps):
        events[t][0].record()
        if form == "batched":
            r.forward(verts, faces, rgb, opacity, cam_arrays[t], images=img, t_final=tfin, want_t=use_sil)
            if use_sil:
                r.silhouette_bce(tfin, masks[t], gradT, sil_losses[t, 0], weight=w_silhouette)
            r.backward_l2(img, targets[t], losses[t, 0], dv, dc, dop, dL_dtfinal=gradT)
        else:
            off = 0
            for k, cam in enumerate(per_view_cams[t]):
                n = int(cam[0].width) * int(cam[0].height)
                sl = slice(off, off + n)
                r.forward(verts, faces, rgb, opacity, cam, images=img[sl], t_final=tfin[sl] if use_sil else None,
                          want_t=use_sil)
                if use_sil:
                    # the batched form's mean over all views' pixels: weight n / npix per view
                    r.silhouette_bce(tfin[sl], masks[t][sl], gradT[sl], sil_losses[t, k],
                                     weight=w_silhouette * n / npix)
                r.backward_l2(img[sl], targets[t][sl], losses[t, k], dv, dc, dop, accumulate=k > 0,
                              dL_dtfinal=gradT[sl] if use_sil else None)
                off += n
        if use_reg:
            r.mesh_regularizers(verts, faces, w_edge, w_laplacian, dverts=dv, losses=reg_losses[t])
        r.adam_step(verts, dv, m_v, v_v, lr, t + 1, group=gv, betas=betas, eps=eps)
        r.adam_step(rgb, dc, m_c, v_c, lr, t + 1, group=1, betas=betas, eps=eps)
        events[t][1].record()
        if between_steps is not None:
            between_steps()
    cd1 = r.chamfer(verts, tverts).sum()
    torch.cuda.synchronize()
    return {
        "loss": losses.sum(1).cpu().numpy(),
        "silhouette_loss": sil_losses.sum(1).cpu().numpy(),
        "regularizer_losses": reg_losses.cpu().numpy(),
        "ms": np.array([a.elapsed_time(b) for a, b in events]),
        "verts": verts,
        "rgb": rgb,
        "chamfer_initial": float(cd0),
        "chamfer_final": float(cd1),
        "pixels_per_step": npix,
        "status": r.device_status(),
    }
