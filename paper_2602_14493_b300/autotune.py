"""Autotuner for the rasterizer's launch shape: tile size (8, 16 or 32),
threads per tile (forward and backward separately), Gaussians per
shared-memory batch, the compositing layout per direction, and whether the
compositing kernels run as persistent grids.

Every candidate renders the same forward + L2 loss + backward step; the
fastest (median of CUDA-event timings after warm-up) wins. Images do not
depend on the choice (the compositing order and arithmetic are the same for
all shapes), so tuning never changes results. Choices are cached in a JSON
file keyed by the workload signature (faces, views, resolution multiset).
"""

from __future__ import annotations

import hashlib
import json
import os
import statistics

import torch

# (tile, forward threads per tile, backward threads per tile, batch), full-warp
# layout, one CTA per tile
CANDIDATES = [(16, tf, tb, b) for tf in (256, 128, 64) for tb in (256, 128, 64) for b in (256, 128, 64)] + [
    (32, 256, 256, 256), (32, 256, 256, 128),
] + [(8, tf, tb, b) for tf in (64, 32) for tb in (64, 32) for b in (256, 128, 64)]
# threads per tile tried with the half-warp and warp-staged layouts
LAYOUT_THREADS = {8: (64, 32), 16: (128, 256), 32: (256,)}


# A shape is (tile, forward threads, backward threads, batch, persistent,
# forward layout, backward layout); layouts: 0 staging by the thread block,
# 1 half-warp, 2 staging by each warp.
LAYOUT_CTA, LAYOUT_HALF, LAYOUT_WARP = 0, 1, 2


def _full(shape):
    return tuple(shape) + (0,) * (7 - len(shape))


def _apply(renderer, shape):
    tile, threads, threads_bwd, batch, persistent, lf, lb = _full(shape)
    renderer.set_config(tile=tile, threads=threads, threads_bwd=threads_bwd, batch=batch, persistent=bool(persistent),
                        half_fwd=lf == LAYOUT_HALF, half_bwd=lb == LAYOUT_HALF, warp_fwd=lf == LAYOUT_WARP,
                        warp_bwd=lb == LAYOUT_WARP)


def shape_name(shape) -> str:
    return "x".join(str(x) for x in shape)


def cache_path() -> str:
    return os.environ.get("GMR_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gmr_b300_autotune.json"))


def signature(n_faces, cams) -> str:
    res = sorted((int(c["width"]) if not hasattr(c, "width") else int(c.width),
                  int(c["height"]) if not hasattr(c, "height") else int(c.height)) for c in cams)
    dev = torch.cuda.get_device_name()
    key = json.dumps([n_faces, len(res), res, dev])
    return hashlib.sha1(key.encode()).hexdigest()[:16]


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        with open(p + ".tmp", "w") as f:
            json.dump(d, f, indent=1)
        os.replace(p + ".tmp", p)
    except OSError:
        pass


def tune(renderer, verts, faces, rgb, opacity, cams, target, reps=15, candidates=CANDIDATES, use_cache=True):
    """Times each candidate shape on this workload with one CTA per tile;
    then, from the fastest of each tile size among 8 and 16, the half-warp
    and the warp-staged layouts in the forward and in the
    backward (each thread count of ``LAYOUT_THREADS``, separately, then the
    best of each direction together), and the fastest block-staged shape as a
    persistent grid; configures ``renderer`` with the fastest of all.
    Returns (best (tile, threads, threads_bwd, batch, persistent,
    forward layout, backward layout), {shape: median ms})."""
    sig = signature(faces.shape[0], cams)
    cache = _load() if use_cache else {}
    if use_cache and sig in cache and len(cache[sig]["best"]) == 7:
        best = tuple(cache[sig]["best"])
        _apply(renderer, best)
        return best, {}
    stream = torch.cuda.current_stream()
    img = torch.empty((target.shape[0], 3), device=verts.device)
    loss = torch.empty((), dtype=torch.float64, device=verts.device)
    dv, dc = torch.empty_like(verts), torch.empty_like(rgb)
    do = torch.empty_like(opacity) if opacity is not None else None
    results = {}

    def time_shape(shape):
        _apply(renderer, shape)
        ts = []
        for rep in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            renderer.forward(verts, faces, rgb, opacity, cams, images=img, want_t=False)
            renderer.backward_l2(img, target, loss, dv, dc, do)
            b.record(stream)
            b.synchronize()
            if rep >= 2:
                ts.append(a.elapsed_time(b))
        results[shape] = statistics.median(ts)

    for shape in candidates:
        time_shape(_full(shape[:4]))
    best_cta = min(results, key=results.get)
    for tile in (16, 8):
        of_tile = [k for k in results if k[0] == tile]
        if not of_tile:
            continue
        base = min(of_tile, key=results.get)
        _, tf, tb, batch = base[:4]
        layouts = [LAYOUT_HALF, LAYOUT_WARP]
        threads = LAYOUT_THREADS[tile]
        # the half-warp layout stages per batch: both larger batch sizes (the
        # warp-staged layout has no batch)
        batches = lambda lay: sorted({batch, 128, 256}) if lay == LAYOUT_HALF else [batch]
        fwd = [(tile, t, tb, b, 0, lay, 0) for lay in layouts for t in threads for b in batches(lay)]
        bwd = [(tile, tf, t, b, 0, 0, lay) for lay in layouts for t in threads for b in batches(lay)]
        for shape in fwd + bwd:
            time_shape(shape)
        bf = min(fwd + [base], key=results.get)
        bb = min(bwd + [base], key=results.get)
        if bf != base and bb != base:
            # one batch size for both directions: the backward's (it weighs more)
            time_shape((tile, bf[1], bb[2], bb[3], 0, bf[5], bb[6]))
    time_shape(tuple(best_cta[:4]) + (1, 0, 0))
    best = min(results, key=results.get)
    _apply(renderer, best)
    if use_cache:
        cache[sig] = {"best": list(best), "ms": {shape_name(k): v for k, v in results.items()}}
        _store(cache)
    return best, results
