"""Shared helpers of the GPU tests: move a synthetic scene to the device,
render it through the C ABI, compare with the oracle."""

import numpy as np
import torch

import oracle

DEV = torch.device("cuda:0")

# Parity bars: FP32 images vs the FP64 oracle (max abs over pixels whose
# discrete decisions are not within the ambiguity bands), gradients as
# relative L2 per tensor.
IMG_TOL = 1e-5
GRAD_TOL = 1e-4


def to_dev(scene, rgb=None):
    v = torch.from_numpy(np.ascontiguousarray(scene.verts)).to(DEV)
    f = torch.from_numpy(np.ascontiguousarray(scene.faces)).to(DEV)
    c = torch.from_numpy(np.ascontiguousarray(scene.rgb if rgb is None else rgb)).to(DEV)
    o = torch.from_numpy(np.ascontiguousarray(scene.opacity)).to(DEV) if scene.opacity is not None else None
    return v, f, c, o


def render_gpu(renderer, scene, rgb=None):
    v, f, c, o = to_dev(scene, rgb)
    img, T = renderer.forward(v, f, c, o, scene.cams)
    torch.cuda.synchronize()
    return (v, f, c, o), img, T


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def sample_pixels(cams, n, seed, window=16):
    """n random pixels over all views plus one full window x window block at
    the centre of each view."""
    rng = np.random.default_rng(seed)
    off = oracle.pixel_offsets(cams)
    out = []
    for c, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        k = max(1, n // len(cams))
        xs = rng.integers(0, W, k)
        ys = rng.integers(0, H, k)
        out.append(np.stack([np.full(k, c), xs, ys], 1))
        x0, y0 = W // 2 - window // 2, H // 2 - window // 2
        yy, xx = np.meshgrid(np.arange(y0, y0 + window), np.arange(x0, x0 + window), indexing="ij")
        out.append(np.stack([np.full(window * window, c), xx.ravel(), yy.ravel()], 1))
    pix = np.concatenate(out, 0).astype(np.int32)
    pix = np.unique(pix, axis=0)
    lin = off[pix[:, 0]] + pix[:, 2] * np.array([int(cams[c]["width"]) for c in pix[:, 0]]) + pix[:, 1]
    return np.ascontiguousarray(pix), lin
