"""Parity at the full sizes of the two largest workloads, on sampled pixels
the FP64 oracle computes one by one:

* 64 views of uneven resolution (256^2 ... 1024^2, 27.4 Mpixel) of a
  level-6 icosphere with value-noise face colours, in one batched call, with
  8x8, 16x16 and 32x32 tiles and the launch shapes the autotuner picks;
* 16 views of 1024^2 of a level-8 icosphere (1.31M faces) with Perlin
  displacement, in one batched call, with 16x16 and 8x8 tiles;

each also with the compositing kernels as persistent grids, in the
half-warp layout, in the warp-staged layout and in the autotuner's mix of
the two (warp-staged forward, half-warp backward).

Images: max abs error 1e-5 on pixels whose discrete decisions are not in the
ambiguity bands. Gradients: dL/dI is non-zero on the sampled pixels only, so
the oracle's backward over those pixels is the exact reference (relative L2
1e-4 per tensor)."""

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from gpu_util import DEV, GRAD_TOL, IMG_TOL, rel_l2, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


# launch shapes (tile, forward threads, backward threads[, persistent[,
# layout of both directions | forward layout, backward layout]]); layouts:
# 0 staging by the thread block, 1 half-warp, 2 staging by each warp. The
# autotuner's shapes: (16, 128, 128, 0, 2, 1) on the 64-view workload,
# (16, 128, 128, 0, 2, 0) on the ring, (8, 64, 32, 0, 2, 2) on the level-8 mesh.
BENCH_SHAPE = (16, 256, 128)
TUNED_SHAPE = (16, 128, 128, 0, 2, 1)


def _check(scene, shapes, n_random, window, seed):
    from paper_2602_14493_b300 import Renderer

    pix, lin = sample_pixels(scene.cams, n_random, seed, window=window)
    ref = oracle.render(scene, pixels=pix)
    amb = (ref["flags"] & (oracle.FLAG_ALPHA_SKIP | oracle.FLAG_TERMINATE)) != 0
    assert (~amb).sum() > 0.9 * len(pix)
    rng = np.random.default_rng(seed + 1)
    gs = rng.normal(size=(len(pix), 3))
    gs[ref["flags"] != 0] = 0.0
    ob = oracle.backward(scene, gs.astype(np.float32).astype(np.float64), pixels=pix)
    v, f, c, o = to_dev(scene)
    g = np.zeros((scene.n_pixels, 3), dtype=np.float32)
    g[lin] = gs
    g = torch.from_numpy(g).to(DEV)
    for shape in shapes:
        tile, threads, threads_bwd = shape[:3]
        persistent = len(shape) > 3 and bool(shape[3])
        lf = shape[4] if len(shape) > 4 else 0
        lb = shape[5] if len(shape) > 5 else lf
        r = Renderer(tile=tile, threads=threads, threads_bwd=threads_bwd, persistent=persistent, half_fwd=lf == 1,
                     half_bwd=lb == 1, warp_fwd=lf == 2, warp_bwd=lb == 2)
        img, T = r.forward(v, f, c, o, scene.cams)
        dv, dc, do = r.backward(g)
        torch.cuda.synchronize()
        err = np.abs(img.cpu().numpy()[lin] - ref["rgb"]).max(1)
        assert err[~amb].max() <= IMG_TOL, (tile, threads, float(err[~amb].max()))
        assert np.abs(T.cpu().numpy()[lin] - ref["T"])[~amb].max() <= IMG_TOL
        assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
        assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
        assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
        assert r.device_status() == 0
        r.close()


def test_fibonacci_64_uneven_views_full_size():
    s = gi.scene_fibonacci_uneven()
    assert len(s.cams) == 64 and s.n_pixels > 20_000_000
    _check(s, ((16, 128, 128), BENCH_SHAPE, (32, 256, 256), BENCH_SHAPE + (1,), BENCH_SHAPE + (0, 1),
               BENCH_SHAPE + (0, 2), TUNED_SHAPE, (16, 128, 128, 0, 2, 0), (8, 64, 64), (8, 32, 64, 0, 2),
               (8, 64, 32, 0, 2, 1)),
           n_random=256, window=4, seed=301)


def test_large_mesh_16_views_1024_full_size():
    s = gi.scene_large()
    assert len(s.faces) == 1_310_720 and s.n_pixels == 16 * 1024 * 1024
    _check(s, (BENCH_SHAPE, BENCH_SHAPE + (1,), BENCH_SHAPE + (0, 1), BENCH_SHAPE + (0, 2), TUNED_SHAPE, (8, 64, 64),
               (8, 64, 64, 0, 2), (8, 64, 32, 1), (8, 64, 32, 0, 2, 1), (8, 32, 64, 0, 1, 2), (8, 64, 32, 0, 2, 2)),
           n_random=128,
           window=4, seed=401)
