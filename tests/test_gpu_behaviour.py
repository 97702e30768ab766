"""GPU behaviour beyond parity: invariances (tile size, batch size, batched
vs per-view), CUDA-graph capture, edge cases and error reporting (host-side
errors and device status words; nothing here faults or hangs a GPU)."""

import ctypes

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from gpu_util import DEV, GRAD_TOL, IMG_TOL, rel_l2, render_gpu, to_dev

pytestmark = pytest.mark.gpu


def _renderer(**kw):
    from paper_2602_14493_b300 import Renderer

    return Renderer(**kw)


def _uneven():
    v, f = gi.icosphere(4)
    rng = np.random.default_rng(5)
    cams = gi.fibonacci_cameras(6, 3.0, [(256, 256), (384, 384), (100, 37), (512, 512), (33, 65), (128, 128)])
    return gi.Scene("uneven4", v.astype(np.float32), f, rng.random((len(f), 3)).astype(np.float32),
                    np.full(len(f), 0.9, np.float32), cams)


def test_image_invariant_to_tile_and_batch_size():
    """Every launch shape, the half-warp layout included, takes the same
    decisions with the same arithmetic per pixel: identical images."""
    s = _uneven()
    ref = None
    for tile, threads, lay in ((16, 256, 0), (16, 128, 0), (16, 64, 0), (32, 256, 0), (8, 64, 0), (8, 32, 0),
                               (16, 256, 1), (16, 128, 1), (8, 64, 1), (8, 32, 1), (16, 256, 2), (16, 128, 2),
                               (16, 64, 2), (32, 256, 2), (8, 64, 2), (8, 32, 2)):
        for batch in (64, 128, 256):
            r = _renderer(tile=tile, batch=batch, threads=threads, half_fwd=lay == 1, warp_fwd=lay == 2)
            _, img, T = render_gpu(r, s)
            a = img.cpu().numpy()
            if ref is None:
                ref = a
            else:
                np.testing.assert_array_equal(a, ref)
            r.close()


def test_gradients_invariant_to_backward_shape():
    """The backward's launch shape (the half-warp layout included) changes
    only the order of the float atomics, so gradients agree to rounding
    across all shapes."""
    s = _uneven()
    ref = None
    for tile, threads_bwd, lay in ((16, 256, 0), (16, 128, 0), (16, 64, 0), (32, 256, 0), (8, 64, 0), (8, 32, 0),
                                   (16, 256, 1), (16, 128, 1), (8, 64, 1), (8, 32, 1), (16, 256, 2), (16, 128, 2),
                                   (16, 64, 2), (32, 256, 2), (8, 64, 2), (8, 32, 2)):
        for batch in (64, 256):
            r = _renderer(tile=tile, batch=batch, threads=64 if tile == 8 else 256, threads_bwd=threads_bwd,
                          half_bwd=lay == 1, warp_bwd=lay == 2)
            _, img, T = render_gpu(r, s)
            g = torch.sin(torch.arange(img.numel(), device=DEV, dtype=torch.float32)).reshape(img.shape)
            got = [x.cpu().numpy().copy() for x in r.backward(g.contiguous())]
            if ref is None:
                ref = got
            else:
                for a, b in zip(got, ref):
                    assert rel_l2(a, b) < 1e-5
            r.close()


@pytest.mark.parametrize("n", [1, 4095, 4096, 3 * 100003, 1 << 22])
def test_l2_loss_against_fp64(n):
    """gmr_l2_loss on ragged sizes (partial blocks, unaligned tails): the
    gradient 2 (img - target) bit for bit (the same two FP32 roundings as
    NumPy), the loss within its stated 1.3e-6 relative of the FP64 sum."""
    from paper_2602_14493_b300 import Renderer

    rng = np.random.default_rng(n)
    a = rng.random(n, dtype=np.float32)
    b = rng.random(n, dtype=np.float32)
    r = Renderer()
    loss, grad = r.l2_loss(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV))
    d = a - b
    np.testing.assert_array_equal(grad.cpu().numpy(), np.float32(2.0) * d)
    ref = float(np.sum(d.astype(np.float64) ** 2))
    assert abs(float(loss) - ref) <= 1.3e-6 * ref
    r.close()


def test_fused_forward_loss_matches_separate():
    """gmr_render_fwd_l2: same image, the same dL/dI bit for bit, and the
    same loss up to the FP32 rounding of the per-thread partial sums as
    gmr_render_fwd + gmr_l2_loss; twice in a row, on views of uneven
    sizes, in the block-staged, warp-staged and half-warp forward layouts."""
    s = _uneven()
    shapes = [dict(tile=t, threads=n) for t, n in ((16, 256), (16, 128), (32, 256), (8, 64), (8, 32))]
    shapes += [dict(tile=16, threads=128, warp_fwd=True), dict(tile=16, threads=256, half_fwd=True),
               dict(tile=8, threads=64, warp_fwd=True), dict(tile=8, threads=32, half_fwd=True)]
    for kw in shapes:
        r = _renderer(**kw)
        (v, f, c, o), img, T = render_gpu(r, s)
        img = img.clone()
        target = torch.rand_like(img)
        loss, grad = r.l2_loss(img, target)
        grad, loss = grad.clone(), float(loss)
        for _ in range(2):
            img2, grad2, loss2 = r.forward_l2(v, f, c, o, s.cams, target)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(img2.cpu().numpy(), img.cpu().numpy())
            np.testing.assert_array_equal(grad2.cpu().numpy(), grad.cpu().numpy())
            # FP32 sums of <= 16 squares per thread and a 5-level FP32 warp
            # tree on both sides: each within 21 u = 1.3e-6 relative
            assert abs(float(loss2) - loss) <= 2.6e-6 * abs(loss)
        # the backward after the fused forward matches the one after the plain forward
        dv2 = r.backward(grad2)[0].clone()
        r.forward(v, f, c, o, s.cams)
        dv1 = r.backward(grad)[0].clone()
        assert rel_l2(dv2.cpu().numpy(), dv1.cpu().numpy()) < 1e-5
        r.close()


def test_backward_with_fused_loss_matches_separate():
    """gmr_render_bwd_l2 (the loss formed in the compositing backward): the
    same gradients as gmr_l2_loss + gmr_render_bwd up to the order of the
    float atomics, the same loss up to the FP32 partial sums, on views of
    uneven sizes, for every backward shape and layout, also with
    dL/dT_final."""
    s = _uneven()
    shapes = [dict(tile=t, threads=n) for t, n in ((16, 128), (16, 256), (16, 64), (32, 256), (8, 64), (8, 32))]
    shapes += [dict(tile=16, threads_bwd=128, half_bwd=True), dict(tile=16, threads_bwd=256, half_bwd=True),
               dict(tile=16, threads_bwd=128, warp_bwd=True), dict(tile=8, threads_bwd=32, warp_bwd=True),
               dict(tile=8, threads_bwd=32, half_bwd=True), dict(tile=8, threads_bwd=64, half_bwd=True)]
    for kw in shapes:
        r = _renderer(**kw)
        (v, f, c, o), img, T = render_gpu(r, s)
        img, T = img.clone(), T.clone()
        target = torch.rand_like(img)
        loss, grad = r.l2_loss(img, target)
        loss = float(loss)
        ref = [t.clone() for t in r.backward(grad)]
        gT = torch.randn_like(T) * 1e-3
        ref_t = [t.clone() for t in r.backward(grad, dL_dtfinal=gT)]
        for _ in range(2):
            loss2, dv, dc, do = r.backward_l2(img, target)
            torch.cuda.synchronize()
            assert abs(float(loss2) - loss) <= 2.6e-6 * abs(loss)
            for a, b in zip((dv, dc, do), ref):
                assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
        _, dv, dc, do = r.backward_l2(img, target, dL_dtfinal=gT)
        for a, b in zip((dv, dc, do), ref_t):
            assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
        # accumulate adds to the given gradients
        _, dv2, _, _ = r.backward_l2(img, target, dverts=dv.clone(), accumulate=True)
        assert rel_l2(dv2.cpu().numpy(), dv.cpu().numpy() + ref[0].cpu().numpy()) < 1e-6
        r.close()


def test_batched_equals_per_view():
    s = _uneven()
    r = _renderer()
    (v, f, c, o), img, T = render_gpu(r, s)
    g = torch.randn_like(img)
    dv, dc, do = r.backward(g)
    dv, dc, do = dv.clone(), dc.clone(), do.clone()
    off = oracle.pixel_offsets(s.cams)
    dv2 = torch.zeros_like(dv)
    dc2 = torch.zeros_like(dc)
    do2 = torch.zeros_like(do)
    for k in range(len(s.cams)):
        im1, _ = r.forward(v, f, c, o, s.cams[k:k + 1])
        np.testing.assert_array_equal(im1.cpu().numpy(), img[off[k]:off[k + 1]].cpu().numpy())
        r.backward(g[off[k]:off[k + 1]].contiguous(), dv2, dc2, do2, accumulate=True)
    torch.cuda.synchronize()
    assert rel_l2(dv2.cpu().numpy(), dv.cpu().numpy()) < 1e-5
    assert rel_l2(dc2.cpu().numpy(), dc.cpu().numpy()) < 1e-5
    assert rel_l2(do2.cpu().numpy(), do.cpu().numpy()) < 1e-5
    r.close()


def test_cuda_graph_capture_replays_fwd_loss_bwd():
    s = gi.scene_ring(level=4, n_views=4, res=256)
    r = _renderer(sync_check=True)
    v, f, c, o = to_dev(s)
    target = torch.rand((s.n_pixels, 3), device=DEV)
    img0, _ = r.forward(v, f, c, o, s.cams)
    P = r.stats()["n_pairs"]
    r.set_config(sync_check=False)
    r.reserve(len(s.faces), len(s.cams), s.n_pixels, int(P * 1.5) + 1024)
    cams = __import__("paper_2602_14493_b300").camera_array(s.cams)
    img = torch.empty((s.n_pixels, 3), device=DEV)
    dv = torch.empty_like(v)
    dc = torch.empty_like(c)
    do = torch.empty_like(o)
    grad = torch.empty_like(img)
    loss = torch.empty((), dtype=torch.float64, device=DEV)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # eager warm-up on the capture stream (uploads the camera table)
        r.forward(v, f, c, o, cams, images=img, want_t=False, stream=stream)
        r.l2_loss(img, target, grad, loss, stream=stream)
        r.backward(grad, dv, dc, do, stream=stream)
    stream.synchronize()
    eager = (img.clone(), dv.clone(), dc.clone(), do.clone(), loss.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        r.forward(v, f, c, o, cams, images=img, want_t=False, stream=stream)
        r.l2_loss(img, target, grad, loss, stream=stream)
        r.backward(grad, dv, dc, do, stream=stream)
    for _ in range(3):
        img.zero_(); dv.zero_()
        graph.replay()
    torch.cuda.synchronize()
    assert r.device_status() == 0
    np.testing.assert_array_equal(img.cpu().numpy(), eager[0].cpu().numpy())
    np.testing.assert_array_equal(img.cpu().numpy(), img0.cpu().numpy())
    assert rel_l2(dv.cpu().numpy(), eager[1].cpu().numpy()) < 1e-5
    assert abs(float(loss) - float(eager[4])) <= 1e-9 * abs(float(eager[4]))
    r.close()


def test_repeated_and_separately_captured_backwards_start_from_zero():
    """The forward zeroes the backward's gradient sums; a second backward
    after one forward, and a backward captured alone and replayed, must
    clear them themselves (same gradients every time)."""
    s = gi.scene_ring(level=4, n_views=4, res=256)
    r = _renderer()
    v, f, c, o = to_dev(s)
    g = torch.rand((s.n_pixels, 3), device=DEV) - 0.5
    img, _ = r.forward(v, f, c, o, s.cams)
    outs = []
    for _ in range(3):  # three backwards after one forward
        dv, dc, do = torch.empty_like(v), torch.empty_like(c), torch.empty_like(o)
        r.backward(g, dv, dc, do)
        outs.append((dv.cpu().numpy(), dc.cpu().numpy(), do.cpu().numpy()))
    # equal up to the order of the float atomics (a sum left over from the
    # previous backward would double them: relative L2 distance ~1)
    for k in range(1, 3):
        for a, b in zip(outs[0], outs[k]):
            assert rel_l2(a, b) < 1e-5
    # forward eager, backward alone in a graph, replayed several times
    P = r.stats()["n_pairs"]
    r.reserve(len(s.faces), len(s.cams), s.n_pixels, int(P * 1.5) + 1024)
    cams = __import__("paper_2602_14493_b300").camera_array(s.cams)
    stream = torch.cuda.Stream()
    img2 = torch.empty_like(img)
    dv, dc, do = torch.empty_like(v), torch.empty_like(c), torch.empty_like(o)
    with torch.cuda.stream(stream):
        r.forward(v, f, c, o, cams, images=img2, want_t=False, stream=stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        r.backward(g, dv, dc, do, stream=stream)
    for _ in range(3):
        graph.replay()
        torch.cuda.synchronize()
        assert rel_l2(dv.cpu().numpy(), outs[0][0]) < 1e-5
        assert rel_l2(dc.cpu().numpy(), outs[0][1]) < 1e-5
    assert r.device_status() == 0
    r.close()


def test_empty_mesh_and_offscreen_views_render_background():
    r = _renderer(bg=(0.25, 0.5, 0.75))
    s = gi.scene_single_view(level=1, width=40, height=24)
    v, f, c, o = to_dev(s)
    img, T = r.forward(v, f[:0].contiguous(), c[:0].contiguous(), o[:0].contiguous(), s.cams)
    torch.cuda.synchronize()
    np.testing.assert_allclose(img.cpu().numpy(), np.tile([0.25, 0.5, 0.75], (40 * 24, 1)), atol=0)
    assert np.all(T.cpu().numpy() == 1.0)
    dv, dc, do = r.backward(torch.ones_like(img))
    # camera looking away from the mesh
    cam = gi.look_at((0.0, 0.0, 3.0), 31, 17, target=(0.0, 0.0, 10.0))
    cams = np.array([cam], dtype=gi.CAMERA_DTYPE)
    img, T = r.forward(v, f, c, o, cams)
    torch.cuda.synchronize()
    assert np.all(T.cpu().numpy() == 1.0)
    dv, dc, do = r.backward(torch.ones_like(img))
    torch.cuda.synchronize()
    assert float(dv.abs().max()) == 0.0
    assert r.device_status() == 0
    r.close()


def test_tiny_and_degenerate_inputs_match_oracle():
    r = _renderer()
    # one facet; a collinear (zero-area) facet; a facet behind the camera
    cams = gi.ring_cameras(2, 10.0, 2.5, 9, 13)
    v = np.array([[0, 0, 0], [0.3, 0, 0.1], [0, 0.25, 0.2],
                  [0.1, 0.1, 0.1], [0.2, 0.2, 0.2], [0.3, 0.3, 0.3],
                  [0, 0, 9], [0.1, 0, 9], [0, 0.1, 9]], dtype=np.float32)
    faces = np.arange(9, dtype=np.int32).reshape(3, 3)
    s = gi.Scene("tiny", v, faces, np.random.default_rng(0).random((3, 3)).astype(np.float32),
                 np.array([0.8, 0.9, 1.0], np.float32), cams)
    _, img, T = render_gpu(r, s)
    ref = oracle.render(s)
    ok = ref["flags"] == 0
    assert np.abs(img.cpu().numpy() - ref["rgb"]).max(1)[ok].max() <= IMG_TOL
    g = np.random.default_rng(1).normal(size=ref["rgb"].shape).astype(np.float32)
    g[~ok] = 0
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV))
    ob = oracle.backward(s, g.astype(np.float64))
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    r.close()


def test_host_side_argument_errors():
    from paper_2602_14493_b300 import GmrError, _lib

    r = _renderer()
    for bad in (dict(tile=32, threads=256, threads_bwd=256, half_fwd=True), dict(threads=64, half_fwd=True),
                dict(tile=8, threads=64, threads_bwd=32, half_bwd=True, persistent=True),
                dict(threads_bwd=64, half_bwd=True), dict(persistent=True, half_bwd=True),
                dict(persistent=True, warp_fwd=True), dict(half_fwd=True, warp_fwd=True)):
        with pytest.raises(GmrError):
            r.set_config(**bad)
        r.set_config(tile=16, threads=128, threads_bwd=128, half_fwd=False, half_bwd=False, warp_fwd=False,
                     warp_bwd=False, persistent=False)
    s = gi.scene_single_view(level=1, width=16, height=16)
    v, f, c, o = to_dev(s)
    # backward before any forward
    st = r._L.gmr_render_bwd(r._ctx, ctypes.c_void_p(torch.zeros(3, device=DEV).data_ptr()), None, None, None, 0, None)
    assert st == 6  # GMR_ERR_STATE
    with pytest.raises(GmrError):
        r.set_config(tile=12)
    with pytest.raises(GmrError):
        r.set_config(tile=8, threads=128, threads_bwd=64)
    r.set_config(tile=16, threads=128, threads_bwd=128)
    with pytest.raises(GmrError):
        r.set_config(batch=100)
    assert r.cfg.batch == 256  # a refused change leaves the configuration as it was
    bad = s.cams.copy()
    bad[0]["width"] = 0
    with pytest.raises(GmrError):
        r.forward(v, f, c, o, bad)
    L = r._L
    assert L.gmr_render_fwd(r._ctx, None, 5, None, 3, None, None, None, 1, None, None, None) == 1
    # size limits of the packed formats, refused on the host before any
    # device work (the device pointers below are never read)
    from paper_2602_14493_b300 import camera_array

    img = torch.zeros(16 * 16 * 3, device=DEV)
    p = [ctypes.c_void_p(t.data_ptr()) for t in (v, f, c, img)]

    def fwd(cams, F=len(s.faces), C=None):
        C = len(cams) if C is None else C
        return L.gmr_render_fwd(r._ctx, p[0], len(s.verts), p[1], F, p[2], None, camera_array(cams), C, p[3], None,
                                None)

    assert fwd(s.cams) == 0
    cams8 = np.repeat(s.cams, 8)
    assert fwd(cams8, F=1 << 28) == 1                    # views x faces >= 2^31
    assert fwd(s.cams, C=70000) == 1                     # more than 65535 views
    wide = s.cams.copy()
    wide[0]["width"] = (1 << 20) + 1                     # a side beyond 2^20 pixels
    assert fwd(wide) == 1
    r.set_config(tile=8, threads=64, threads_bwd=64)
    wide[0]["width"] = 1 << 20                           # 131,072 tiles of 8 px across
    assert fwd(wide) == 1
    nan = s.cams.copy()
    nan["R"][0, 4] = np.nan                              # a non-finite camera
    assert fwd(nan) == 1
    torch.cuda.synchronize()
    r.close()


def test_device_status_bad_face_and_pair_overflow():
    r = _renderer()
    s = gi.scene_single_view(level=4, width=256, height=256)
    v, f, c, o = to_dev(s)
    fb = f.clone()
    fb[3, 1] = 10 ** 6
    img, T = r.forward(v, fb, c, o, s.cams)
    torch.cuda.synchronize()
    assert r.device_status() & 1
    assert r.device_status() == 0  # cleared by the read
    # no-sync mode with a pair buffer that is too small: reported, no fault
    r2 = _renderer(sync_check=False)
    r2.reserve(len(s.faces), 1, 256 * 256, 16)
    img, T = r2.forward(v, f, c, o, s.cams)
    torch.cuda.synchronize()
    assert r2.device_status() & 2
    r2.close()
    r.close()


def test_stats_and_launch_count():
    r = _renderer()
    s = gi.scene_single_view()
    (v, f, c, o), img, T = render_gpu(r, s)
    st0 = r.stats()
    r.backward(torch.ones_like(img))
    st = r.stats()
    assert st["n_pairs"] == len(oracle.sorted_pairs(s.verts, s.faces, s.cams, 16)[0])
    assert st["n_pixels"] == 128 * 128 and st["n_tiles"] == 64
    assert st["evals_fwd"] > 0 and st["evals_bwd"] > 0
    assert st["launches"] > st0["launches"] >= 6
    # the workspace holds at least the per-record buffers (80 B per record)
    assert st["workspace_bytes"] >= 80 * st["n_records"]
    r.close()


def test_copy_h2d_kernel_copy():
    """gmr_copy_h2d: bytes equal after the copy for sizes with and without a
    16-byte tail, for offset (unaligned) views and from 64 MiB up (the copy
    engine's path); a pageable source is refused before anything is
    launched."""
    from paper_2602_14493_b300 import GmrError, copy_h2d

    rng = np.random.default_rng(5)
    for nbytes in (1, 15, 16, 17, 4096, 1 << 20, (25 << 20) + 12, (64 << 20) + 5):
        src = torch.from_numpy(rng.integers(0, 256, nbytes, dtype=np.uint8)).pin_memory()
        dst = torch.zeros(nbytes, dtype=torch.uint8, device=DEV)
        copy_h2d(dst, src)
        torch.cuda.synchronize()
        assert torch.equal(dst.cpu(), src)
    big = torch.from_numpy(rng.integers(0, 256, 1 << 16, dtype=np.uint8)).pin_memory()
    dst = torch.zeros(1 << 16, dtype=torch.uint8, device=DEV)
    copy_h2d(dst[3:1003], big[7:1007])  # both views unaligned: the byte path
    torch.cuda.synchronize()
    assert torch.equal(dst[3:1003].cpu(), big[7:1007]) and int(dst[:3].sum()) == 0
    with pytest.raises(GmrError):
        copy_h2d(torch.zeros(64, dtype=torch.uint8, device=DEV), torch.zeros(64, dtype=torch.uint8))
    # the library itself refuses pageable memory (no launch)
    import ctypes

    from paper_2602_14493_b300 import _lib

    pageable = torch.zeros(64, dtype=torch.uint8)
    d64 = torch.zeros(64, dtype=torch.uint8, device=DEV)
    st = _lib.load().gmr_copy_h2d(ctypes.c_void_p(d64.data_ptr()), ctypes.c_void_p(pageable.data_ptr()), 64,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1  # GMR_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(16, 128, 128), (16, 256, 128), (16, 64, 256), (32, 256, 256), (8, 64, 32)])
def test_persistent_grid_matches_per_tile_grid(shape):
    """The compositing kernels as persistent grids (resident CTAs taking
    tiles from a counter) give the same images and final T bit for bit and
    the same gradients up to the order of the float atomics, also for a
    second forward and a second backward (each must start its counter
    again)."""
    tile, threads, threads_bwd = shape
    s = _uneven()
    g = torch.sin(torch.arange(s.n_pixels * 3, device=DEV, dtype=torch.float32)).reshape(-1, 3).contiguous()
    outs = {}
    for persistent in (False, True):
        r = _renderer(tile=tile, threads=threads, threads_bwd=threads_bwd, persistent=persistent)
        v, f, c, o = to_dev(s)
        res = []
        for _ in range(2):  # two forwards, each with two backwards
            img, T = r.forward(v, f, c, o, s.cams)
            for _ in range(2):
                dv, dc, do = r.backward(g)
                res.append((img.cpu().numpy().copy(), T.cpu().numpy().copy(), dv.cpu().numpy().copy(),
                            dc.cpu().numpy().copy(), do.cpu().numpy().copy()))
        assert r.device_status() == 0
        outs[persistent] = res
        r.close()
    ref = outs[False][0]
    for res in (outs[False], outs[True]):
        for img, T, dv, dc, do in res:
            np.testing.assert_array_equal(img, ref[0])
            np.testing.assert_array_equal(T, ref[1])
            assert rel_l2(dv, ref[2]) < 1e-5
            assert rel_l2(dc, ref[3]) < 1e-5
            assert rel_l2(do, ref[4]) < 1e-5


def test_inplace_modification_between_forward_and_backward_raises():
    from paper_2602_14493_b300 import GmrError

    r = _renderer()
    s = gi.scene_single_view(level=2, width=32, height=32)
    v, f, c, o = to_dev(s)
    img, _ = r.forward(v, f, c, o, s.cams)
    r.backward(torch.ones_like(img))  # unchanged inputs: fine
    v.add_(0.01)  # e.g. an optimiser step taken before the backward
    with pytest.raises(GmrError, match="verts"):
        r.backward(torch.ones_like(img))
    img, _ = r.forward(v, f, c, o, s.cams)
    c.mul_(0.5)
    with pytest.raises(GmrError, match="rgb"):
        r.backward_l2(img, torch.zeros_like(img))
    r.close()


def test_workspace_limit_returns_oom_and_context_recovers():
    """GMR_ERR_OOM without exhausting the device: a workspace cap below what
    the forward needs fails the call before anything is enqueued; with the
    cap lifted the same context renders the reference image."""
    from paper_2602_14493_b300 import GmrError

    s = gi.scene_single_view(level=3, width=96, height=64)
    v, f, c, o = to_dev(s)
    ref = _renderer()
    img_ref, _ = ref.forward(v, f, c, o, s.cams)
    torch.cuda.synchronize()
    need = ref.stats()["workspace_bytes"]
    ref.close()
    r = _renderer()
    r.set_workspace_limit(need // 4)
    with pytest.raises(GmrError, match="GMR_ERR_OOM"):
        r.forward(v, f, c, o, s.cams)
    with pytest.raises(GmrError, match="GMR_ERR_OOM"):
        r.reserve(len(s.faces), 1, s.n_pixels, 10 ** 6)
    assert r.stats()["workspace_bytes"] <= need // 4
    r.set_workspace_limit(0)
    img, _ = r.forward(v, f, c, o, s.cams)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(img.cpu().numpy(), img_ref.cpu().numpy())
    assert r.device_status() == 0
    r.close()


def test_nonfinite_vertices_are_culled_and_match_oracle():
    """Faces with a NaN or infinite vertex fail the binning's finiteness test
    (they reach no tile): the rest of the image matches the oracle, the
    device status stays clear, and every gradient is finite (exactly zero
    for the non-finite vertices)."""
    s = gi.scene_single_view(level=3, width=96, height=80)
    verts = s.verts.copy()
    bad = [0, 17, 101, 300]
    verts[bad[0]] = np.nan
    verts[bad[1], 2] = np.inf
    verts[bad[2], 0] = -np.inf
    verts[bad[3], 1] = np.nan
    s = gi.Scene(s.name, verts, s.faces, s.rgb, s.opacity, s.cams)
    r = _renderer()
    (v, f, c, o), img, T = render_gpu(r, s)
    ref = oracle.render(s)
    amb = (ref["flags"] & 3) != 0
    assert np.isfinite(img.cpu().numpy()).all()
    assert np.abs(img.cpu().numpy() - ref["rgb"])[~amb].max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T"])[~amb].max() <= IMG_TOL
    nb = r.stats()
    assert nb["n_pairs"] > 0
    gs = np.random.default_rng(3).normal(size=(s.n_pixels, 3))
    gs[ref["flags"] != 0] = 0.0
    dv, dc, do = r.backward(torch.from_numpy(gs.astype(np.float32)).to(DEV))
    torch.cuda.synchronize()
    assert r.device_status() == 0
    ob = oracle.backward(s, gs.astype(np.float32).astype(np.float64))
    dvn = dv.cpu().numpy()
    assert np.isfinite(dvn).all() and np.isfinite(dc.cpu().numpy()).all() and np.isfinite(do.cpu().numpy()).all()
    assert np.isfinite(ob["dverts"]).all()
    np.testing.assert_array_equal(dvn[bad], 0.0)
    np.testing.assert_array_equal(ob["dverts"][bad], 0.0)
    assert rel_l2(dvn, ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    r.close()


def test_view_beyond_2_31_pixels_matches_oracle():
    """A single 50,000 x 46,000 view (2.3G pixels: packed pixel indices past
    2^31 in its bottom 3,050 rows, image element indices past 2^32), the
    sphere placed low in the view so that those rows cover it: the image,
    the final transmittance and the gradients match the oracle at sampled
    pixels on both sides of 2^31, in the default and the benchmark's launch
    shape. About 120 GB of device memory."""
    from paper_2602_14493_b300 import Renderer

    W, H = 50_000, 46_000
    v, f = gi.icosphere(2)
    rng = np.random.default_rng(231)
    cam = gi.look_at((3.0, 0.0, 0.0), W, H, target=(0.0, 0.0, 0.8))
    s = gi.Scene("sphere2_50000x46000", v.astype(np.float32), f, rng.random((len(f), 3)).astype(np.float32),
                 np.full(len(f), 0.9, np.float32), np.array([cam]))
    assert s.n_pixels > 2 ** 31
    xs = rng.integers(0, W, 96)
    ys = np.concatenate([rng.integers(0, H, 48), rng.integers(43_000, H, 48)])
    win_y, win_x = np.meshgrid(np.arange(45_000, 45_008), np.arange(24_996, 25_004), indexing="ij")
    pix = np.concatenate([np.stack([np.zeros(96, int), xs, ys], 1),
                          np.stack([np.zeros(64, int), win_x.ravel(), win_y.ravel()], 1),
                          [[0, W - 1, H - 1], [0, 0, H - 1]]]).astype(np.int32)
    pix = np.unique(pix, axis=0)
    lin = pix[:, 2].astype(np.int64) * W + pix[:, 1]
    assert (lin >= 2 ** 31).sum() >= 60
    ref = oracle.render(s, pixels=pix)
    amb = (ref["flags"] & (oracle.FLAG_ALPHA_SKIP | oracle.FLAG_TERMINATE)) != 0
    inside = ref["n_contrib"] > 0
    assert inside[lin >= 2 ** 31].sum() >= 30  # the sphere covers pixels past 2^31
    gs = rng.normal(size=(len(pix), 3))
    gs[ref["flags"] != 0] = 0.0
    ob = oracle.backward(s, gs.astype(np.float32).astype(np.float64), pixels=pix)
    vd, fd, cd, od = to_dev(s)
    lin_t = torch.from_numpy(lin).to(DEV)
    for shape in ({}, dict(threads=128, threads_bwd=128, warp_fwd=True, half_bwd=True)):
        r = Renderer(**shape)
        img, T = r.forward(vd, fd, cd, od, s.cams)
        g = torch.zeros_like(img)
        g[lin_t] = torch.from_numpy(gs.astype(np.float32)).to(DEV)
        dv, dc, do = r.backward(g)
        torch.cuda.synchronize()
        err = np.abs(img[lin_t].cpu().numpy() - ref["rgb"]).max(1)
        assert err[~amb].max() <= IMG_TOL, (shape, float(err[~amb].max()))
        assert np.abs(T[lin_t].cpu().numpy() - ref["T"])[~amb].max() <= IMG_TOL
        assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
        assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
        assert r.device_status() == 0
        del img, T, g
        r.close()
        torch.cuda.empty_cache()
