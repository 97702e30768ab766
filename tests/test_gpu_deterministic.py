"""The deterministic backward (GMR_FLAG_DETERMINISTIC): every gradient sum in
a fixed order, so a repeated backward (and the same backward in a second
context) gives the same gradients bit for bit; they agree with the
float-atomic backward to rounding and with the FP64 oracle within the parity
bar; images do not change. Covers every tile size, the colour modes, the
fused loss, persistent grids, accumulation, and a mesh with a vertex of high
degree (the incidence list's long-list sort)."""

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from gpu_util import DEV, GRAD_TOL, rel_l2, render_gpu, to_dev

pytestmark = pytest.mark.gpu


def _scene():
    v, f = gi.icosphere(4)
    rng = np.random.default_rng(9)
    cams = gi.fibonacci_cameras(6, 3.0, [(256, 256), (200, 120), (64, 200), (17, 5), (384, 384), (96, 96)])
    return gi.Scene("det", v.astype(np.float32), f, rng.random((len(f), 3)).astype(np.float32),
                    rng.uniform(0.3, 1.0, len(f)).astype(np.float32), cams)


def _renderer(**kw):
    from paper_2602_14493_b300 import Renderer

    return Renderer(**kw)


def _grads(r, s, g, rgb=None, repeats=2):
    """Gradients of `repeats` backwards after one forward, and of one more
    forward + backward, as numpy arrays."""
    v, f, c, o = to_dev(s, rgb)
    out = []
    for fwd in range(2):
        img, T = r.forward(v, f, c, o, s.cams)
        for _ in range(repeats if fwd == 0 else 1):
            res = r.backward(g)
            out.append([x.cpu().numpy().copy() for x in res])
    return img.cpu().numpy().copy(), out


@pytest.mark.parametrize("shape", [(16, 128, 128, 256), (16, 256, 256, 128), (16, 64, 64, 64), (32, 256, 256, 128),
                                   (8, 64, 64, 128), (8, 32, 32, 64)])
def test_repeated_backward_bit_identical(shape):
    tile, tf, tb, batch = shape
    s = _scene()
    g = torch.sin(torch.arange(s.n_pixels * 3, device=DEV, dtype=torch.float32)).reshape(-1, 3).contiguous()
    r = _renderer(tile=tile, threads=tf, threads_bwd=tb, batch=batch, deterministic=True, bg=(0.2, 0.1, 0.4))
    img, out = _grads(r, s, g)
    assert r.device_status() == 0
    r.close()
    for res in out[1:]:
        for a, b in zip(res, out[0]):
            np.testing.assert_array_equal(a, b)
    assert np.abs(out[0][0]).sum() > 0
    # a second context: the same bits
    r2 = _renderer(tile=tile, threads=tf, threads_bwd=tb, batch=batch, deterministic=True, bg=(0.2, 0.1, 0.4))
    img2, out2 = _grads(r2, s, g, repeats=1)
    r2.close()
    np.testing.assert_array_equal(img2, img)
    for a, b in zip(out2[0], out[0]):
        np.testing.assert_array_equal(a, b)
    # the float-atomic backward: same image, gradients to rounding
    r3 = _renderer(tile=tile, threads=tf, threads_bwd=tb, batch=batch, bg=(0.2, 0.1, 0.4))
    img3, out3 = _grads(r3, s, g, repeats=1)
    r3.close()
    np.testing.assert_array_equal(img3, img)
    for a, b in zip(out3[0], out[0]):
        assert rel_l2(a, b) < 1e-5


def test_matches_oracle():
    s = _scene()
    ref = oracle.render(s, bg=(0.2, 0.1, 0.4))
    rng = np.random.default_rng(12)
    gn = rng.normal(size=ref["rgb"].shape).astype(np.float32)
    gn[ref["flags"] != 0] = 0.0
    ob = oracle.backward(s, gn.astype(np.float64), bg=(0.2, 0.1, 0.4))
    r = _renderer(deterministic=True, bg=(0.2, 0.1, 0.4), persistent=True)
    render_gpu(r, s)
    dv, dc, do = r.backward(torch.from_numpy(gn).to(DEV))
    torch.cuda.synchronize()
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    r.close()


@pytest.mark.parametrize("color_mode", ["vertex", "sh"])
def test_colour_modes(color_mode):
    s = _scene()
    rng = np.random.default_rng(4)
    if color_mode == "vertex":
        rgb = rng.random((len(s.verts), 3)).astype(np.float32)
        kw = {}
    else:
        rgb = rng.normal(scale=0.3, size=(len(s.faces), 9, 3)).astype(np.float32)
        kw = {"sh_degree": 2}
    g = torch.cos(torch.arange(s.n_pixels * 3, device=DEV, dtype=torch.float32)).reshape(-1, 3).contiguous()
    r = _renderer(color_mode=color_mode, deterministic=True, **kw)
    img, out = _grads(r, s, g, rgb=rgb)
    r.close()
    for res in out[1:]:
        for a, b in zip(res, out[0]):
            np.testing.assert_array_equal(a, b)
    r3 = _renderer(color_mode=color_mode, **kw)
    img3, out3 = _grads(r3, s, g, rgb=rgb, repeats=1)
    r3.close()
    np.testing.assert_array_equal(img3, img)
    for a, b in zip(out3[0], out[0]):
        assert rel_l2(a, b) < 1e-5
    assert np.abs(out[0][1]).sum() > 0


def test_fused_loss_and_accumulate():
    s = _scene()
    r = _renderer(deterministic=True)
    v, f, c, o = to_dev(s)
    img, T = r.forward(v, f, c, o, s.cams)
    img = img.clone()
    target = torch.rand_like(img)
    runs = []
    for _ in range(2):
        loss, dv, dc, do = r.backward_l2(img, target)
        torch.cuda.synchronize()
        runs.append((float(loss), dv.cpu().numpy().copy(), dc.cpu().numpy().copy(), do.cpu().numpy().copy()))
    assert runs[0][0] == runs[1][0]
    for a, b in zip(runs[0][1:], runs[1][1:]):
        np.testing.assert_array_equal(a, b)
    # accumulate: a second backward into the same buffers doubles them exactly
    g = (2.0 * (img - target)).contiguous()
    dv, dc, do = r.backward(g)
    dv2, dc2, do2 = dv.clone(), dc.clone(), do.clone()
    r.backward(g, dverts=dv2, drgb=dc2, dopacity=do2, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dv2.cpu().numpy(), 2.0 * dv.cpu().numpy())
    np.testing.assert_array_equal(dc2.cpu().numpy(), 2.0 * dc.cpu().numpy())
    np.testing.assert_array_equal(do2.cpu().numpy(), 2.0 * do.cpu().numpy())
    # and the fused-loss gradients are those of the explicit dL/dI
    assert rel_l2(runs[0][1], dv.cpu().numpy()) < 1e-5
    r.close()


def _fan(n=400, bad=False):
    ang = np.linspace(0.0, 2.0 * np.pi, n, endpoint=False)
    rim = np.stack([0.8 * np.cos(ang), 0.8 * np.sin(ang), 0.1 * np.sin(3 * ang)], 1)
    verts = np.concatenate([[[0.0, 0.0, 0.2]], rim]).astype(np.float32)
    faces = [[0, 1 + i, 1 + (i + 1) % n] for i in range(n)]
    if bad:
        faces += [[0, 1, n + 7], [-1, 2, 3]]
    faces = np.array(faces, np.int32)
    cams = gi.fibonacci_cameras(3, 3.0, [(160, 160), (96, 128), (200, 64)])
    rng = np.random.default_rng(2)
    rgb = rng.random((len(faces), 3)).astype(np.float32)
    return gi.Scene("fan", verts, faces, rgb, np.full(len(faces), 0.8, np.float32), cams)


def test_high_degree_vertex_and_bad_faces():
    """A fan of 400 triangles around one vertex (a list longer than the
    first gaps of the incidence sort): bit for bit on repeat, and close to
    the oracle (the hub's gradient is a sum of 400 shares; the atomic and
    the fixed order differ there by ~1e-4 relative, the FP32 rounding of
    such a sum). With two faces of out-of-range indices added
    (reported, left out of the projection and of the incidence lists) the
    gradients of the valid faces and of every vertex are the same bits, and
    the bad faces' own gradients are zero."""
    s = _fan()
    ref = oracle.render(s)
    gn = np.sin(np.arange(s.n_pixels * 3, dtype=np.float64)).reshape(-1, 3).astype(np.float32)
    gn[ref["flags"] != 0] = 0.0  # pixels whose discrete decisions are near a threshold
    g = torch.from_numpy(gn).to(DEV)
    r = _renderer(deterministic=True)
    img, out = _grads(r, s, g)
    assert r.device_status() == 0
    r.close()
    for res in out[1:]:
        for a, b in zip(res, out[0]):
            np.testing.assert_array_equal(a, b)
    assert np.abs(out[0][0][0]).sum() > 0  # the hub vertex has a gradient
    ob = oracle.backward(s, gn.astype(np.float64))
    assert rel_l2(out[0][0], ob["dverts"]) < 1e-3
    assert rel_l2(out[0][1], ob["drgb"]) <= GRAD_TOL
    sb = _fan(bad=True)
    rb = _renderer(deterministic=True)
    imgb, outb = _grads(rb, sb, g, repeats=1)
    assert rb.device_status() != 0  # the bad faces are reported
    rb.close()
    np.testing.assert_array_equal(imgb, img)
    nf = len(s.faces)
    np.testing.assert_array_equal(outb[0][0], out[0][0])
    np.testing.assert_array_equal(outb[0][1][:nf], out[0][1])
    np.testing.assert_array_equal(outb[0][2][:nf], out[0][2])
    np.testing.assert_array_equal(outb[0][1][nf:], 0.0)
    np.testing.assert_array_equal(outb[0][2][nf:], 0.0)


def test_refused_with_other_backward_layouts():
    from paper_2602_14493_b300 import GmrError

    for kw in (dict(half_bwd=True), dict(warp_bwd=True)):
        with pytest.raises(GmrError):
            _renderer(deterministic=True, **kw)
    r = _renderer(deterministic=True, warp_fwd=True)  # the forward's layout is free
    s = _scene()
    g = torch.ones((s.n_pixels, 3), device=DEV)
    _, out = _grads(r, s, g)
    for a, b in zip(out[1], out[0]):
        np.testing.assert_array_equal(a, b)
    r.close()
