"""GPU parity of the CUDA path (called through the C ABI) against the FP64
oracle: conversion, binning (bit-exact), projected records, images, and
gradients."""

import functools

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from gpu_util import DEV, GRAD_TOL, IMG_TOL, rel_l2, render_gpu, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2602_14493_b300 import Renderer

    r = Renderer()
    yield r
    r.close()


def _uneven_scene():
    v, f = gi.icosphere(3)
    rng = np.random.default_rng(31)
    cams = gi.fibonacci_cameras(5, 3.0, [(256, 256), (100, 37), (64, 200), (17, 5), (384, 384)])
    return gi.Scene("uneven", v.astype(np.float32), f, rng.random((len(f), 3)).astype(np.float32),
                    rng.uniform(0.3, 1.0, len(f)).astype(np.float32), cams)


def _scenes():
    return {
        "icosphere3_1x128": gi.scene_single_view(),
        "soup": gi.random_triangle_soup(7, 150, n_views=3, res=(100, 37)),
        "uneven": _uneven_scene(),
    }


# ------------------------------------------------------------------ conversion
@pytest.mark.parametrize("cov_mode", ["area", "embed_raw"])
@pytest.mark.parametrize("color_mode", ["face", "vertex"])
def test_convert_matches_oracle(cov_mode, color_mode):
    from paper_2602_14493_b300 import Renderer

    r = Renderer(cov_mode=cov_mode, color_mode=color_mode)
    for s in (gi.scene_ring(), gi.random_triangle_soup(3, 1000)):
        rgb = s.rgb if color_mode == "face" else np.random.default_rng(1).random((len(s.verts), 3)).astype(np.float32)
        v, f, c, o = to_dev(s, rgb)
        o_in = o.clone()
        o_in[::7] = 1.7
        o_in[1::11] = -0.2
        out = r.convert(v, f, c, o_in)
        torch.cuda.synchronize()
        ref = oracle.convert(s.verts.astype(np.float64), s.faces, cov_mode=0 if cov_mode == "area" else 1)
        means = out["means"].cpu().numpy()
        np.testing.assert_allclose(means, ref["means"], atol=3e-7 * np.abs(ref["means"]).max())
        cov = out["cov"].cpu().numpy()
        full = ref["cov"]
        six = np.stack([full[:, 0, 0], full[:, 0, 1], full[:, 0, 2], full[:, 1, 1], full[:, 1, 2], full[:, 2, 2]], 1)
        scale = np.abs(six).max(1, keepdims=True)
        assert np.all(np.abs(cov - six) <= 1e-5 * scale + 1e-13)
        fc = rgb if color_mode == "face" else rgb.astype(np.float64)[s.faces].mean(1)
        np.testing.assert_allclose(out["rgb"].cpu().numpy(), fc, atol=1e-7)
        np.testing.assert_array_equal(out["opacity"].cpu().numpy(), np.clip(o_in.cpu().numpy(), 0, 1))
    assert r.device_status() == 0
    r.close()


@pytest.mark.parametrize("cov_mode", ["area", "embed_raw"])
def test_convert_invariant_to_vertex_order_and_rigid_motion(cov_mode):
    """The GPU conversion does not depend on which vertex of a face comes
    first or on the face's orientation (the covariance is a symmetric
    function of the three vertices and enters through n n^T), and it is
    equivariant under rigid motions: mu(Q v + t) = Q mu(v) + t and
    Sigma(Q v + t) = Q Sigma(v) Q^T (Sec. 2.2). Both FP32 results are within
    1e-5 of the exact covariance (test above), so they agree to 2e-5."""
    from paper_2602_14493_b300 import Renderer

    r = Renderer(cov_mode=cov_mode)
    s = gi.random_triangle_soup(7, 2000)
    v, f, c, o = to_dev(s, s.rgb)

    def conv(vv, ff):
        out = r.convert(vv, ff, c, o)
        torch.cuda.synchronize()
        cv = out["cov"].cpu().numpy().astype(np.float64)
        full = np.stack([cv[:, [0, 1, 2]], cv[:, [1, 3, 4]], cv[:, [2, 4, 5]]], 1)
        return out["means"].cpu().numpy().astype(np.float64), full

    m0, c0 = conv(v, f)
    scale = np.abs(c0).reshape(len(c0), -1).max(1)[:, None, None]
    mscale = np.abs(m0).max()
    for perm in ([1, 2, 0], [2, 0, 1], [0, 2, 1]):
        m1, c1 = conv(v, f[:, perm].contiguous())
        assert np.abs(m1 - m0).max() <= 1e-6 * mscale
        assert np.all(np.abs(c1 - c0) <= 2e-5 * scale + 1e-13)
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    t = rng.normal(size=3)
    vq = (s.verts.astype(np.float64) @ Q.T + t).astype(np.float32)
    m2, c2 = conv(torch.from_numpy(vq).to(v.device), f)
    np.testing.assert_allclose(m2, m0 @ Q.T + t, atol=2e-6 * (mscale + np.abs(t).max()))
    rot = np.einsum("ij,fjk,lk->fil", Q, c0, Q)
    # the moved vertices are rounded to FP32 (relative 2^-24 of their
    # magnitude), which moves a face's covariance by up to ~4 |edge| |dv|
    vv = s.verts.astype(np.float64)[s.faces]
    edge = np.linalg.norm(vv - vv.mean(1, keepdims=True), axis=2).max(1)[:, None, None]
    dv = 2.0 ** -24 * max(np.abs(vq).max(), np.abs(s.verts).max())
    assert np.all(np.abs(c2 - rot) <= 2e-5 * scale + 8.0 * edge * dv + 1e-13)
    assert r.device_status() == 0
    r.close()


# ------------------------------------------------------------------ binning
def _dense_scene():
    """A level-6 icosphere (81,920 faces) in a 128^2 and a 256^2 view: with
    16x16 tiles, segments of every length class of the per-tile sort (up to
    256 keys in registers, 257-512 as two register halves merged, 513-1024 and 1025-4096
    by the CTA merge sort, longer by radix passes: the longest holds 4,920
    keys)."""
    v, f = gi.icosphere(6)
    rng = np.random.default_rng(61)
    cams = np.concatenate([gi.ring_cameras(1, 20.0, 3.0, 128, 128),
                           gi.ring_cameras(1, 35.0, 3.0, 256, 256, azimuth0_deg=40.0)])
    return gi.Scene("dense6_128_256", v.astype(np.float32), f, rng.random((len(f), 3)).astype(np.float32),
                    np.full(len(f), 0.9, np.float32), cams)


SORT_CLASSES = [(0, 256), (256, 512), (512, 1024), (1024, 4096), (4096, 1 << 30)]


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("name", ["icosphere3_1x128", "soup", "uneven", "dense6_128_256"])
def test_binning_bit_exact(renderer, tile, name):
    s = _dense_scene() if name == "dense6_128_256" else _scenes()[name]
    renderer.set_config(tile=tile)
    render_gpu(renderer, s)
    tx, ty = oracle.tile_counts(s.cams, tile)
    n_tiles = int(sum(a * b for a, b in zip(tx, ty)))
    st = renderer.debug_state(len(s.cams), len(s.faces), n_tiles, s.n_pixels)
    ob = oracle.bins(s.verts, s.faces, s.cams, tile)
    vis = ob["visible"]
    gvis = st["depth_bits"] != 0xFFFFFFFF
    np.testing.assert_array_equal(gvis, vis)
    np.testing.assert_array_equal(st["depth_bits"][vis], ob["depth_bits"][vis])
    # rectangles: identical where non-empty; empty on both sides otherwise
    orect, grect = ob["rect"], st["rects"]
    oe = (orect[:, 0] > orect[:, 1]) | (orect[:, 2] > orect[:, 3]) | ~vis
    ge = (grect[:, 0] > grect[:, 1]) | (grect[:, 2] > grect[:, 3])
    np.testing.assert_array_equal(ge, oe)
    np.testing.assert_array_equal(grect[~oe], orect[~oe])
    tiles, fids, ranges = oracle.sorted_pairs(s.verts, s.faces, s.cams, tile)
    if name == "dense6_128_256" and tile == 16:
        seg = (ranges[:, 1] - ranges[:, 0]).astype(np.int64)
        assert all(((seg > a) & (seg <= b)).sum() >= 5 for a, b in SORT_CLASSES)
    assert st["n_pairs"] == len(tiles)
    np.testing.assert_array_equal(st["tile_ids"], tiles)
    np.testing.assert_array_equal(st["face_ids"], fids)
    np.testing.assert_array_equal(st["ranges"], ranges)
    renderer.set_config(tile=16)


def test_records_match_oracle_projection(renderer):
    s = _scenes()["uneven"]
    render_gpu(renderer, s)
    tx, ty = oracle.tile_counts(s.cams, 16)
    st = renderer.debug_state(len(s.cams), len(s.faces), int(sum(a * b for a, b in zip(tx, ty))), s.n_pixels)
    conv = oracle.convert(s.verts.astype(np.float64), s.faces)
    pr = oracle.project(conv["means"], conv["cov"], s.cams)
    rect = st["rects"]
    live = rect[:, 0] <= rect[:, 1]
    u = st["rec_u"][:, :2].astype(np.float64) + st["rec_u"][:, 2:].astype(np.float64)
    assert np.abs(u[live] - pr["u"][live]).max() < 1e-5
    q = st["conic"][live].astype(np.float64)
    qo = pr["conic"][live]
    scale = np.abs(qo).max(1, keepdims=True)
    assert np.all(np.abs(q - qo) <= 2e-5 * scale)


# ------------------------------------------------------------------ images
@pytest.mark.parametrize("name", ["icosphere3_1x128", "soup", "uneven"])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_image_matches_oracle(renderer, name, tile):
    s = _scenes()[name]
    renderer.set_config(tile=tile, bg=(0.1, 0.2, 0.3))
    _, img, T = render_gpu(renderer, s)
    ref = oracle.render(s, bg=(0.1, 0.2, 0.3))
    amb = (ref["flags"] & (oracle.FLAG_ALPHA_SKIP | oracle.FLAG_TERMINATE)) != 0
    err = np.abs(img.cpu().numpy() - ref["rgb"]).max(1)
    terr = np.abs(T.cpu().numpy() - ref["T"])
    assert amb.mean() < 1e-3
    assert err[~amb].max() <= IMG_TOL, (err[~amb].max(), np.argmax(np.where(amb, 0, err)))
    assert terr[~amb].max() <= IMG_TOL
    assert renderer.device_status() == 0
    renderer.set_config(tile=16, bg=(0.0, 0.0, 0.0))


@pytest.mark.parametrize("threads", [(128, 128), (256, 128)])
def test_image_full_size_ring_sampled(renderer, threads):
    """The 8 x 512^2 ring workload at full size, batched, tile 16, batch 256,
    in the default launch shape and the one the benchmark times (256
    forward threads per tile), on sampled pixels."""
    s = gi.scene_ring()
    renderer.set_config(threads=threads[0], threads_bwd=threads[1])
    _, img, T = render_gpu(renderer, s)
    pix, lin = sample_pixels(s.cams, 2400, 5)
    ref = oracle.render(s, pixels=pix)
    amb = (ref["flags"] & (oracle.FLAG_ALPHA_SKIP | oracle.FLAG_TERMINATE)) != 0
    g = img.cpu().numpy()[lin]
    err = np.abs(g - ref["rgb"]).max(1)
    assert err[~amb].max() <= IMG_TOL
    assert np.abs(T.cpu().numpy()[lin] - ref["T"])[~amb].max() <= IMG_TOL
    # whole-image invariants
    a = img.cpu().numpy()
    t = T.cpu().numpy()
    assert np.all(a >= 0) and np.all(a <= 1.0 + 1e-6) and np.all(t >= 1e-4 - 1e-9) and np.all(t <= 1.0)
    renderer.set_config(threads=128, threads_bwd=128)


# ------------------------------------------------------------------ gradients
@pytest.mark.parametrize("name", ["icosphere3_1x128", "soup", "uneven"])
@pytest.mark.parametrize("cov_mode", ["area", "embed_raw"])
def test_gradients_match_oracle(name, cov_mode):
    from paper_2602_14493_b300 import Renderer

    r = Renderer(cov_mode=cov_mode, bg=(0.2, 0.1, 0.4))
    s = _scenes()[name]
    cm = 0 if cov_mode == "area" else 1
    ref = oracle.render(s, cov_mode=cm, bg=(0.2, 0.1, 0.4))
    rng = np.random.default_rng(11)
    g = rng.normal(size=ref["rgb"].shape).astype(np.float32)
    g[ref["flags"] != 0] = 0.0
    (v, f, c, o), img, T = render_gpu(r, s)
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV))
    torch.cuda.synchronize()
    ob = oracle.backward(s, g.astype(np.float64), cov_mode=cm, bg=(0.2, 0.1, 0.4))
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    r.close()


@pytest.mark.parametrize("threads", [(128, 128), (256, 128)])
def test_gradients_full_size_ring_sparse(renderer, threads):
    """Full-size ring workload (default and benchmark launch shapes); dL/dI
    non-zero on sampled pixels only, so the oracle's backward over those
    pixels is the exact reference."""
    s = gi.scene_ring()
    renderer.set_config(threads=threads[0], threads_bwd=threads[1])
    (v, f, c, o), img, T = render_gpu(renderer, s)
    pix, lin = sample_pixels(s.cams, 2400, 6)
    ref = oracle.render(s, pixels=pix)
    rng = np.random.default_rng(12)
    gs = rng.normal(size=(len(pix), 3))
    gs[ref["flags"] != 0] = 0.0
    g = np.zeros((s.n_pixels, 3), dtype=np.float32)
    g[lin] = gs
    dv, dc, do = renderer.backward(torch.from_numpy(g).to(DEV))
    torch.cuda.synchronize()
    ob = oracle.backward(s, gs.astype(np.float32).astype(np.float64), pixels=pix)
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    renderer.set_config(threads=128, threads_bwd=128)


def test_per_vertex_colour_gradients():
    from paper_2602_14493_b300 import Renderer

    r = Renderer(color_mode="vertex")
    s0 = gi.scene_single_view()
    vcol = np.random.default_rng(3).random((len(s0.verts), 3)).astype(np.float32)
    s = gi.Scene("v", s0.verts, s0.faces, vcol, s0.opacity, s0.cams)
    ref = oracle.render(s, color_mode=1)
    g = np.random.default_rng(4).normal(size=ref["rgb"].shape).astype(np.float32)
    g[ref["flags"] != 0] = 0
    _, img, _ = render_gpu(r, s)
    amb = ref["flags"] != 0
    assert np.abs(img.cpu().numpy() - ref["rgb"]).max(1)[~amb].max() <= IMG_TOL
    dv, dc, _ = r.backward(torch.from_numpy(g).to(DEV))
    ob = oracle.backward(s, g.astype(np.float64), color_mode=1)
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    r.close()


# ------------------------------------------------------------------ view-dependent colour
def _sh_scene(name, L, seed):
    s0 = _scenes()[name]
    rng = np.random.default_rng(seed)
    K = (L + 1) ** 2
    coef = rng.normal(scale=0.3, size=(len(s0.faces), K, 3)).astype(np.float32)
    coef[:, 0, :] = rng.uniform(-0.2, 1.2, size=(len(s0.faces), 3))  # some colours clamp at zero
    return gi.Scene(s0.name, s0.verts, s0.faces, coef, s0.opacity, s0.cams)


@pytest.mark.parametrize("L", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["soup", "uneven"])
def test_sh_colour_image_and_gradients_match_oracle(L, name):
    """Spherical-harmonic colour (GMR_COLOR_SH): per-view colours in the
    projection, the compositing reads them per record, and the projection
    backward chains the colour gradients to the coefficients and, through
    the view direction, to the vertices."""
    from paper_2602_14493_b300 import Renderer

    s = _sh_scene(name, L, seed=40 + L)
    bg = (0.2, 0.1, 0.4)
    r = Renderer(color_mode="sh", sh_degree=L, bg=bg)
    ref = oracle.render(s, color_mode=2, sh_degree=L, bg=bg)
    (v, f, c, o), img, T = render_gpu(r, s)
    amb = (ref["flags"] & 3) != 0
    assert amb.mean() < 1e-3
    assert np.abs(img.cpu().numpy() - ref["rgb"]).max(1)[~amb].max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T"])[~amb].max() <= IMG_TOL
    g = np.random.default_rng(12).normal(size=ref["rgb"].shape).astype(np.float32)
    g[ref["flags"] != 0] = 0.0
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV))
    torch.cuda.synchronize()
    assert dc.shape == c.shape
    ob = oracle.backward(s, g.astype(np.float64), color_mode=2, sh_degree=L, bg=bg)
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    assert r.device_status() == 0
    # the same through one call per view, accumulating the gradients
    dv2, dc2, do2 = torch.zeros_like(dv), torch.zeros_like(dc), torch.zeros_like(do)
    off = oracle.pixel_offsets(s.cams)
    gd = torch.from_numpy(g).to(DEV)
    for k in range(len(s.cams)):
        img_k, _ = r.forward(v, f, c, o, s.cams[k:k + 1])
        np.testing.assert_array_equal(img_k.cpu().numpy(), img[off[k]:off[k + 1]].cpu().numpy())
        r.backward(gd[off[k]:off[k + 1]].contiguous(), dv2, dc2, do2, accumulate=True)
    assert rel_l2(dv2.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc2.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    r.close()


SH_LAYOUTS = [
    dict(threads=128, threads_bwd=128, warp_fwd=True, half_bwd=True),
    dict(threads=128, threads_bwd=128, warp_fwd=True, warp_bwd=True),
    dict(threads=256, threads_bwd=128, half_fwd=True, half_bwd=True),
    dict(threads=128, threads_bwd=128, persistent=True),
    dict(tile=8, threads=64, threads_bwd=32, warp_fwd=True, warp_bwd=True),
    dict(tile=8, threads=64, threads_bwd=64, persistent=True),
    dict(tile=8, threads=64, threads_bwd=32, warp_fwd=True, half_bwd=True),
    dict(tile=32, threads=256, threads_bwd=256),
    dict(threads=128, threads_bwd=128, deterministic=True),
]


@functools.lru_cache(maxsize=1)
def _sh_layout_reference():
    s = _sh_scene("uneven", 3, seed=77)
    bg = (0.2, 0.1, 0.4)
    ref = oracle.render(s, color_mode=2, sh_degree=3, bg=bg)
    g = np.random.default_rng(78).normal(size=ref["rgb"].shape).astype(np.float32)
    g[ref["flags"] != 0] = 0.0
    ob = oracle.backward(s, g.astype(np.float64), color_mode=2, sh_degree=3, bg=bg)
    return s, bg, ref, g, ob


@pytest.mark.parametrize("shape", range(len(SH_LAYOUTS)))
def test_sh_colour_in_every_layout_matches_oracle(shape):
    """Spherical-harmonic colour (degree 3) through each compositing layout:
    the warp-staged, half-warp and block-staged kernels, the persistent
    grid, 8x8 tiles with split binning and 32x32 tiles, and the
    deterministic backward all read the per-(view, face) colours of the
    projection; image and gradients match the oracle."""
    from paper_2602_14493_b300 import Renderer

    s, bg, ref, g, ob = _sh_layout_reference()
    amb = (ref["flags"] & 3) != 0
    r = Renderer(color_mode="sh", sh_degree=3, bg=bg, **SH_LAYOUTS[shape])
    (v, f, c, o), img, T = render_gpu(r, s)
    assert np.abs(img.cpu().numpy() - ref["rgb"]).max(1)[~amb].max() <= IMG_TOL
    assert np.abs(T.cpu().numpy() - ref["T"])[~amb].max() <= IMG_TOL
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV))
    torch.cuda.synchronize()
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    assert r.device_status() == 0
    r.close()


def test_sh_degree_zero_equals_face_colour():
    """GMR_COLOR_SH with degree 0 renders exactly what GMR_COLOR_PER_FACE
    renders with colour a_0 Y_0 + 1/2 (bit for bit when that colour is
    representable)."""
    from paper_2602_14493_b300 import Renderer

    s = _scenes()["uneven"]
    y0 = np.float32(0.282094791773878)
    col = s.rgb.astype(np.float32)
    a0 = ((col - np.float32(0.5)) / y0).astype(np.float32)[:, None, :]
    rs = Renderer(color_mode="sh", sh_degree=0)
    rf = Renderer()
    _, img_sh, _ = render_gpu(rs, s, rgb=a0)
    _, img_f, _ = render_gpu(rf, s)
    assert np.abs(img_sh.cpu().numpy() - img_f.cpu().numpy()).max() <= 1e-6
    rs.close()
    rf.close()


# ------------------------------------------------------------------ silhouette
@pytest.mark.parametrize("name", ["icosphere3_1x128", "soup", "uneven"])
@pytest.mark.parametrize("with_image", [False, True])
def test_final_transmittance_gradients_match_oracle(name, with_image):
    """dL/dT_final (the silhouette loss's gradient) through gmr_render_bwd_ex,
    alone and with dL/dI, against the oracle's reverse pass."""
    from paper_2602_14493_b300 import Renderer

    r = Renderer(bg=(0.2, 0.1, 0.4))
    s = _scenes()[name]
    ref = oracle.render(s, bg=(0.2, 0.1, 0.4))
    rng = np.random.default_rng(21)
    gT = rng.normal(size=ref["T"].shape).astype(np.float32)
    gT[ref["flags"] != 0] = 0.0
    g = rng.normal(size=ref["rgb"].shape).astype(np.float32)
    g[ref["flags"] != 0] = 0.0
    if not with_image:
        g[:] = 0.0
    (v, f, c, o), img, T = render_gpu(r, s)
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV) if with_image else None,
                            dL_dtfinal=torch.from_numpy(gT).to(DEV))
    torch.cuda.synchronize()
    ob = oracle.backward(s, g.astype(np.float64), bg=(0.2, 0.1, 0.4), dLdT=gT.astype(np.float64))
    assert np.abs(ob["dverts"]).max() > 0
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    if with_image:
        assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    else:
        assert np.all(dc.cpu().numpy() == 0.0)
    r.close()


BWD_LAYOUTS = [
    dict(threads_bwd=128, half_bwd=True),
    dict(threads_bwd=256, half_bwd=True),
    dict(threads_bwd=128, warp_bwd=True),
    dict(threads_bwd=128, persistent=True),
    dict(tile=8, threads=64, threads_bwd=32, warp_fwd=True, warp_bwd=True),
    dict(tile=8, threads=64, threads_bwd=32, half_bwd=True),
    dict(tile=8, threads=64, threads_bwd=64, persistent=True),
    dict(tile=32, threads=256, threads_bwd=256),
    dict(threads_bwd=128, deterministic=True),
]


@functools.lru_cache(maxsize=1)
def _silhouette_reference():
    s = _scenes()["uneven"]
    bg = (0.2, 0.1, 0.4)
    ref = oracle.render(s, bg=bg)
    rng = np.random.default_rng(23)
    gT = rng.normal(size=ref["T"].shape).astype(np.float32)
    g = rng.normal(size=ref["rgb"].shape).astype(np.float32)
    gT[ref["flags"] != 0] = 0.0
    g[ref["flags"] != 0] = 0.0
    ob = oracle.backward(s, g.astype(np.float64), bg=bg, dLdT=gT.astype(np.float64))
    return s, bg, g, gT, ob


@pytest.mark.parametrize("shape", range(len(BWD_LAYOUTS)))
def test_final_transmittance_gradients_in_every_backward_layout(shape):
    """dL/dT_final together with dL/dI through each backward layout (half-warp
    at 128 and 256 threads, warp-staged, block-staged as a persistent grid,
    8x8 tiles with split binning, 32x32 tiles, the deterministic backward)
    against the oracle's reverse pass."""
    from paper_2602_14493_b300 import Renderer

    s, bg, g, gT, ob = _silhouette_reference()
    r = Renderer(bg=bg, **BWD_LAYOUTS[shape])
    render_gpu(r, s)
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV), dL_dtfinal=torch.from_numpy(gT).to(DEV))
    torch.cuda.synchronize()
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    assert rel_l2(do.cpu().numpy(), ob["dopacity"]) <= GRAD_TOL
    assert r.device_status() == 0
    r.close()


def test_silhouette_bce_against_fp64():
    """The loss and dL/dT_final of gmr_silhouette_bce against the FP64
    oracle on random transmittances (including clamped ends) and binary and
    fractional masks."""
    from paper_2602_14493_b300 import Renderer

    rng = np.random.default_rng(5)
    n = 100003
    T = rng.uniform(1e-4, 1.0, n).astype(np.float32)
    T[:50] = 1.0  # empty pixels: mask 0 exactly, clamped
    m = (rng.random(n) < 0.5).astype(np.float32)
    m[::7] = rng.random(len(m[::7])).astype(np.float32)
    r = Renderer()
    loss, grad = r.silhouette_bce(torch.from_numpy(T).to(DEV), torch.from_numpy(m).to(DEV))
    from oracle import fit_terms

    ref, gref = fit_terms.silhouette_bce(T, m)
    assert abs(float(loss) - ref) <= 1e-5 * abs(ref)
    np.testing.assert_allclose(grad.cpu().numpy(), gref, rtol=1e-5, atol=1e-12)
    r.close()
