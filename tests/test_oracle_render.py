"""Pins of the oracle's EWA projection, FP32 binning specification and
brute-force compositing (Sec. 2.1, standard 3DGS image formation) against
hand-derived renders, closed forms and invariants."""

import math

import numpy as np
import pytest

import gmr_inputs as gi
import oracle

KAPPA = 6.0 * math.sqrt(3.0) / math.pi


def _axis_camera(W=32, H=32, f=100.0):
    """Camera at the origin looking down +z (R = I, t = 0)."""
    cams = np.zeros(1, dtype=gi.CAMERA_DTYPE)
    cams[0]["R"] = np.eye(3, dtype=np.float32).ravel()
    cams[0]["t"] = 0.0
    cams[0]["fx"] = f
    cams[0]["fy"] = f
    cams[0]["cx"] = W / 2
    cams[0]["cy"] = H / 2
    cams[0]["width"] = W
    cams[0]["height"] = H
    cams[0]["znear"] = 0.01
    return cams


def _equilateral(rho, z, rot=0.0):
    a = rot + np.array([0.0, 2 * math.pi / 3, 4 * math.pi / 3])
    return np.stack([rho * np.cos(a), rho * np.sin(a), np.full(3, z)], 1)


def _scene(verts, faces, rgb, op, cams):
    return gi.Scene("t", np.asarray(verts, np.float32), np.asarray(faces, np.int32), np.asarray(rgb, np.float32),
                    np.asarray(op, np.float32), cams)


def test_projection_on_axis_closed_form():
    cams = _axis_camera(f=200.0)
    z = 4.0
    cov = np.array([[0.02, 0.005, 0.0], [0.005, 0.01, 0.0], [0.0, 0.0, 0.0]])
    p = oracle.project(np.array([[0.0, 0.0, z]]), cov[None], cams)
    s = (200.0 / z) ** 2
    np.testing.assert_allclose(p["sigma"][0], [s * 0.02 + 0.3, s * 0.005, s * 0.01 + 0.3], rtol=1e-14)
    np.testing.assert_allclose(p["u"][0], [16.0, 16.0], atol=1e-12)
    A, B, C = p["sigma"][0]
    a, b, c = p["conic"][0]
    np.testing.assert_allclose(np.array([[a, b], [b, c]]) @ np.array([[A, B], [B, C]]), np.eye(2), atol=1e-12)


def test_projection_jacobian_matches_finite_difference():
    """Sigma' = J W Sigma W^T J^T + 0.3 I with J the derivative of the
    perspective map at the camera-space mean (EWA, Sec. 2.1)."""
    cams = gi.ring_cameras(3, 20.0, 3.0, 64, 48)
    rng = np.random.default_rng(1)
    means = rng.normal(scale=0.4, size=(5, 3))
    A = rng.normal(size=(5, 3, 3)) * 0.05
    cov = A @ A.transpose(0, 2, 1)
    p = oracle.project(means, cov, cams)
    for c in range(3):
        R = cams[c]["R"].astype(np.float64).reshape(3, 3)
        t = cams[c]["t"].astype(np.float64)
        fx, fy = float(cams[c]["fx"]), float(cams[c]["fy"])
        cx, cy = float(cams[c]["cx"]), float(cams[c]["cy"])

        def pix(tc):
            return np.array([fx * tc[0] / tc[2] + cx, fy * tc[1] / tc[2] + cy])

        for k in range(5):
            tc = R @ means[k] + t
            h = 1e-6
            J = np.stack([(pix(tc + h * e) - pix(tc - h * e)) / (2 * h) for e in np.eye(3)], 1)
            S = J @ R @ cov[k] @ R.T @ J.T + 0.3 * np.eye(2)
            r = c * 5 + k
            np.testing.assert_allclose(p["sigma"][r], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-7)
            np.testing.assert_allclose(p["u"][r], pix(tc), rtol=1e-13)
            np.testing.assert_allclose(p["tcam"][r], tc, rtol=1e-13, atol=1e-14)


def _hand_alpha(o, d2, sigma2):
    g = o * math.exp(-0.5 * d2 / sigma2)
    return min(0.99, g)


def test_single_triangle_render_by_hand():
    """Equilateral facet facing the camera on the axis: Sigma' is isotropic,
    (f/z)^2 kappa L^2/24 + 0.3, and each pixel is c * alpha (one layer)."""
    W = H = 32
    f, z, rho = 100.0, 5.0, 0.12
    cams = _axis_camera(W, H, f)
    v = _equilateral(rho, z)
    L = rho * math.sqrt(3.0)
    sigma2 = (f / z) ** 2 * KAPPA * L * L / 24.0 + 0.3
    col = np.array([[0.2, 0.5, 0.9]])
    s = _scene(v, [[0, 1, 2]], col, [0.8], cams)
    r = oracle.render(s)
    img = r["rgb"].reshape(H, W, 3)
    for (y, x) in [(16, 16), (15, 16), (16, 20), (10, 12), (3, 29), (0, 0)]:
        d2 = (x + 0.5 - 16.0) ** 2 + (y + 0.5 - 16.0) ** 2
        a = _hand_alpha(0.8, d2, sigma2)
        if a < 1 / 255:
            a = 0.0
        np.testing.assert_allclose(img[y, x], col[0] * a, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(r["T"][y * W + x], 1 - a, rtol=1e-6, atol=1e-12)


def test_two_layers_and_termination_by_hand():
    W = H = 16
    f = 60.0
    cams = _axis_camera(W, H, f)
    rho = 0.1
    depths = [2.0, 2.5, 3.0, 3.5, 4.0]
    verts = np.concatenate([_equilateral(rho * z / 2.0, z, rot=0.3 * i) for i, z in enumerate(depths)], 0)
    faces = np.arange(15).reshape(5, 3)[::-1].copy()  # depth order differs from index order
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]], np.float64)[::-1].copy()
    ops = np.full(5, 0.95)
    s = _scene(verts, faces, cols, ops, cams)
    r = oracle.render(s)
    # each facet is scaled with depth so that all have the same image-plane size
    L = rho / 2.0 * math.sqrt(3.0)
    sigma2 = f * f * KAPPA * L * L / 24.0 + 0.3
    for (y, x) in [(8, 8), (7, 9), (5, 10)]:
        d2 = (x + 0.5 - 8.0) ** 2 + (y + 0.5 - 8.0) ** 2
        T, C, nc, stopped = 1.0, np.zeros(3), 0, False
        for k in range(5):  # nearest first: face 4 (depth 2.0) ... face 0
            fidx = 4 - k
            a = _hand_alpha(0.95, d2, sigma2)
            if a < 1 / 255:
                continue
            if T * (1 - a) < 1e-4:
                stopped = True
                break
            C += cols[fidx] * a * T
            T *= 1 - a
            nc += 1
        i = y * W + x
        np.testing.assert_allclose(r["rgb"][i], C, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(r["T"][i], T, rtol=1e-6)
        assert r["n_contrib"][i] == nc
        if (y, x) == (8, 8):
            assert stopped and nc == 4  # the fifth layer would take T below 1e-4
    # two facets at exactly the same depth: the lower face index is in front
    v2 = np.concatenate([_equilateral(0.1, 2.0), _equilateral(0.1, 2.0, rot=0.5)], 0)
    s2 = _scene(v2, [[0, 1, 2], [3, 4, 5]], [[1, 0, 0], [0, 0, 1]], [0.6, 0.6], cams)
    r2 = oracle.render(s2, pixels=np.array([[0, 8, 8]]))
    a = r2["rgb"][0]
    assert a[0] > a[2]  # red (face 0) composited first


def test_render_invariants_icosphere():
    s = gi.scene_single_view()
    r = oracle.render(s)
    T, img = r["T"], r["rgb"]
    assert np.all(T <= 1.0) and np.all(T >= 1e-4)
    assert np.all(img >= -1e-15) and np.all(img <= 1.0 + 1e-12)
    none = r["n_contrib"] == 0
    assert np.array_equal(none, r["last_face"] < 0)
    assert np.all(T[none] == 1.0)
    # background enters as T * bg
    r1 = oracle.render(s, bg=(1.0, 0.5, 0.25))
    np.testing.assert_allclose(r1["rgb"] - img, T[:, None] * np.array([1.0, 0.5, 0.25]), atol=1e-12)
    # ambiguous pixels are rare
    assert (r["flags"] & (oracle.FLAG_ALPHA_SKIP | oracle.FLAG_TERMINATE)).mean() < 2e-3


def test_per_vertex_colour_mode_is_face_mean():
    """Eq. 16: the face colour is the mean of its three vertex colours."""
    s = gi.scene_single_view()
    rng = np.random.default_rng(2)
    vcol = rng.random((len(s.verts), 3)).astype(np.float32)
    pix = oracle.all_pixels(s.cams)[::7]
    sv = gi.Scene("v", s.verts, s.faces, vcol, s.opacity, s.cams)
    a = oracle.render(sv, pixels=pix, color_mode=1)
    fcol = vcol.astype(np.float64)[s.faces].mean(1)
    # per-face colours rounded to FP32: agreement up to that rounding
    sf = gi.Scene("f", s.verts, s.faces, fcol.astype(np.float32), s.opacity, s.cams)
    b = oracle.render(sf, pixels=pix, color_mode=0)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-6)
    np.testing.assert_array_equal(a["T"], b["T"])


def test_opacity_is_clamped_to_unit_interval():
    s = gi.scene_single_view()
    pix = oracle.all_pixels(s.cams)[::5]
    hi = gi.Scene("h", s.verts, s.faces, s.rgb, np.full(len(s.faces), 1.7, np.float32), s.cams)
    one = gi.Scene("o", s.verts, s.faces, s.rgb, np.full(len(s.faces), 1.0, np.float32), s.cams)
    a, b = oracle.render(hi, pixels=pix), oracle.render(one, pixels=pix)
    np.testing.assert_array_equal(a["rgb"], b["rgb"])


def _visible_alpha_boxes(scene, tile):
    """Closed-form bound: pixel centres with o*G >= 1/255 satisfy
    d^T Sigma'^-1 d <= 2 ln(255 o), whose x-extent is sqrt(k Sigma'_xx)."""
    conv = oracle.convert(scene.verts.astype(np.float64), scene.faces, cov_mode=0)
    pr = oracle.project(conv["means"], conv["cov"], scene.cams)
    o = np.clip(scene.opacity.astype(np.float64), 0, 1)
    F = len(scene.faces)
    out = []
    for c, cam in enumerate(scene.cams):
        W, H = int(cam["width"]), int(cam["height"])
        for f in range(F):
            r = c * F + f
            if o[f] * 255 < 1:
                out.append(None)
                continue
            k = 2 * math.log(255 * o[f])
            A, B, C = pr["sigma"][r]
            ux, uy = pr["u"][r]
            if pr["tcam"][r][2] <= float(cam["znear"]):
                out.append(None)
                continue
            hx, hy = math.sqrt(k * A), math.sqrt(k * C)
            px0, px1 = math.ceil(ux - hx - 0.5), math.floor(ux + hx - 0.5)
            py0, py1 = math.ceil(uy - hy - 0.5), math.floor(uy + hy - 0.5)
            px0, py0 = max(px0, 0), max(py0, 0)
            px1, py1 = min(px1, W - 1), min(py1, H - 1)
            if px0 > px1 or py0 > py1:
                out.append(None)
                continue
            out.append((px0 // tile, px1 // tile, py0 // tile, py1 // tile))
    return out, pr


@pytest.mark.parametrize("tile", [16, 32])
def test_bin_rect_is_conservative(tile):
    for s in (gi.scene_single_view(), gi.random_triangle_soup(4, 60, n_views=2, res=(70, 45))):
        b = oracle.bins(s.verts, s.faces, s.cams, tile)
        boxes, pr = _visible_alpha_boxes(s, tile)
        n_checked = 0
        for r, box in enumerate(boxes):
            if box is None:
                continue
            assert b["visible"][r]
            x0, x1, y0, y1 = b["rect"][r]
            assert x0 <= box[0] and box[1] <= x1 and y0 <= box[2] and box[3] <= y1, (r, box, b["rect"][r])
            n_checked += 1
        assert n_checked > 0
        # the FP32 key depth and screen mean follow the FP64 projection
        vis = b["visible"]
        depth = b["depth_bits"].view(np.float32).astype(np.float64)
        np.testing.assert_allclose(depth[vis], pr["tcam"][vis, 2], rtol=1e-6)
        np.testing.assert_allclose(b["uxyr"][vis, :2], pr["u"][vis], atol=2e-3)


def test_bins_cull_behind_camera_and_nonfinite():
    cams = _axis_camera()
    v = np.concatenate([_equilateral(0.1, 2.0), _equilateral(0.1, -1.0), _equilateral(0.1, 0.005),
                        _equilateral(0.1, 3.0)], 0).astype(np.float32)
    v[9, 0] = np.nan
    f = np.arange(12, dtype=np.int32).reshape(4, 3)
    b = oracle.bins(v, f, cams, 16)
    assert list(b["visible"]) == [True, False, False, False]


@pytest.mark.parametrize("tile", [16, 32])
def test_sorted_pairs_and_ranges(tile):
    s = gi.random_triangle_soup(7, 80, n_views=3, res=(100, 37))
    b = oracle.bins(s.verts, s.faces, s.cams, tile)
    tiles, fids, ranges = oracle.sorted_pairs(s.verts, s.faces, s.cams, tile)
    tx, ty = oracle.tile_counts(s.cams, tile)
    base = np.concatenate([[0], np.cumsum(np.array(tx) * np.array(ty))])
    # expected pairs from the rectangles, ordered with numpy's stable lexsort
    F = len(s.faces)
    exp_t, exp_d, exp_f = [], [], []
    for c in range(3):
        for f in range(F):
            r = c * F + f
            if not b["visible"][r]:
                continue
            x0, x1, y0, y1 = b["rect"][r]
            for y in range(y0, y1 + 1):
                for x in range(x0, x1 + 1):
                    exp_t.append(base[c] + y * tx[c] + x)
                    exp_d.append(b["depth_bits"][r])
                    exp_f.append(f)
    exp_t, exp_d, exp_f = map(np.array, (exp_t, exp_d, exp_f))
    order = np.lexsort((exp_f, exp_d, exp_t))
    np.testing.assert_array_equal(tiles, exp_t[order])
    np.testing.assert_array_equal(fids, exp_f[order])
    for g in range(base[-1]):
        lo, hi = ranges[g]
        sel = np.nonzero(tiles == g)[0]
        if len(sel) == 0:
            assert lo == 0 and hi == 0
        else:
            assert lo == sel[0] and hi == sel[-1] + 1
