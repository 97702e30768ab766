"""Pins of the oracle's view-dependent (spherical-harmonic) colour, the
extension of the facet colour named in the colour assignment of Sec. 2.2:
the basis against scipy's complex spherical harmonics, quadrature
orthonormality, the degree-0 case against the plain per-face colour, the
clamp at zero, and the reverse pass against dual numbers."""

import math

import numpy as np
import pytest
import scipy.special as sp

import gmr_inputs as gi
import oracle


def _real_sh_scipy(L, d):
    """Real spherical harmonics without the Condon-Shortley phase, from
    scipy's complex ones: Y_l^m(real) = sqrt(2) (-1)^m Re Y_l^m (m > 0),
    sqrt(2) (-1)^m Im Y_l^|m| (m < 0), Y_l^0 (m = 0)."""
    th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    ph = np.arctan2(d[:, 1], d[:, 0])
    out = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            if m == 0:
                out.append(sp.sph_harm_y(l, 0, th, ph).real)
            elif m > 0:
                out.append(math.sqrt(2.0) * (-1) ** m * sp.sph_harm_y(l, m, th, ph).real)
            else:
                out.append(math.sqrt(2.0) * (-1) ** m * sp.sph_harm_y(l, -m, th, ph).imag)
    return np.stack(out, 1)


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_basis_matches_scipy(L):
    rng = np.random.default_rng(L)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = np.concatenate([d, np.eye(3), -np.eye(3)])
    np.testing.assert_allclose(oracle.sh_basis(L, d), _real_sh_scipy(L, d), atol=1e-13)


def test_basis_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi is exact for the products
    of two degree-3 harmonics (degree 6): the Gram matrix is the identity."""
    x, w = np.polynomial.legendre.leggauss(8)
    n_phi = 16
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    wt = np.repeat(w, n_phi) * (2.0 * np.pi / n_phi)
    st = np.sqrt(1.0 - ct ** 2)
    d = np.stack([(st * np.cos(ph)).ravel(), (st * np.sin(ph)).ravel(), ct.ravel()], 1)
    Y = oracle.sh_basis(3, d)
    gram = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-13)


def _sh_scene(L, seed=3, soup=False):
    if soup:
        s = gi.random_triangle_soup(31, 14, spread=0.3, size=0.2, n_views=3, res=(40, 30))
    else:
        # radii jittered: an equilateral facet has lambda1 = lambda2, where the
        # dual numbers through the eigendecomposition (Eq. 10) are singular
        v, f = gi.icosphere(1)
        v = (v * (1.0 + 0.1 * np.random.default_rng(8).normal(size=(len(v), 1)))).astype(np.float32)
        cams = gi.ring_cameras(2, 25.0, 2.7, 48, 40, azimuth0_deg=35.0)
        s = gi.Scene("ico1", v, f, np.zeros((len(f), 3), np.float32), np.full(len(f), 0.85, np.float32), cams)
    rng = np.random.default_rng(seed)
    K = (L + 1) ** 2
    coef = rng.normal(scale=0.3, size=(len(s.faces), K, 3)).astype(np.float32)
    coef[:, 0, :] = rng.uniform(0.2, 1.2, size=(len(s.faces), 3))  # mostly positive colours
    return gi.Scene(s.name, s.verts, s.faces, coef, s.opacity, s.cams)


def test_degree_zero_is_the_face_colour():
    """With only the constant term, colour = a_0 Y_0 + 1/2 in every view:
    the render equals the per-face colour render with that colour."""
    s = _sh_scene(0)
    y0 = 0.5 / math.sqrt(math.pi)
    col = (s.rgb[:, 0, :].astype(np.float64) * y0 + 0.5)
    face = gi.Scene(s.name, s.verts, s.faces, col.astype(np.float32), s.opacity, s.cams)
    # the per-face render reads FP32 colours: compare against the FP32-rounded SH colour
    a0 = ((col.astype(np.float32).astype(np.float64) - 0.5) / y0).astype(np.float32)
    s0 = gi.Scene(s.name, s.verts, s.faces, a0[:, None, :], s.opacity, s.cams)
    r_sh = oracle.render(s0, color_mode=2, sh_degree=0)
    r_face = oracle.render(face)
    np.testing.assert_allclose(r_sh["rgb"], r_face["rgb"], atol=1e-6)
    np.testing.assert_array_equal(r_sh["n_contrib"], r_face["n_contrib"])


def test_colour_depends_on_view_and_clamps_at_zero():
    """A degree-1 colour along the camera axis: the two ring cameras see
    different colours, and a strongly negative coefficient renders black
    (colour clamped at zero, zero colour gradient)."""
    s = _sh_scene(1)
    r = oracle.render(s, color_mode=2, sh_degree=1)
    n = s.cams[0]["width"] * s.cams[0]["height"]
    assert np.abs(r["rgb"][:n].mean(0) - r["rgb"][n:].mean(0)).max() > 1e-3
    neg = s.rgb.copy()
    neg[:, 0, :] = -10.0  # raw colour < 0 in every direction
    sn = gi.Scene(s.name, s.verts, s.faces, neg, s.opacity, s.cams)
    rn = oracle.render(sn, color_mode=2, sh_degree=1)
    np.testing.assert_array_equal(rn["rgb"], 0.0)
    b = oracle.backward(sn, np.ones_like(rn["rgb"]), color_mode=2, sh_degree=1)
    np.testing.assert_array_equal(b["drgb"], 0.0)


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("soup", [False, True])
def test_reverse_matches_dual_numbers(L, soup):
    s = _sh_scene(L, seed=L, soup=soup)
    bg = (0.2, 0.1, 0.4)
    r = oracle.render(s, color_mode=2, sh_degree=L, bg=bg)
    rng = np.random.default_rng(5)
    w = rng.normal(size=r["rgb"].shape)
    w[r["flags"] != 0] = 0.0
    g = oracle.backward(s, w, color_mode=2, sh_degree=L, bg=bg)
    assert g["drgb"].shape == s.rgb.shape
    for _ in range(2):
        dv = rng.normal(size=s.verts.shape)
        dc = rng.normal(size=s.rgb.shape)
        do = rng.normal(size=len(s.faces))
        j = oracle.jvp(s, w, dverts=dv, drgb=dc, dop=do, color_mode=2, sh_degree=L, bg=bg)
        rev = (g["dverts"] * dv).sum() + (g["drgb"] * dc).sum() + (g["dopacity"] * do).sum()
        assert abs(j) > 1e-6
        np.testing.assert_allclose(rev, j, rtol=1e-9)
        # the vertices alone: the colour's direction d depends on the centroid
        jv = oracle.jvp(s, w, dverts=dv, color_mode=2, sh_degree=L, bg=bg)
        np.testing.assert_allclose((g["dverts"] * dv).sum(), jv, rtol=1e-9, atol=1e-12)
        jc = oracle.jvp(s, w, drgb=dc, color_mode=2, sh_degree=L, bg=bg)
        np.testing.assert_allclose((g["drgb"] * dc).sum(), jc, rtol=1e-9, atol=1e-12)


def test_vertex_gradient_by_central_differences():
    """FD of the FP64 render on FP32-representable moves of single vertex
    coordinates (the view direction of the colour moves with the centroid),
    kept only where the +-h renders take the same discrete decisions."""
    s = _sh_scene(2, seed=11)
    r = oracle.render(s, color_mode=2, sh_degree=2)
    rng = np.random.default_rng(2)
    w = rng.normal(size=r["rgb"].shape)
    w[r["flags"] != 0] = 0.0
    g = oracle.backward(s, w, color_mode=2, sh_degree=2)
    checked = 0
    for _ in range(60):
        vi, k = int(rng.integers(len(s.verts))), int(rng.integers(3))
        x0 = np.float32(s.verts[vi, k])
        h = np.float32(2.0 ** -16)
        xs = (np.float32(x0 + h), np.float32(x0 - h))
        vals, same = [], True
        for x in xs:
            v = s.verts.copy()
            v[vi, k] = x
            rp = oracle.render(gi.Scene("p", v, s.faces, s.rgb, s.opacity, s.cams), color_mode=2, sh_degree=2)
            same &= np.array_equal(rp["n_contrib"], r["n_contrib"]) and np.array_equal(rp["last_face"],
                                                                                    r["last_face"])
            vals.append((w * rp["rgb"]).sum())
        if not same:
            continue
        fd = (vals[0] - vals[1]) / (float(xs[0]) - float(xs[1]))
        np.testing.assert_allclose(g["dverts"][vi, k], fd, rtol=2e-3, atol=2e-4)
        checked += 1
    assert checked >= 15
