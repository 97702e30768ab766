"""Pins of the oracle's hand-derived reverse pass: forward-mode dual numbers
through the forward code (including the eigen route of Eq. 10-13), and
central finite differences of the FP64 render."""

import numpy as np
import pytest

import gmr_inputs as gi
import oracle


def _weights(scene, seed, **kw):
    """Random dL/dI, zero on pixels with a decision near its threshold."""
    r = oracle.render(scene, **kw)
    rng = np.random.default_rng(seed)
    w = rng.normal(size=r["rgb"].shape)
    w[r["flags"] != 0] = 0.0
    return w


def _scenes():
    soup = gi.random_triangle_soup(21, 12, spread=0.3, size=0.2, n_views=2, res=(40, 30))
    v, f = gi.icosphere(1)
    rng = np.random.default_rng(8)
    v = (v * (1.0 + 0.1 * rng.normal(size=(len(v), 1)))).astype(np.float32)
    cams = gi.ring_cameras(1, 30.0, 2.6, 48, 48, azimuth0_deg=10.0)
    ico = gi.Scene("ico1", v, f, rng.random((len(f), 3)).astype(np.float32),
                   rng.uniform(0.5, 1.0, len(f)).astype(np.float32), cams)
    return [soup, ico]


@pytest.mark.parametrize("cov_mode", [0, 1])
@pytest.mark.parametrize("color_mode", [0, 1])
@pytest.mark.parametrize("which", [0, 1])
def test_reverse_matches_dual_numbers(cov_mode, color_mode, which):
    s = _scenes()[which]
    if color_mode == 1:
        rng = np.random.default_rng(4)
        s = gi.Scene(s.name, s.verts, s.faces, rng.random((len(s.verts), 3)).astype(np.float32), s.opacity, s.cams)
    bg = (0.3, 0.6, 0.1)
    w = _weights(s, 1, cov_mode=cov_mode, color_mode=color_mode, bg=bg)
    g = oracle.backward(s, w, cov_mode=cov_mode, color_mode=color_mode, bg=bg)
    rng = np.random.default_rng(2)
    for trial in range(3):
        dv = rng.normal(size=s.verts.shape)
        dc = rng.normal(size=s.rgb.shape)
        do = rng.normal(size=len(s.faces))
        j = oracle.jvp(s, w, dverts=dv, drgb=dc, dop=do, cov_mode=cov_mode, color_mode=color_mode, bg=bg)
        rev = (g["dverts"] * dv).sum() + (g["drgb"] * dc).sum() + (g["dopacity"] * do).sum()
        assert abs(j) > 1e-6
        np.testing.assert_allclose(rev, j, rtol=1e-9)
        # each input group separately
        jv = oracle.jvp(s, w, dverts=dv, cov_mode=cov_mode, color_mode=color_mode, bg=bg)
        np.testing.assert_allclose((g["dverts"] * dv).sum(), jv, rtol=1e-9, atol=1e-12)


def test_reverse_matches_central_differences():
    """FD on FP32-representable perturbations of single vertex coordinates;
    only components whose +-h renders take the same discrete decisions."""
    s = _scenes()[1]
    w = _weights(s, 5)
    g = oracle.backward(s, w)
    base = oracle.render(s)
    rng = np.random.default_rng(9)
    checked = 0
    for _ in range(40):
        vi, k = int(rng.integers(len(s.verts))), int(rng.integers(3))
        x0 = np.float32(s.verts[vi, k])
        h = np.float32(2.0 ** -12)
        xp, xm = np.float32(x0 + h), np.float32(x0 - h)
        vals, same = [], True
        for x in (xp, xm):
            v = s.verts.copy()
            v[vi, k] = x
            sv = gi.Scene("p", v, s.faces, s.rgb, s.opacity, s.cams)
            r = oracle.render(sv)
            same &= np.array_equal(r["n_contrib"], base["n_contrib"]) and np.array_equal(r["last_face"], base["last_face"])
            vals.append((w * r["rgb"]).sum())
        if not same:
            continue
        fd = (vals[0] - vals[1]) / (float(xp) - float(xm))
        an = g["dverts"][vi, k]
        assert abs(fd - an) <= 2e-3 * max(abs(an), 1e-3 * np.abs(g["dverts"]).max()), (vi, k, fd, an)
        checked += 1
    assert checked >= 15


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("with_image", [False, True])
def test_reverse_with_final_transmittance_matches_dual_numbers(which, with_image):
    """dL/dT_final (the silhouette's gradient, T_N = prod (1 - alpha_j)) in
    the reverse pass against dual numbers through the forward, alone and
    together with dL/dI."""
    s = _scenes()[which]
    bg = (0.3, 0.6, 0.1)
    r = oracle.render(s, bg=bg)
    rng = np.random.default_rng(13)
    wT = rng.normal(size=len(r["T"]))
    wT[r["flags"] != 0] = 0.0
    w = _weights(s, 3, bg=bg) if with_image else np.zeros_like(r["rgb"])
    g = oracle.backward(s, w, bg=bg, dLdT=wT)
    for trial in range(3):
        dv = rng.normal(size=s.verts.shape)
        do = rng.normal(size=len(s.faces))
        j = oracle.jvp(s, w, dverts=dv, dop=do, bg=bg, wT=wT)
        rev = (g["dverts"] * dv).sum() + (g["dopacity"] * do).sum()
        assert abs(j) > 1e-6
        np.testing.assert_allclose(rev, j, rtol=1e-9)
    if not with_image:
        # T_final does not depend on the colours
        assert np.all(g["drgb"] == 0.0)


def test_final_transmittance_reverse_matches_central_differences():
    s = _scenes()[1]
    base = oracle.render(s)
    rng = np.random.default_rng(17)
    wT = rng.normal(size=len(base["T"]))
    wT[base["flags"] != 0] = 0.0
    g = oracle.backward(s, np.zeros_like(base["rgb"]), dLdT=wT)
    checked = 0
    for _ in range(80):
        vi, k = int(rng.integers(len(s.verts))), int(rng.integers(3))
        x0 = np.float32(s.verts[vi, k])
        h = np.float32(2.0 ** -12)
        xp, xm = np.float32(x0 + h), np.float32(x0 - h)
        vals, same = [], True
        for x in (xp, xm):
            v = s.verts.copy()
            v[vi, k] = x
            r = oracle.render(gi.Scene("p", v, s.faces, s.rgb, s.opacity, s.cams))
            same &= np.array_equal(r["n_contrib"], base["n_contrib"]) and np.array_equal(r["last_face"], base["last_face"])
            vals.append((wT * r["T"]).sum())
        if not same:
            continue
        fd = (vals[0] - vals[1]) / (float(xp) - float(xm))
        an = g["dverts"][vi, k]
        assert abs(fd - an) <= 2e-3 * max(abs(an), 1e-3 * np.abs(g["dverts"]).max()), (vi, k, fd, an)
        checked += 1
    assert checked >= 15
