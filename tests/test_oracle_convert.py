"""Pins of the oracle's facet-to-Gaussian conversion (Sec. 2.2, Eq. 3-15)
against closed forms, exact quadrature, and invariants of the mathematics."""

import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KAPPA = 6.0 * math.sqrt(3.0) / math.pi
SZ2 = 1e-12


def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def _tri(a, b, c):
    return np.array([a, b, c], dtype=np.float64), np.array([[0, 1, 2]], dtype=np.int32)


def test_right_isosceles_golden():
    g = _golden_kv("right_isosceles.txt")
    v, f = _tri((0, 0, 0), (1, 0, 0), (0, 1, 0))
    r = oracle.convert(v, f, cov_mode=1)
    sxx, sxy, syy, l1, l2, kap, area, deg = r["aux"][0]
    assert deg == 0
    np.testing.assert_allclose(r["means"][0], [g["mean_x"], g["mean_y"], g["mean_z"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose([sxx, sxy, syy], [g["sxx"], g["sxy"], g["syy"]], rtol=1e-13)
    np.testing.assert_allclose([l1, l2], [g["lam1"], g["lam2"]], rtol=1e-13)
    np.testing.assert_allclose([area, kap], [g["area"], g["kappa"]], rtol=1e-13)
    # Eq. 15 literally: the raw 2D covariance embedded in the facet plane.
    expect = np.array([[g["sxx"], g["sxy"], 0], [g["sxy"], g["syy"], 0], [0, 0, 0]])
    np.testing.assert_allclose(r["cov"][0], expect, atol=1e-15)
    # Eq. 13 (default): kappa-scaled in-plane, s_z^2 along the normal.
    r0 = oracle.convert(v, f, cov_mode=0)
    expect0 = KAPPA * expect + np.diag([0, 0, SZ2])
    np.testing.assert_allclose(r0["cov"][0], expect0, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("row", [0, 1])
def test_equilateral_golden(row):
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "equilateral.txt"))
            if l.strip() and not l.startswith("#")]
    L, lam, area, sx2 = rows[row]
    # an arbitrarily placed and oriented equilateral triangle
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    base = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * math.sqrt(3) / 2, 0]])
    v = base @ Q.T + np.array([0.3, -0.2, 0.7])
    r = oracle.convert(v, np.array([[0, 1, 2]], dtype=np.int32), cov_mode=0)
    _, _, _, l1, l2, kap, ar, _ = r["aux"][0]
    np.testing.assert_allclose([l1, l2], [lam, lam], rtol=1e-9)
    np.testing.assert_allclose(ar, area, rtol=1e-12)
    ev = np.linalg.eigvalsh(r["cov"][0])
    np.testing.assert_allclose(ev[1:], [sx2, sx2], rtol=1e-9)
    # area matching of Eq. 12: the 1-sigma ellipse has the facet's area
    np.testing.assert_allclose(math.pi * math.sqrt(ev[1] * ev[2]), area, rtol=1e-9)


def _random_tris(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n * 3, 3)) * scale
    f = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    return v, f


def test_edge_midpoint_quadrature():
    """Eq. 6-9 against an independent exact rule: the mean of a quadratic
    over a triangle equals its mean over the three edge midpoints, so the
    covariance of the uniform density is the covariance of those points
    about the centroid (Eq. 15 embeds exactly that 2D covariance)."""
    v, f = _random_tris(200, 11)
    r = oracle.convert(v, f, cov_mode=1)
    for k in range(len(f)):
        p = v[f[k]]
        m = p.mean(0)
        mids = np.array([(p[0] + p[1]) / 2, (p[1] + p[2]) / 2, (p[2] + p[0]) / 2])
        cov = (mids.T @ mids) / 3.0 - np.outer(m, m)
        np.testing.assert_allclose(r["means"][k], m, atol=1e-12 * np.abs(p).max())
        np.testing.assert_allclose(r["cov"][k], cov, atol=1e-12 * np.abs(cov).max())


def test_area_mode_is_kappa_times_embed():
    """Eq. 13 via Eq. 14 equals the kappa-scaled Eq. 15 plus s_z^2 n n^T;
    lambda1 lambda2 = det Sigma2D = |A|^2/108, so kappa = 6 sqrt(3)/pi."""
    v, f = _random_tris(300, 12)
    a = oracle.convert(v, f, cov_mode=0)
    b = oracle.convert(v, f, cov_mode=1)
    n = a["frame"][:, 2, :]
    for k in range(len(f)):
        expect = KAPPA * b["cov"][k] + SZ2 * np.outer(n[k], n[k])
        np.testing.assert_allclose(a["cov"][k], expect, rtol=1e-10, atol=1e-13 * np.abs(expect).max())
    sxx, sxy, syy, l1, l2, kap, area = [a["aux"][:, i] for i in range(7)]
    np.testing.assert_allclose(l1 * l2, sxx * syy - sxy ** 2, rtol=1e-10)
    np.testing.assert_allclose(l1 * l2, area ** 2 / 108.0, rtol=1e-10)
    np.testing.assert_allclose(kap, KAPPA, rtol=1e-10)
    assert np.all(l1 >= l2)


def test_eigen_matches_library():
    v, f = _random_tris(100, 13)
    r = oracle.convert(v, f, cov_mode=0)
    for k in range(len(f)):
        sxx, sxy, syy, l1, l2 = r["aux"][k][:5]
        ev = np.linalg.eigvalsh(np.array([[sxx, sxy], [sxy, syy]]))
        np.testing.assert_allclose([l2, l1], ev, rtol=1e-10, atol=1e-16)


def test_invariants_permutation_rigid_psd_planar():
    v, f = _random_tris(100, 14)
    base = oracle.convert(v, f, cov_mode=0)
    for perm in ([1, 2, 0], [2, 0, 1], [0, 2, 1], [2, 1, 0]):
        r = oracle.convert(v, f[:, perm], cov_mode=0)
        np.testing.assert_allclose(r["means"], base["means"], atol=1e-12)
        np.testing.assert_allclose(r["cov"], base["cov"], atol=1e-11 * np.abs(base["cov"]).max())
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    t = np.array([1.5, -0.25, 3.0])
    r = oracle.convert(v @ Q.T + t, f, cov_mode=0)
    np.testing.assert_allclose(r["means"], base["means"] @ Q.T + t, atol=1e-12)
    rot = np.einsum("ij,fjk,lk->fil", Q, base["cov"], Q)
    np.testing.assert_allclose(r["cov"], rot, atol=1e-11 * np.abs(rot).max())
    for k in range(len(f)):
        ev = np.linalg.eigvalsh(base["cov"][k])
        assert ev.min() > -1e-15
        n = base["frame"][k, 2]
        p = v[f[k]]
        nn = np.cross(p[1] - p[0], p[2] - p[0])
        nn /= np.linalg.norm(nn)
        np.testing.assert_allclose(abs(n @ nn), 1.0, rtol=1e-12)
        # planar: the normal is an eigenvector with eigenvalue s_z^2
        np.testing.assert_allclose(base["cov"][k] @ n, SZ2 * n, atol=1e-12 * np.abs(base["cov"][k]).max())


def test_degenerate_and_tiny_facets():
    # collinear vertices: zero area -> zero-covariance point at the mean
    v, f = _tri((0, 0, 0), (1, 0, 0), (2, 0, 0))
    r = oracle.convert(v, f, cov_mode=0)
    assert r["aux"][0][7] == 1
    np.testing.assert_allclose(r["means"][0], [1, 0, 0])
    assert np.all(r["cov"][0] == 0)
    # coincident vertices
    v, f = _tri((0.5, 0.5, 0.5), (0.5, 0.5, 0.5), (1, 0, 0))
    assert oracle.convert(v, f)["aux"][0][7] == 1
    # tiny facet below the epsilon clamp of Eq. 12: kappa = |A| / (pi sqrt(eps))
    s = 1e-4
    v, f = _tri((0, 0, 0), (s, 0, 0), (0, s, 0))
    r = oracle.convert(v, f, cov_mode=0)
    area = r["aux"][0][6]
    np.testing.assert_allclose(area, s * s / 2, rtol=1e-12)
    assert area ** 2 / 108 < 1e-14
    np.testing.assert_allclose(r["aux"][0][5], area / (math.pi * 1e-7), rtol=1e-12)
    # face index out of range is an error
    with pytest.raises(ValueError):
        oracle.convert(np.zeros((3, 3)), np.array([[0, 1, 3]], dtype=np.int32))
