"""Pins of the FP64 oracle of the fitting loop's extra terms
(oracle/fit_terms.py): closed forms, invariances and central differences."""

import math

import numpy as np
import pytest

from oracle import fit_terms as ft


def _fd_grad(fun, v, h=1e-6):
    g = np.zeros_like(v)
    for i in range(v.shape[0]):
        for k in range(v.shape[1]):
            vp, vm = v.copy(), v.copy()
            vp[i, k] += h
            vm[i, k] -= h
            g[i, k] = (fun(vp) - fun(vm)) / (2 * h)
    return g


def _rot():
    a, b, c = 0.3, -1.1, 0.7
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    return Rz @ Ry @ Rx


def _octahedron():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    return v, f


def _hexagon():
    ang = np.arange(6) * math.pi / 3
    v = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang), np.zeros(6)], 1)])
    f = np.array([[0, 1 + k, 1 + (k + 1) % 6] for k in range(6)])
    return v, f


def _bumpy():
    rng = np.random.default_rng(3)
    v, f = _octahedron()
    return v + 0.1 * rng.normal(size=v.shape), f


# ------------------------------------------------------------------ silhouette
def test_bce_closed_forms():
    T = np.array([0.5, 0.25, 1.0, 1e-4])
    m = np.array([1.0, 0.0, 0.0, 1.0])
    loss, dT = ft.silhouette_bce(T, m)
    # -log(0.5), -log(0.25), -log(1 - 1e-6) (clamped mask 1e-6, m = 0), -log(0.9999)
    ref = (math.log(2) + math.log(4) - math.log(1 - 1e-6) - math.log(0.9999)) / 4
    assert abs(loss - ref) <= 1e-15
    np.testing.assert_allclose(dT[:2], [2 / 4, -4 / 4], rtol=1e-15)
    assert dT[2] == 0.0  # M = 0 is clamped
    np.testing.assert_allclose(dT[3], 1 / 0.9999 / 4, rtol=1e-12)


def test_bce_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    T = rng.uniform(0.05, 0.95, 20)
    m = rng.random(20)
    _, dT = ft.silhouette_bce(T, m)
    for i in range(20):
        h = 1e-7
        tp, tm = T.copy(), T.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ft.silhouette_bce(tp, m)[0] - ft.silhouette_bce(tm, m)[0]) / (2 * h)
        assert abs(fd - dT[i]) <= 1e-6 * max(1.0, abs(dT[i]))


# ------------------------------------------------------------------ edge length
def test_edge_loss_closed_forms():
    v = np.array([[0, 0, 0], [3, 0, 0], [3, 4, 0]], dtype=np.float64)
    loss, g = ft.edge_length_loss(v, np.array([[0, 1, 2]]))
    assert abs(loss - 2.0 / 3.0) <= 1e-15  # lengths 3, 4, 5
    s = math.sqrt(2.0)
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / s
    loss, g = ft.edge_length_loss(tet, np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]))
    assert loss <= 1e-30 and np.abs(g).max() <= 1e-15


def test_edge_loss_invariances_and_gradient():
    v, f = _bumpy()
    loss, g = ft.edge_length_loss(v, f)
    assert loss > 1e-4
    R = _rot()
    l2, g2 = ft.edge_length_loss(v @ R.T + np.array([0.3, -2.0, 5.0]), f)
    assert abs(l2 - loss) <= 1e-13 * loss
    np.testing.assert_allclose(g2, g @ R.T, atol=1e-13)
    assert abs(ft.edge_length_loss(2.5 * v, f)[0] - 6.25 * loss) <= 1e-12 * loss
    np.testing.assert_allclose(g.sum(0), 0.0, atol=1e-14)  # translation invariance
    np.testing.assert_allclose(_fd_grad(lambda x: ft.edge_length_loss(x, f)[0], v), g, atol=1e-8)


# ------------------------------------------------------------------ Laplacian
def test_laplacian_closed_forms():
    v, f = _octahedron()
    loss, g = ft.laplacian_loss(v, f)
    assert abs(loss - 1.0) <= 1e-15  # every vertex's face neighbours average to the origin
    v, f = _hexagon()
    loss, _ = ft.laplacian_loss(v, f)
    # centre: delta 0; rim: neighbours (centre twice, two rim neighbours) average to r / 4
    assert abs(loss - 6 * 0.75 ** 2 / 7) <= 1e-15


def test_laplacian_invariances_and_gradient():
    v, f = _bumpy()
    loss, g = ft.laplacian_loss(v, f)
    R = _rot()
    l2, g2 = ft.laplacian_loss(v @ R.T + np.array([1.0, 2.0, -3.0]), f)
    assert abs(l2 - loss) <= 1e-13 * loss
    np.testing.assert_allclose(g2, g @ R.T, atol=1e-13)
    np.testing.assert_allclose(g.sum(0), 0.0, atol=1e-14)
    np.testing.assert_allclose(_fd_grad(lambda x: ft.laplacian_loss(x, f)[0], v), g, atol=1e-8)


# ------------------------------------------------------------------ optimiser, metric
def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=12)
    g = rng.normal(size=12)
    # m_hat = g, v_hat = g^2 after one step
    np.testing.assert_allclose(ft.adam(p0, [g], 1e-3), p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    gn = np.repeat(np.linalg.norm(g.reshape(-1, 3), axis=1), 3)
    np.testing.assert_allclose(ft.adam(p0, [g], 1e-3, group=3), p0 - 1e-3 * g / (gn + 1e-8), rtol=1e-15)


def test_vector_adam_is_rotation_equivariant_and_adam_is_not():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=(5, 3))
    gs = [rng.normal(size=(5, 3)) for _ in range(4)]
    R = _rot()
    for group, equivariant in ((3, True), (1, False)):
        a = ft.adam(p0.ravel(), [g.ravel() for g in gs], 1e-2, group=group).reshape(5, 3)
        b = ft.adam((p0 @ R.T).ravel(), [(g @ R.T).ravel() for g in gs], 1e-2, group=group).reshape(5, 3)
        err = np.abs(a @ R.T - b).max()
        assert (err <= 1e-12) if equivariant else (err >= 1e-6)


def test_chamfer_closed_forms():
    rng = np.random.default_rng(6)
    a = rng.uniform(-1, 1, size=(40, 3)) * np.array([1.0, 1.0, 1.0])
    assert ft.chamfer(a, a) == (0.0, 0.0)
    gaps = np.sqrt(((a[:, None] - a[None]) ** 2).sum(2) + np.eye(40) * 1e9).min()
    t = np.array([1.0, -2.0, 0.5])
    t *= 0.2 * gaps / np.linalg.norm(t)
    ab, ba = ft.chamfer(a, a + t)
    assert abs(ab - t @ t) <= 1e-15 and abs(ba - t @ t) <= 1e-15
    assert ft.chamfer(np.zeros((1, 3)), np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 2.0]])) == (4.0, (4.0 + 25.0) / 2)
