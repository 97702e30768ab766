"""Synthetic inputs: mesh topology, camera geometry, determinism."""

import math

import numpy as np
import pytest

import gmr_inputs as gi


@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_icosphere_counts_and_topology(level):
    v, f = gi.icosphere(level)
    assert len(v) == 10 * 4 ** level + 2 and len(f) == 20 * 4 ** level
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)
    # closed 2-manifold: every undirected edge in exactly two faces, Euler = 2
    e = np.sort(np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(cnt == 2)
    assert len(v) - len(cnt) + len(f) == 2
    # outward orientation
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    assert np.all(np.einsum("ij,ij->i", n, v[f].mean(1)) > 0)


def test_look_at_geometry():
    cam = gi.look_at((3.0, 0.0, 0.0), 64, 32)
    R = cam["R"].reshape(3, 3).astype(np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert np.linalg.det(R) > 0.99
    # the target projects to the principal point, in front of the camera
    tc = R @ np.zeros(3) + cam["t"]
    assert tc[2] > 2.99
    assert abs(float(cam["fx"]) - 32 / math.tan(math.radians(25))) < 1e-3
    # world +z points up in the image (negative image y)
    up = R @ np.array([0, 0, 1.0])
    assert up[1] < -0.99


def test_scenes_deterministic_and_shaped():
    a, b = gi.scene_ring(), gi.scene_ring()
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.rgb, b.rgb)
    assert a.verts.dtype == np.float32 and a.faces.dtype == np.int32
    assert len(a.cams) == 8 and a.n_pixels == 8 * 512 * 512
    r = np.linalg.norm(a.verts, axis=1)
    assert r.min() > 0.89 and r.max() < 1.11
    s3 = gi.scene_fibonacci_uneven(level=2, n_views=64)
    res = set(int(c["width"]) for c in s3.cams)
    assert res <= set(gi.RESOLUTION_SET) and len(res) >= 4
    assert np.all((s3.rgb >= 0) & (s3.rgb <= 1))


def test_noise_fields():
    p = np.random.default_rng(0).normal(size=(1000, 3))
    n = gi.perlin_noise3(p, 3)
    assert np.all(np.abs(n) <= 1.5) and n.std() > 0.05
    # Perlin noise vanishes on the integer lattice
    np.testing.assert_allclose(gi.perlin_noise3(np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]]), 3), 0, atol=1e-12)
    vn = gi.value_noise3(p, 5)
    assert np.all((vn >= 0) & (vn <= 1))
