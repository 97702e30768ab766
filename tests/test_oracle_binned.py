"""The oracle's binned mode (each pixel walks the faces its 16 x 16-pixel grid
cell lists, from each face's FP64 support, instead of every visible face)
against its brute force: the same decisions in the same order, so images,
final transmittance, last contributor, contributor counts, ambiguity flags,
reverse-mode gradients and dual-number derivatives agree bit for bit -- on
the single-view workload (every pixel), a random sample of the 8-view ring
workload, and random triangle soups with large, elongated, overlapping faces
on ragged image sizes."""

import numpy as np
import pytest

import gmr_inputs as gi
import oracle


@pytest.fixture
def brute_after():
    yield
    oracle.set_binned(False)


def _both(scene, pixels=None, color_mode=0, sh_degree=0, with_T=True, jvp=False):
    out = []
    for binned in (False, True):
        oracle.set_binned(binned)
        r = oracle.render(scene, pixels=pixels, color_mode=color_mode, sh_degree=sh_degree)
        rng = np.random.default_rng(5)
        g = rng.normal(size=r["rgb"].shape)
        gT = rng.normal(size=r["T"].shape) if with_T else None
        b = oracle.backward(scene, g, pixels=pixels, color_mode=color_mode, sh_degree=sh_degree, dLdT=gT)
        j = None
        if jvp:
            dv = np.random.default_rng(6).normal(size=scene.verts.shape)
            j = oracle.jvp(scene, g, dverts=dv, pixels=pixels, color_mode=color_mode, sh_degree=sh_degree)
        out.append((r, b, j))
    return out


def _assert_same(a, b):
    (r0, b0, j0), (r1, b1, j1) = a, b
    for k in r0:
        np.testing.assert_array_equal(r0[k], r1[k], err_msg=k)
    for k in b0:
        np.testing.assert_array_equal(b0[k], b1[k], err_msg=k)
    if j0 is not None:
        np.testing.assert_array_equal(np.asarray(j0), np.asarray(j1))


def test_binned_equals_brute_force_single_view(brute_after):
    s = gi.scene_single_view()
    a, b = _both(s, jvp=True)
    _assert_same(a, b)
    assert a[0]["n_contrib"].sum() > 0 and np.abs(a[1]["dverts"]).sum() > 0


def test_binned_equals_brute_force_ring_sample(brute_after):
    s = gi.scene_ring()
    rng = np.random.default_rng(12)
    pix = []
    for _ in range(3000):
        c = int(rng.integers(len(s.cams)))
        pix.append((c, int(rng.integers(int(s.cams[c]["width"]))), int(rng.integers(int(s.cams[c]["height"])))))
    pix = np.unique(np.array(pix, dtype=np.int32), axis=0)
    a, b = _both(s, pixels=pix, with_T=False)
    _assert_same(a, b)
    assert a[0]["n_contrib"].sum() > 1000


@pytest.mark.parametrize("seed,size,res", [(1, 0.15, (64, 48)), (2, 0.45, (37, 53)), (3, 0.8, (90, 17))])
def test_binned_equals_brute_force_soups(brute_after, seed, size, res):
    s = gi.random_triangle_soup(seed, 80, size=size, n_views=3, res=res)
    a, b = _both(s, jvp=True)
    _assert_same(a, b)
    assert a[0]["n_contrib"].sum() > 0


def test_binned_equals_brute_force_view_dependent_colour(brute_after):
    s0 = gi.random_triangle_soup(4, 50, size=0.3, n_views=2, res=(48, 40))
    sh = np.random.default_rng(9).normal(0.0, 0.3, size=(len(s0.faces), 4, 3)).astype(np.float32)
    s = gi.Scene(s0.name, s0.verts, s0.faces, sh, s0.opacity, s0.cams)
    a, b = _both(s, color_mode=2, sh_degree=1)
    _assert_same(a, b)


def test_binned_mode_refuses_wider_bands(brute_after):
    s = gi.random_triangle_soup(1, 10, n_views=1, res=(16, 16))
    oracle.set_binned(True)
    with pytest.raises(ValueError):
        oracle.render(s, bands=(2 * oracle.BINNED_MAX_ALPHA_BAND, 2e-4))
    assert oracle.set_binned(False) is True
