"""The oracle's OpenMP loops (over pixels, records and faces) give results
that do not depend on the thread count: every sum is formed in the same order
as with one thread, so one and eight threads agree bit for bit."""

import numpy as np
import pytest

import gmr_inputs as gi
import oracle


@pytest.fixture
def restore_threads():
    yield
    oracle.set_threads(0)


def _run(scene, threads, color_mode=0, with_T=False):
    oracle.set_threads(threads)
    r = oracle.render(scene, color_mode=color_mode)
    rng = np.random.default_rng(7)
    g = rng.normal(size=r["rgb"].shape)
    gT = rng.normal(size=r["T"].shape) if with_T else None
    b = oracle.backward(scene, g, color_mode=color_mode, dLdT=gT)
    return r, b


@pytest.mark.parametrize("color_mode", [0, 1])
def test_threads_bit_identical_single_view(restore_threads, color_mode):
    s = gi.scene_single_view(level=3, width=72, height=56)
    if color_mode == 1:
        s = gi.Scene(s.name, s.verts, s.faces,
                     np.random.default_rng(3).uniform(size=(len(s.verts), 3)).astype(np.float32), s.opacity, s.cams)
    r1, b1 = _run(s, 1, color_mode)
    r8, b8 = _run(s, 8, color_mode)
    for k in r1:
        np.testing.assert_array_equal(r1[k], r8[k], err_msg=k)
    for k in b1:
        np.testing.assert_array_equal(b1[k], b8[k], err_msg=k)
    assert np.abs(b1["dverts"]).sum() > 0


def test_threads_bit_identical_several_views_with_final_T(restore_threads):
    s = gi.random_triangle_soup(11, 60, n_views=3, res=(40, 36))
    r1, b1 = _run(s, 1, with_T=True)
    r3, b3 = _run(s, 3, with_T=True)
    for k in r1:
        np.testing.assert_array_equal(r1[k], r3[k], err_msg=k)
    for k in b1:
        np.testing.assert_array_equal(b1[k], b3[k], err_msg=k)


def test_set_threads_all_cores(restore_threads):
    import os

    n = oracle.set_threads(0)
    assert n >= 1
    assert n <= (os.cpu_count() or n)
    assert oracle.set_threads(2) == 2
