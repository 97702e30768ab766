"""The fitting loop around the renderer: the Adam / VectorAdam step, the
chamfer distance and the mesh regularisers against the FP64 oracle of
these terms, a
short fit that lowers the image loss and the chamfer distance in both the
batched and the per-view form, and the first step's gradients on the
level-7 fitting problem (4 views of 512^2) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from oracle import fit_terms
from gpu_util import DEV, GRAD_TOL, rel_l2, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("group", [1, 3])
def test_adam_step_against_fp64(group):
    from paper_2602_14493_b300 import Renderer

    rng = np.random.default_rng(group)
    n = 3 * 5003
    p0 = rng.normal(size=n).astype(np.float32)
    gs = [rng.normal(scale=s, size=n).astype(np.float32) for s in (1.0, 0.01, 3.0, 1e-4)]
    r = Renderer()
    p = torch.from_numpy(p0).to(DEV)
    m = torch.zeros_like(p)
    v = torch.zeros(n // group, device=DEV)
    for t, g in enumerate(gs, start=1):
        r.adam_step(p, torch.from_numpy(g).to(DEV), m, v, 1e-3, t, group=group)
    ref = fit_terms.adam(p0, gs, 1e-3, group=group)
    step = ref - p0
    assert np.abs(p.cpu().numpy().astype(np.float64) - ref).max() <= 1e-6 + 1e-5 * np.abs(step).max()
    r.close()


def test_chamfer_against_brute_force():
    from paper_2602_14493_b300 import Renderer

    rng = np.random.default_rng(7)
    a = rng.normal(size=(3001, 3)).astype(np.float32)
    b = (rng.normal(size=(1777, 3)) * 0.7 + 0.1).astype(np.float32)
    r = Renderer()
    out = r.chamfer(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)).cpu().numpy()
    np.testing.assert_allclose(out, np.array(fit_terms.chamfer(a, b)), rtol=2e-6)
    # identical sets: zero
    z = r.chamfer(torch.from_numpy(a).to(DEV), torch.from_numpy(a).to(DEV)).cpu().numpy()
    assert np.all(z == 0.0)
    r.close()


@pytest.mark.parametrize("optimizer", ["adam", "vectoradam"])
def test_short_fit_lowers_loss_and_chamfer(optimizer):
    from paper_2602_14493_b300.fit import fit

    s = gi.scene_fit(level=5, res=256, views_per_step=4, steps=40)
    out_b = fit(s, lr=2e-3, form="batched", optimizer=optimizer)
    out_p = fit(s, lr=2e-3, form="per_view", optimizer=optimizer)
    for out in (out_b, out_p):
        assert out["status"] == 0
        assert np.all(np.isfinite(out["loss"]))
        assert out["loss"][-5:].mean() < 0.8 * out["loss"][:5].mean()
        assert out["chamfer_final"] < 0.8 * out["chamfer_initial"]
    # the two forms compute the same step (up to the order of float atomics)
    np.testing.assert_allclose(out_b["loss"][:3], out_p["loss"][:3], rtol=1e-5)
    assert abs(out_b["chamfer_final"] - out_p["chamfer_final"]) <= 0.05 * out_b["chamfer_final"]


def test_short_fit_with_silhouette_and_regularizers():
    """All four losses of the paper's fitting loop (image, silhouette,
    edge length, Laplacian) with VectorAdam: every loss term is finite, the
    image and silhouette losses fall, and the batched and per-view forms take
    the same first steps."""
    from paper_2602_14493_b300.fit import fit

    s = gi.scene_fit(level=4, res=128, views_per_step=4, steps=30)
    kw = dict(lr=2e-3, optimizer="vectoradam", w_silhouette=2e3, w_edge=1e2, w_laplacian=1e2)
    out_b = fit(s, form="batched", **kw)
    out_p = fit(s, form="per_view", **kw)
    for out in (out_b, out_p):
        assert out["status"] == 0
        for key in ("loss", "silhouette_loss", "regularizer_losses"):
            assert np.all(np.isfinite(out[key]))
        assert out["loss"][-5:].mean() < 0.9 * out["loss"][:5].mean()
        assert out["silhouette_loss"][-5:].mean() < out["silhouette_loss"][:5].mean()
        assert np.all(out["regularizer_losses"] > 0)
    np.testing.assert_allclose(out_b["loss"][:3], out_p["loss"][:3], rtol=1e-5)
    np.testing.assert_allclose(out_b["silhouette_loss"][:3], out_p["silhouette_loss"][:3], rtol=1e-5)


def test_fit_first_step_gradients_match_oracle():
    """Level-7 fitting problem (327,680 faces, 4 views of 512^2): the first
    step's dL/dI = 2 (I - I*) kept on sampled pixels; gradients of the
    vertices and colours against the oracle's backward over those pixels."""
    from paper_2602_14493_b300 import Renderer, camera_array

    s = gi.scene_fit(steps=1)
    cams = s.extra["view_sets"][0]
    r = Renderer()
    v, f, c, o = to_dev(s)
    tv = torch.from_numpy(s.extra["target_verts"]).to(DEV)
    tc = torch.from_numpy(s.extra["target_rgb"]).to(DEV)
    target, _ = r.forward(tv, f, tc, o, camera_array(cams), want_t=False)
    target = target.clone()
    img, _ = r.forward(v, f, c, o, camera_array(cams), want_t=False)
    pix, lin = sample_pixels(cams, 256, 501, window=8)
    ref = oracle.render(s, pixels=pix)
    g_s = 2.0 * (img.cpu().numpy()[lin] - target.cpu().numpy()[lin])
    g_s[ref["flags"] != 0] = 0.0
    g = np.zeros((img.shape[0], 3), dtype=np.float32)
    g[lin] = g_s
    dv, dc, do = r.backward(torch.from_numpy(g).to(DEV))
    torch.cuda.synchronize()
    ob = oracle.backward(s, g_s.astype(np.float64), pixels=pix)
    assert np.abs(ob["dverts"]).max() > 0
    assert rel_l2(dv.cpu().numpy(), ob["dverts"]) <= GRAD_TOL
    assert rel_l2(dc.cpu().numpy(), ob["drgb"]) <= GRAD_TOL
    r.close()


@pytest.mark.parametrize("level", [2, 4])
def test_mesh_regularizers_match_oracle(level):
    """Edge-length and Laplacian losses and their weighted vertex gradients
    (added to a non-zero dL/dverts) against the FP64 oracle, on a randomly
    bumped icosphere."""
    from paper_2602_14493_b300 import Renderer

    v, f = gi.icosphere(level)
    rng = np.random.default_rng(level)
    v = (v * (1.0 + 0.1 * rng.normal(size=(len(v), 1)))).astype(np.float32)
    r = Renderer()
    vd = torch.from_numpy(v).to(DEV)
    fd = torch.from_numpy(f).to(DEV)
    base = (1e-6 * rng.normal(size=v.shape)).astype(np.float32)  # small: recovering g = dv - base stays exact-ish
    dv = torch.from_numpy(base).to(DEV)
    losses = r.mesh_regularizers(vd, fd, w_edge=0.7, w_lap=1.3, dverts=dv).cpu().numpy()
    le, ge = fit_terms.edge_length_loss(v, f)
    ll, gl = fit_terms.laplacian_loss(v, f)
    # FP32: the edge variance cancels (l - mean l) to ~10% of l
    assert abs(losses[0] - le) <= 1e-4 * le
    assert abs(losses[1] - ll) <= 1e-5 * ll
    g = dv.cpu().numpy().astype(np.float64) - base
    assert rel_l2(g, 0.7 * ge + 1.3 * gl) <= 1e-5
    # losses only (the neighbour sums are float atomics: equal up to their order)
    l2 = r.mesh_regularizers(vd, fd).cpu().numpy()
    np.testing.assert_allclose(l2, losses, rtol=1e-6)
    r.close()
