"""The fitting loop around the renderer: the Adam / VectorAdam step and the
chamfer distance against plain FP64 restatements of their definitions, a
short fit that lowers the image loss and the chamfer distance in both the
batched and the per-view form, and the first step's gradients on the
level-7 fitting problem (4 views of 512^2) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import gmr_inputs as gi
import oracle
from gpu_util import DEV, GRAD_TOL, rel_l2, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


def _adam_ref(p, g_steps, lr, b1, b2, eps, group):
    """FP64 Adam (group 1) / VectorAdam (group 3), written from the update
    rule: m and v are exponential averages of g and g^2 (|g|^2 per 3-vector),
    bias-corrected by 1 - b^t."""
    p = p.astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros(p.size // group)
    for t, g in enumerate(g_steps, start=1):
        g = g.astype(np.float64)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * (g.reshape(-1, group) ** 2).sum(1)
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p = p - lr * mh / (np.repeat(np.sqrt(vh), group) + eps)
    return p


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
    ref = _adam_ref(p0, gs, 1e-3, 0.9, 0.999, 1e-8, group)
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
    d = ((a[:, None, :].astype(np.float64) - b[None, :, :]) ** 2).sum(2)
    ref = np.array([d.min(1).mean(), d.min(0).mean()])
    np.testing.assert_allclose(out, ref, rtol=2e-6)
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
