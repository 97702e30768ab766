"""FP64 oracle of the fitting loop's extra terms (test infrastructure; only
the tests import it).

Sec. 3.1 names the losses of the fitting loop without formulas; these are
the definitions the CUDA path implements, written out plainly:

* silhouette loss: binary cross-entropy between the rendered mask
  M = 1 - T_final (clamped to [eps, 1 - eps]) and the target mask m, mean
  over pixels;
* edge-length loss: the variance of the lengths of the 3F face edges
  (interior edges counted once per face that holds them);
* Laplacian smoothing: mean over vertices of |v - n_v|^2, n_v the mean of
  the two other vertices of every face at v;
* Adam / VectorAdam step (VectorAdam is the paper's optimiser);
* chamfer distance (the paper's CD): mean squared nearest-neighbour distance
  from A to B plus from B to A.

Each loss comes with its gradient from the chain rule by hand.
"""

from __future__ import annotations

import numpy as np

BCE_EPS = 1e-6


def silhouette_bce(t_final, mask, eps=BCE_EPS):
    """Mean BCE of M = 1 - T against m and dL/dT (0 where M is clamped)."""
    T = np.asarray(t_final, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    n = T.size
    Mraw = 1.0 - T
    M = np.clip(Mraw, eps, 1.0 - eps)
    Tc = np.clip(T, eps, 1.0 - eps)
    loss = -np.mean(m * np.log(M) + (1.0 - m) * np.log(Tc))
    inside = (Mraw > eps) & (Mraw < 1.0 - eps)
    # dL/dM = -(1/n) (m / M - (1 - m) / (1 - M)); dM/dT = -1
    dT = np.where(inside, (m / M - (1.0 - m) / Tc) / n, 0.0)
    return loss, dT


def edge_length_loss(verts, faces):
    """Variance of the 3F face-edge lengths and its vertex gradient."""
    v = np.asarray(verts, dtype=np.float64)
    f = np.asarray(faces, dtype=np.int64)
    a = np.concatenate([f[:, 0], f[:, 1], f[:, 2]])
    b = np.concatenate([f[:, 1], f[:, 2], f[:, 0]])
    d = v[a] - v[b]
    length = np.sqrt((d * d).sum(1))
    n = len(length)
    mean = length.mean()
    loss = np.mean((length - mean) ** 2)
    # dL/dl_i = (2/n) (l_i - mean) (the mean's own term sums to zero)
    gl = 2.0 / n * (length - mean)
    gd = (gl / np.where(length > 0, length, 1.0))[:, None] * d
    grad = np.zeros_like(v)
    np.add.at(grad, a, gd)
    np.add.at(grad, b, -gd)
    return loss, grad


def laplacian_loss(verts, faces):
    """Mean over vertices of |v - n_v|^2 (n_v over the faces at v) and its
    vertex gradient."""
    v = np.asarray(verts, dtype=np.float64)
    f = np.asarray(faces, dtype=np.int64)
    V = len(v)
    nsum = np.zeros_like(v)
    ncnt = np.zeros(V)
    for k in range(3):
        c, u, w = f[:, k], f[:, (k + 1) % 3], f[:, (k + 2) % 3]
        np.add.at(nsum, c, v[u] + v[w])
        np.add.at(ncnt, c, 2.0)
    has = ncnt > 0
    delta = np.zeros_like(v)
    delta[has] = v[has] - nsum[has] / ncnt[has, None]
    loss = np.mean((delta * delta).sum(1))
    # L = (1/V) sum_w |delta_w|^2, delta_w = w - (1/ncnt_w) sum over faces at
    # w of its two other corners: dL/dv = (2/V) (delta_v - sum over faces at
    # w holding v of delta_w / ncnt_w)
    grad = 2.0 / V * delta
    dn = np.zeros_like(v)
    dn[has] = delta[has] / ncnt[has, None]
    for k in range(3):
        c = f[:, k]
        for j in (1, 2):
            np.add.at(grad, f[:, (k + j) % 3], -2.0 / V * dn[c])
    return loss, grad


def adam(p, grads, lr, b1=0.9, b2=0.999, eps=1e-8, group=1):
    """Parameters after len(grads) Adam (group 1) or VectorAdam (group 3)
    steps from zero moments."""
    p = np.asarray(p, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros(p.size // group)
    for t, g in enumerate(grads, start=1):
        g = np.asarray(g, dtype=np.float64)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * (g.reshape(-1, group) ** 2).sum(1)
        p = p - lr * (m / (1 - b1 ** t)) / (np.repeat(np.sqrt(v / (1 - b2 ** t)), group) + eps)
    return p


def chamfer(a, b):
    """(mean_a min_b |a - b|^2, mean_b min_a |b - a|^2) by brute force."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = ((a[:, None, :] - b[None, :, :]) ** 2).sum(2)
    return d.min(1).mean(), d.min(0).mean()
