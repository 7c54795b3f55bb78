"""Cell-subdivision proposer: a small ReLU MLP with a sigmoid output that predicts, for a cell and
an iso-value, whether the cell's subtree holds a finest cell crossed by that iso-surface.

Test infrastructure: see the package docstring.  The paper has no proposer (its cells are kept or
culled by range analysis alone, Algorithm 1); this model is an addition whose labels the method
itself generates (dense evaluation plus the marching-cubes crossing test of Sec. IV-D), and range
analysis stays the fallback wherever the model is not confident.

Model (float64 here):
  x_norm = (x - mu) / sd                                   (fixed per-feature standardisation)
  a_0 = x_norm;  a_l = relu(W_l a_{l-1} + b_l) for hidden l;  z = W_out a + b_out;  p = sigmoid(z)
Loss: binary cross-entropy, mean over the batch, in its stable form
  l(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)),   dl/dz = sigmoid(z) - y.
Backward: the chain rule written out layer by layer (no autograd).
Optimiser: Adam (Kingma & Ba, Algorithm 1) with bias correction.

Features of a (cell, iso) pair (8; the reading of the proposer's input list):
  0-2  cell centre (x, y, z) in [-1, 1]^3
  3    log2 of the cell's half-width h (= -level on the [-1, 1] octree)
  4    the iso-value c_q
  5    (centre of the nearest bounded ancestor's bound) - c_q
  6    spread of that bound (radius for sound bounds, sigma for the Gaussian bound)
  7    level gap between the cell and that ancestor (1 for the parent)
"""
from __future__ import annotations

import numpy as np

DIMS = (8, 64, 64, 64, 1)


def init_params(seed, dims=DIMS):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, from default_rng(seed), layer by layer."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(dims[:-1], dims[1:]):
        params.append((rng.normal(0.0, np.sqrt(2.0 / fi), size=(fo, fi)), np.zeros(fo)))
    return params


def sigmoid(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    pos = z >= 0
    out[pos] = 1.0 / (1.0 + np.exp(-z[pos]))
    ez = np.exp(z[~pos])
    out[~pos] = ez / (1.0 + ez)
    return out


def forward(params, X, mu=None, sd=None):
    """Logits z [n] and the cache of pre-activations / activations for backward."""
    a = np.asarray(X, dtype=np.float64)
    if mu is not None:
        a = (a - mu) / sd
    acts, pres = [a], []
    for l, (W, b) in enumerate(params):
        W = np.asarray(W, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        zl = a @ W.T + b
        pres.append(zl)
        a = np.maximum(zl, 0.0) if l < len(params) - 1 else zl
        acts.append(a)
    return a[:, 0], (acts, pres)


def bce(z, y):
    """Mean binary cross-entropy of logits z against labels y in {0, 1} (stable form)."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def backward(params, cache, y):
    """Gradients of the mean BCE with respect to every (W, b), by the chain rule."""
    acts, pres = cache
    n = acts[0].shape[0]
    z = acts[-1][:, 0]
    delta = ((sigmoid(z) - np.asarray(y, dtype=np.float64)) / n)[:, None]   # dL/dz_out, [n, 1]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], dtype=np.float64)
        grads[l] = (delta.T @ acts[l], delta.sum(axis=0))                    # dL/dW_l, dL/db_l
        if l > 0:
            delta = (delta @ W) * (pres[l - 1] > 0.0)                       # through ReLU l-1
    return grads


def adam_init(params):
    return {"t": 0, "m": [[np.zeros_like(W, dtype=np.float64), np.zeros_like(b, dtype=np.float64)] for W, b in params],
            "v": [[np.zeros_like(W, dtype=np.float64), np.zeros_like(b, dtype=np.float64)] for W, b in params]}


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    state["t"] += 1
    t = state["t"]
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][l][k] = b1 * state["m"][l][k] + (1 - b1) * g
            v = state["v"][l][k] = b2 * state["v"][l][k] + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(np.asarray(p, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps))
        out.append((new[0], new[1]))
    return out


def features(ijk, level, iso, anc_centre, anc_spread, gap):
    """The 8 proposer features of cells (ijk [n, 3] at `level`) for iso-values `iso` [n]."""
    ijk = np.asarray(ijk, dtype=np.float64)
    n = ijk.shape[0]
    level = np.broadcast_to(np.asarray(level, dtype=np.float64), (n,))
    h = 2.0 ** (-level)                                   # half-width: cells of width 2 / 2^level
    X = np.empty((n, 8))
    X[:, 0:3] = -1.0 + (2.0 * ijk + 1.0) * h[:, None]
    X[:, 3] = -level
    X[:, 4] = iso
    X[:, 5] = np.asarray(anc_centre, dtype=np.float64) - iso
    X[:, 6] = anc_spread
    X[:, 7] = gap
    return X


def subtree_labels(crossing_codes, crossing_masks, L, ijk, level):
    """Label masks of cells (ijk at `level`): bit q set iff some finest cell (level L) inside the
    cell is crossed by iso q (its dense corner values straddle c_q).  `crossing_codes` are the
    finest crossing cells as (i, j, k) rows with their iso masks."""
    shift = L - level
    anc = np.asarray(crossing_codes, dtype=np.int64) >> shift
    table = {}
    for key, m in zip(map(tuple, anc.tolist()), np.asarray(crossing_masks, dtype=np.int64).tolist()):
        table[key] = table.get(key, 0) | m
    return np.array([table.get(tuple(c), 0) for c in np.asarray(ijk, dtype=np.int64).tolist()], dtype=np.int64)
