"""Per-result parity bands for the BF16 tensor-core bounds: a rounding-noise model run through the
float64 layer loop (test infrastructure; the exact values always come from the oracle).

Model.  Every quantity the BF16 path rounds to bfloat16 is taken as its exact value times
(1 + u_b d), d independent and uniform on [-1, 1], u_b = 2^-8 (round to nearest; the uniform law
over-states the variance of a rounding error).  Quantities carried as two BF16 terms (the centre and
the three input-symbol rows) take 2^-16 instead.  Per hidden linear layer j = 1 .. H-1 of the
row-batched path the rounded quantities are:
  - W_j as the symbol-row GEMM reads it (one draw per weight, shared by every cell of a draw);
  - the GEMM's A operand x * alpha, every entry of every stored symbol row;
  - every entry of the GEMM's stored result and of the new rows gamma_n W_j[:, n];
  - the operands of the centre and input-row products, W_j and the post-activation centre and rows
    (two-term operands, so an error relative to each product, not to the possibly cancelling sum).
Layer 0 and the output layer run in float32 on stored values and add no rounding of their own;
the reductions and linearisations (Eq. 2 / 7, Eq. 4, Table VII) are float32 and their 2^-24
errors are left out.  The linearisation of every draw is the oracle's, so the feedback of rounding
errors through alpha, beta and gamma is part of the model.

Band.  K draws give K perturbed results per box; the band of a result is B x RMS(draw - exact)
plus a float32 floor 64 u (|x0| + spread), u = 2^-24.  With K = 12 and B = 10, a result whose true
error follows the model leaves its band with probability 3.6e-7 (the RMS of 12 draws is a
chi-distributed estimate of the standard deviation; averaging the Gaussian tail over it gives that
figure).  It is a statistical band: the central-limit argument of Sec. IV applied to rounding
errors.  A worst-case bound for BF16 adds the errors' magnitudes and is about a hundred times wider
than any error measured.
"""
from __future__ import annotations

import numpy as np

from oracle import activations, affine
from oracle.mlp import as_f64_layers

UB = 2.0 ** -8          # bfloat16 unit roundoff
U2 = 2.0 ** -16         # two-term bfloat16 operand
U32 = 2.0 ** -24        # float32 unit roundoff
K_DRAWS = 12
B_FACTOR = 10.0


def _mul(rng, a, u):
    return a * (1.0 + u * rng.uniform(-1.0, 1.0, size=a.shape))


def noisy_propagate(layers, lo, hi, mode, rng, act="relu"):
    """Output centre (B,) and coefficients (B, S) of one draw of the rounding model (the layer loop
    of affine.propagate with the model's perturbations)."""
    L = as_f64_layers(layers)
    prop = affine.CLT if mode == affine.CLT else affine.SOUND
    c, X = affine.input_form(lo, hi, prop)
    n_old = 3                                  # rows of X that existed before the last activation
    H = len(L) - 1
    for l, (W, b) in enumerate(L):
        if 0 < l < H:
            Wr = _mul(rng, W, UB)                 # W_j in bfloat16 (symbol-row GEMM)
            W2 = _mul(rng, W, U2)                 # W_j as two bfloat16 terms (centre, input rows)
            c = _mul(rng, c, U2) @ W2.T + b
            XI = _mul(rng, X[:, :3], U2) @ W2.T
            XG = _mul(rng, _mul(rng, X[:, 3:n_old], UB) @ Wr.T, UB)
            XN = _mul(rng, X[:, n_old:] @ W.T, UB)
            X = np.concatenate([XI, XG, XN], axis=1)
        else:
            c = c @ W.T + b
            X = X @ W.T
        if l == H:
            break
        if prop == affine.CLT:
            sigma = np.sqrt(np.sum(X * X, axis=1))
            if act == "relu":
                alpha, beta, gamma = affine.relu_least_squares(c, sigma)
            else:
                alpha, beta, gamma = activations.least_squares(act, c, sigma)
        else:
            r = np.sum(np.abs(X), axis=1)
            alpha, beta, gamma = affine.relu_chebyshev(c - r, c + r)
        c = alpha * c + beta
        X = X * alpha[:, None, :]
        n_old = X.shape[1]
        Bn, w = gamma.shape
        G = np.zeros((Bn, w, w))
        G[:, np.arange(w), np.arange(w)] = gamma
        X = np.concatenate([X, G], axis=1)
    return c[:, 0], X[:, :, 0]


def _readout(x0, coef, mode):
    if mode == affine.SOUND:
        return x0, np.sum(np.abs(coef), axis=1)
    if mode == affine.CLT:
        return x0, np.sqrt(np.sum(coef * coef, axis=1))
    return x0, np.sqrt(np.sum(coef * coef, axis=1) / 3.0)


def bound_bands(layers, lo, hi, mode, k=3.0, batch=32, seed=0, act="relu", draws=K_DRAWS):
    """Exact oracle bounds and their per-result bands.  Returns a dict of float64 arrays (n,):
    centre, spread (the oracle's), band_c, band_s (bands of centre and spread) and band_lo, band_hi
    (bands of the read-off endpoints centre -+ spread, or centre -+ k spread)."""
    lo = np.asarray(lo).reshape(-1, 3)
    hi = np.asarray(hi).reshape(-1, 3)
    n = lo.shape[0]
    centre, spread = affine.bound(layers, lo, hi, mode, batch=batch, act=act)
    kk = 1.0 if mode == affine.SOUND else k
    acc = {key: np.zeros(n) for key in ("c", "s", "lo", "hi")}
    rng = np.random.default_rng(seed)
    for _ in range(draws):
        for s0 in range(0, n, batch):
            sl = slice(s0, s0 + batch)
            x0, coef = noisy_propagate(layers, lo[sl], hi[sl], mode, rng, act=act)
            cc, ss = _readout(x0, coef, mode)
            acc["c"][sl] += (cc - centre[sl]) ** 2
            acc["s"][sl] += (ss - spread[sl]) ** 2
            acc["lo"][sl] += ((cc - kk * ss) - (centre[sl] - kk * spread[sl])) ** 2
            acc["hi"][sl] += ((cc + kk * ss) - (centre[sl] + kk * spread[sl])) ** 2
    floor = 64 * U32 * (np.abs(centre) + kk * spread) + 1e-7
    out = dict(centre=centre, spread=spread)
    for key in ("c", "s", "lo", "hi"):
        out["band_" + key] = B_FACTOR * np.sqrt(acc[key] / draws) + floor
    return out


def near_iso_bits(levels, isos, layers, mode, k, coarse, batch=32, seed=0, act="relu", draws=K_DRAWS):
    """Per level of an oracle extraction (octree.extract_active's list), an int64 array over its
    bounded cells with bit q set when a read-off endpoint lies within its own band of iso-value q
    (the pairs whose cull decision rounding may flip).  `coarse` (relative) pre-selects the cells
    with an endpoint within coarse (|x0| + k spread) of an iso-value; only they get model draws.
    Returns (per-level bit arrays, number of cells given draws)."""
    from oracle import octree
    isos = np.asarray(isos, dtype=np.float64)
    kk = 1.0 if mode == affine.SOUND else k
    out, n_drawn = [], 0
    for lv in levels:
        n = lv["ijk"].shape[0]
        bits = np.zeros(n, dtype=np.int64)
        if n:
            scale = (np.abs(lv["centre"]) + kk * lv["spread"])[:, None]
            d_lo = np.abs(lv["lower"][:, None] - isos[None, :])
            d_hi = np.abs(lv["upper"][:, None] - isos[None, :])
            cand = np.flatnonzero(np.any((d_lo <= coarse * scale) | (d_hi <= coarse * scale), axis=1))
            if cand.size:
                blo, bhi = octree.cell_box(lv["ijk"][cand], lv["level"])
                b = bound_bands(layers, blo, bhi, mode, k=k, batch=batch, seed=seed + lv["level"], act=act,
                                draws=draws)
                near = (d_lo[cand] <= b["band_lo"][:, None]) | (d_hi[cand] <= b["band_hi"][:, None])
                bits[cand] = (near.astype(np.int64) << np.arange(isos.shape[0])[None, :]).sum(axis=1)
                n_drawn += cand.size
        out.append(bits)
    return out, n_drawn
