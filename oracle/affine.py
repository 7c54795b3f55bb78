"""Affine forms, probabilistic affine forms and their propagation through a ReLU MLP, in float64.

Test infrastructure: see the package docstring.

An affine form over a box is kept as a centre ``x0`` and a coefficient matrix whose row ``i`` holds
the coefficients of noise symbol ``i`` for every neuron (Eq. 1 for intervals eps_i in [-1, 1],
Eq. 6 for unit random variables Z_i).  The propagation is the literal layer loop of Sec. III-B and
Sec. IV-C:

* input box (centre x_c, half-width h) -> x_c + diag(h) eps (Sec. III-B), or x_c + diag(h/sqrt 3) Z
  for the probabilistic form, since a uniform variable on [-h, h] has standard deviation
  h / sqrt 3 (Sec. IV-C; Algorithm 1, node set-up);
* linear layer: Eq. 3 (= Eq. 8), exact: centre W c + b, coefficients X W^T;
* ReLU: fit alpha x + beta, then centre alpha c + beta, coefficients scaled by alpha, and one new
  symbol per neuron with coefficient gamma (Eq. 4 = Eq. 9);
  - sound affine arithmetic: the Chebyshev (minimax) line on [c - r, c + r], r = sum_i |x_i|
    (Eq. 2, Eq. 4);
  - uncertainty propagation: the least-squares line under N(mu, sigma^2), mu = c,
    sigma^2 = sum_i x_i^2 (Eq. 7, Eq. 10), closed form of Table VII, gamma = residual std;
* read-off at the output: [x0 - r, x0 + r] (Eq. 2), or mu +- k sigma (Eq. 7, Algorithm 1), or the
  RA-UA variant: sound propagation with sigma^2 = (1/3) sum_i x_i^2 at the output only
  (Sec. IV-A).
* RA-Fixed (Sec. V-A.4 baselines; App. A): the reduced form that keeps only the three input
  symbols and condenses every other coefficient of a neuron into one non-negative radius of its
  own (``propagate_rafixed``).

Readings where the paper is silent (listed in the design notes):
* The Chebyshev ReLU line is not printed.  For l < 0 < u it is the chord through (l, 0) and
  (u, u) moved down by half its largest gap: alpha = u / (u - l), beta = gamma = -alpha l / 2;
  alpha = beta = gamma = 0 when u <= 0; alpha = 1, beta = gamma = 0 when l >= 0.
* sigma = 0 in the least-squares rule: alpha = 1 if mu > 0, 1/2 if mu = 0, 0 otherwise;
  beta = gamma = 0.  gamma^2 is clamped at 0.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import activations
from .mlp import as_f64_layers

SOUND, CLT, RAUA, RAFIXED = "sound", "clt", "raua", "rafixed"


def relu_chebyshev(l, u):
    """Minimax linear fit of ReLU on [l, u]: returns alpha, beta, gamma (Eq. 4, Chebyshev choice)."""
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    alpha = np.zeros(np.broadcast(l, u).shape)
    beta = np.zeros_like(alpha)
    gamma = np.zeros_like(alpha)
    pos = l >= 0
    alpha[pos] = 1.0
    cross = (l < 0) & (u > 0)
    a = u[cross] / (u[cross] - l[cross])
    alpha[cross] = a
    beta[cross] = -a * l[cross] / 2.0
    gamma[cross] = -a * l[cross] / 2.0
    return alpha, beta, gamma


def relu_least_squares(mu, sigma):
    """Least-squares fit of ReLU under N(mu, sigma^2) (Eq. 10; Table VII, ReLU row)."""
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 0.5, 0.0)).astype(np.float64)
    beta = np.zeros(alpha.shape)
    gamma2 = np.zeros(alpha.shape)
    s = sigma > 0
    m, sg = mu[s], sigma[s]
    a = erf(-m / (np.sqrt(2.0) * sg))
    alpha[s] = 0.5 * (1.0 - a)
    b = sg / np.sqrt(2.0 * np.pi) * np.exp(-m * m / (2.0 * sg * sg))
    beta[s] = b
    gamma2[s] = 0.25 * (1.0 - a * a) * (m * m + sg * sg) + a * m * b - b * b
    return alpha, beta, np.sqrt(np.maximum(gamma2, 0.0))


def input_form(lo, hi, mode):
    """Centre (B, 3) and coefficient matrices (B, 3, 3) of the input box (Sec. III-B / IV-C)."""
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 3)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 3)
    xc = (lo + hi) / 2.0
    h = (hi - lo) / 2.0
    if mode == CLT:
        h = h / np.sqrt(3.0)
    X = np.zeros((lo.shape[0], 3, 3))
    X[:, [0, 1, 2], [0, 1, 2]] = h
    return xc, X


def propagate(layers, lo, hi, mode, act="relu"):
    """Output centre (B,) and output coefficients (B, S) of every box, S = 3 + sum of hidden widths.
    ELU and sine layers (``act``) take the least-squares rule of uncertainty propagation only."""
    if act != "relu" and mode != CLT:
        raise NotImplementedError("sound affine arithmetic is implemented for ReLU layers only")
    L = as_f64_layers(layers)
    c, X = input_form(lo, hi, mode)
    for l, (W, b) in enumerate(L):
        c = c @ W.T + b                      # Eq. 3 / Eq. 8, centre
        X = X @ W.T                          # Eq. 3 / Eq. 8, every symbol's coefficient
        if l == len(L) - 1:
            break
        if mode == CLT:
            sigma = np.sqrt(np.sum(X * X, axis=1))      # Eq. 7
            if act == "relu":
                alpha, beta, gamma = relu_least_squares(c, sigma)
            else:
                alpha, beta, gamma = activations.least_squares(act, c, sigma)
        else:
            r = np.sum(np.abs(X), axis=1)                # Eq. 2
            alpha, beta, gamma = relu_chebyshev(c - r, c + r)
        c = alpha * c + beta                              # Eq. 4 / Eq. 9, centre
        X = X * alpha[:, None, :]                         # Eq. 4 / Eq. 9, old symbols
        B, w = gamma.shape
        G = np.zeros((B, w, w))
        G[:, np.arange(w), np.arange(w)] = gamma          # one new symbol per neuron
        X = np.concatenate([X, G], axis=1)
    return c[:, 0], X[:, :, 0]


def propagate_rafixed(layers, lo, hi):
    """RA-Fixed: sound affine arithmetic that keeps the input symbols eps_1..3 and folds all other
    symbols of a neuron into one radius r >= 0 that belongs to that neuron alone.

    A neuron is c + sum_d A_d eps_d + r eta with eta in [-1, 1] private to the neuron, so
      linear layer (Eq. 3 on the kept symbols; the private terms of the inputs combine as
      sum_k |W_nk| r_k, the largest |sum_k W_nk r_k eta_k| can be):
          c' = W c + b,  A' = A W^T,  r' = r |W|^T;
      ReLU (Eq. 4, Chebyshev line on [c - s, c + s], s = sum_d |A_d| + r):
          c' = alpha c + beta,  A' = alpha A,  r' = alpha r + gamma.
    Returns the output centre (B,) and spread sum_d |A_d| + r (B,): the bound [c - s, c + s]."""
    L = as_f64_layers(layers)
    c, A = input_form(lo, hi, SOUND)
    r = np.zeros(c.shape)
    for l, (W, b) in enumerate(L):
        c = c @ W.T + b
        A = A @ W.T
        r = r @ np.abs(W).T
        if l == len(L) - 1:
            break
        s = np.sum(np.abs(A), axis=1) + r
        alpha, beta, gamma = relu_chebyshev(c - s, c + s)
        c = alpha * c + beta
        A = A * alpha[:, None, :]
        r = alpha * r + gamma
    return c[:, 0], np.sum(np.abs(A[:, :, 0]), axis=1) + r[:, 0]


def bound(layers, lo, hi, mode, batch=64, act="relu"):
    """Centre and spread of every box: (x0, r) for SOUND and RAFIXED, (mu, sigma) for CLT and RAUA."""
    lo = np.asarray(lo).reshape(-1, 3)
    hi = np.asarray(hi).reshape(-1, 3)
    n = lo.shape[0]
    centre = np.empty(n)
    spread = np.empty(n)
    if mode == RAFIXED:
        for s in range(0, n, batch):
            centre[s:s + batch], spread[s:s + batch] = propagate_rafixed(layers, lo[s:s + batch], hi[s:s + batch])
        return centre, spread
    prop_mode = CLT if mode == CLT else SOUND
    for s in range(0, n, batch):
        x0, coef = propagate(layers, lo[s:s + batch], hi[s:s + batch], prop_mode, act=act)
        centre[s:s + batch] = x0
        if mode == SOUND:
            spread[s:s + batch] = np.sum(np.abs(coef), axis=1)             # Eq. 2
        elif mode == CLT:
            spread[s:s + batch] = np.sqrt(np.sum(coef * coef, axis=1))     # Eq. 7
        else:
            spread[s:s + batch] = np.sqrt(np.sum(coef * coef, axis=1) / 3.0)  # Sec. IV-A
    return centre, spread


def interval(centre, spread, mode, k):
    """[lower, upper] of the read-off: [x0 - r, x0 + r] or [mu - k sigma, mu + k sigma]."""
    if mode in (SOUND, RAFIXED):
        return centre - spread, centre + spread
    return centre - k * spread, centre + k * spread


def clt_covariance(layers, lo, hi):
    """CLT mean and sigma by propagating the w x w covariance of the probabilistic form instead of
    its coefficients: C' = W C W^T through linear layers and C' = diag(alpha) C diag(alpha) +
    diag(gamma^2) through ReLU.  Mathematically identical to ``bound(..., CLT)`` because the
    symbols are independent with unit variance (Eq. 6, Eq. 7); used only as a cross-check."""
    L = as_f64_layers(layers)
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 3)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 3)
    c = (lo + hi) / 2.0
    var_in = ((hi - lo) / 2.0) ** 2 / 3.0
    C = np.zeros((lo.shape[0], 3, 3))
    C[:, [0, 1, 2], [0, 1, 2]] = var_in
    for l, (W, b) in enumerate(L):
        c = c @ W.T + b
        C = np.einsum("ij,bjk,lk->bil", W, C, W)
        if l == len(L) - 1:
            break
        sigma = np.sqrt(np.maximum(np.einsum("bii->bi", C), 0.0))
        alpha, beta, gamma = relu_least_squares(c, sigma)
        c = alpha * c + beta
        C = alpha[:, :, None] * C * alpha[:, None, :]
        w = gamma.shape[1]
        C[:, np.arange(w), np.arange(w)] += gamma * gamma
    return c[:, 0], np.sqrt(C[:, 0, 0])
