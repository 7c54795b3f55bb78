"""Activations of the INR and their least-squares linear fits under a Gaussian input, in float64.

Test infrastructure: see the package docstring.

The MLP applies one activation f after every layer but the last: ReLU (App. E), ELU (App. A /
App. E: x for x > 0, e^x - 1 otherwise) or sine (the SIREN INRs of the main text, Sec. V-A.2; a
SIREN's frequency factor omega_0 is folded into the weights and biases, so f(z) = sin z).

Uncertainty propagation (Sec. IV-B/C, Eq. 9-10) replaces f on a neuron whose pre-activation is
X ~ N(mu, sigma^2) by the line alpha X + beta that minimises E[(f(X) - alpha X - beta)^2], and adds
one new symbol whose coefficient gamma is the residual's standard deviation.  The plain definition
of that fit, written out here from Gaussian moments of f:
    alpha   = Cov(f(X), X) / sigma^2,   beta = E f(X) - alpha mu,
    gamma^2 = Var f(X) - alpha^2 sigma^2.
Table VII prints the closed forms of these for ReLU, ELU and sine; the pins compare this module
with the printed forms and with quadrature.  The moments used (t = mu / sigma, Phi = P(X > 0) =
Phi(t), phi = the standard normal density at t):
    E[X; X > 0] = mu Phi + sigma phi,   E[X^2; X > 0] = (mu^2 + sigma^2) Phi + mu sigma phi,
    E[e^{sX}; X <= 0] = exp(s mu + s^2 sigma^2 / 2) Phi(-(mu + s sigma^2) / sigma),
    E[X e^X; X <= 0] = (mu + sigma^2) E[e^X; X <= 0] - sigma phi,
    E sin X = e^{-sigma^2/2} sin mu,  E[X sin X] = mu E sin X + sigma^2 e^{-sigma^2/2} cos mu,
    E sin^2 X = (1 - e^{-2 sigma^2} cos 2 mu) / 2.
sigma = 0: the tangent at mu (alpha = f'(mu), with f'(0) = 1/2 for ReLU as in the ReLU rule),
beta = f(mu) - alpha mu, gamma = 0.  gamma^2 is clamped at 0.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc, ndtr

RELU, ELU, SINE = "relu", "elu", "sine"
ACTS = (RELU, ELU, SINE)


def forward(act, z):
    """f(z) elementwise."""
    z = np.asarray(z, dtype=np.float64)
    if act == RELU:
        return np.maximum(z, 0.0)
    if act == ELU:
        return np.where(z > 0, z, np.expm1(np.minimum(z, 0.0)))
    if act == SINE:
        return np.sin(z)
    raise ValueError(act)


def _moments(act, mu, sigma):
    """E f(X), E[X f(X)], E f(X)^2 for X ~ N(mu, sigma^2), sigma > 0."""
    t = mu / sigma
    Phi = ndtr(t)
    Q = ndtr(-t)
    phi = np.exp(-0.5 * t * t) / np.sqrt(2.0 * np.pi)
    ex_pos = mu * Phi + sigma * phi                       # E[X; X > 0]
    ex2_pos = (mu * mu + sigma * sigma) * Phi + mu * sigma * phi
    if act == RELU:
        return ex_pos, ex2_pos, ex2_pos
    if act == ELU:
        s2 = sigma * sigma

        def e_exp_neg(s):                                 # E[e^{sX}; X <= 0]
            return 0.5 * erfc((mu + s * s2) / (np.sqrt(2.0) * sigma)) * np.exp(s * mu + 0.5 * s * s * s2)

        b1, b2 = e_exp_neg(1.0), e_exp_neg(2.0)
        xb1 = (mu + s2) * b1 - sigma * phi                # E[X e^X; X <= 0]
        ex_neg = mu * Q - sigma * phi                     # E[X; X <= 0]
        ef = ex_pos + b1 - Q
        exf = ex2_pos + xb1 - ex_neg
        ef2 = ex2_pos + b2 - 2.0 * b1 + Q
        return ef, exf, ef2
    if act == SINE:
        a = np.exp(-0.5 * sigma * sigma)
        ef = a * np.sin(mu)
        exf = mu * ef + sigma * sigma * a * np.cos(mu)
        ef2 = 0.5 * (1.0 - np.exp(-2.0 * sigma * sigma) * np.cos(2.0 * mu))
        return ef, exf, ef2
    raise ValueError(act)


def _tangent(act, mu):
    if act == RELU:
        alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 0.5, 0.0))
    elif act == ELU:
        alpha = np.where(mu > 0, 1.0, np.exp(np.minimum(mu, 0.0)))
    else:
        alpha = np.cos(mu)
    return alpha, forward(act, mu) - alpha * mu


def least_squares(act, mu, sigma):
    """alpha, beta, gamma of the least-squares line of f under N(mu, sigma^2) (Eq. 10, Table VII)."""
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    mu, sigma = np.broadcast_arrays(mu, sigma)
    alpha, beta = _tangent(act, mu)
    alpha = np.array(alpha, dtype=np.float64)
    beta = np.array(beta, dtype=np.float64)
    gamma2 = np.zeros(mu.shape)
    s = sigma > 0
    if np.any(s):
        m, sg = mu[s], sigma[s]
        ef, exf, ef2 = _moments(act, m, sg)
        a = (exf - m * ef) / (sg * sg)
        alpha[s] = a
        beta[s] = ef - a * m
        gamma2[s] = ef2 - ef * ef - a * a * sg * sg
    return alpha, beta, np.sqrt(np.maximum(gamma2, 0.0))
