"""MLP evaluation in float64 (the INR f_theta of Sec. III-B): ReLU (App. E), ELU or sine activations
(oracle/activations.py).

Test infrastructure: see the package docstring.  Parity pinned by tests/test_oracle_pins.py
(linear networks against closed forms, brute-force containment).
"""
from __future__ import annotations

import numpy as np


def as_f64_layers(layers):
    """Widen float32 ``(W, b)`` pairs to float64 exactly."""
    return [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in layers]


def mlp_forward(layers, x, chunk=1 << 16, act="relu"):
    """f(x) = W_H act(... act(W_0 x + b_0) ...) + b_H for points ``x`` of shape (n, 3)."""
    from .activations import forward
    L = as_f64_layers(layers)
    x = np.asarray(x, dtype=np.float64).reshape(-1, L[0][0].shape[1])
    out = np.empty(x.shape[0])
    for s in range(0, x.shape[0], chunk):
        a = x[s:s + chunk]
        for l, (W, b) in enumerate(L):
            a = a @ W.T + b
            if l < len(L) - 1:
                a = np.maximum(a, 0.0) if act == "relu" else forward(act, a)
        out[s:s + chunk] = a[:, 0]
    return out
