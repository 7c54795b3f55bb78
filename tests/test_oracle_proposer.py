"""Pins of the proposer oracle (oracle/proposer.py) against the mathematics, independent of it:
central finite differences, the logistic-regression special case, the closed form of Adam's
first step, the textbook cross-entropy, and brute-force subtree labels."""
import numpy as np
import pytest

from oracle import proposer as P


def _batch(n=37, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 8))
    y = (rng.uniform(size=n) < 0.4).astype(np.float64)
    return X, y


def test_backward_matches_central_finite_differences():
    params = P.init_params(5, dims=(8, 16, 12, 10, 1))
    params = [(W, b + 0.05 * np.arange(b.size)) for W, b in params]      # non-zero biases
    X, y = _batch()
    z, cache = P.forward(params, X)
    grads = P.backward(params, cache, y)
    h = 1e-6
    worst = 0.0
    for l, (W, b) in enumerate(params):
        for k, arr in enumerate((W, b)):
            flat = arr.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 25)):
                old = flat[idx]
                flat[idx] = old + h
                lp = P.bce(P.forward(params, X)[0], y)
                flat[idx] = old - h
                lm = P.bce(P.forward(params, X)[0], y)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                g = grads[l][k].reshape(-1)[idx]
                worst = max(worst, abs(fd - g) / max(1e-8, abs(fd) + abs(g)))
    assert worst < 1e-5


def test_single_layer_reduces_to_logistic_regression():
    """With no hidden layer the model is logistic regression: dL/dw = X^T (sigmoid(Xw + b) - y) / n."""
    rng = np.random.default_rng(1)
    X, y = _batch(50, 2)
    w = rng.normal(size=8)
    b = 0.3
    z, cache = P.forward([(w[None, :], np.array([b]))], X)
    grads = P.backward([(w[None, :], np.array([b]))], cache, y)
    p = 1.0 / (1.0 + np.exp(-(X @ w + b)))
    assert np.allclose(grads[0][0][0], X.T @ (p - y) / 50, rtol=1e-12, atol=1e-14)
    assert np.isclose(grads[0][1][0], np.mean(p - y), rtol=1e-12)
    # cross-entropy in its textbook form
    assert np.isclose(P.bce(z, y), -np.mean(y * np.log(p) + (1 - y) * np.log(1 - p)), rtol=1e-12)


def test_bce_at_zero_logit_is_log2_and_stable_for_large_logits():
    assert np.isclose(P.bce(np.zeros(4), np.array([0, 1, 0, 1])), np.log(2.0))
    assert np.isfinite(P.bce(np.array([800.0, -800.0]), np.array([0.0, 1.0])))
    assert np.isclose(P.bce(np.array([800.0]), np.array([0.0])), 800.0)


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is -lr g / (|g| + eps)."""
    params = P.init_params(2, dims=(8, 4, 1))
    rng = np.random.default_rng(4)
    grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in params]
    st = P.adam_init(params)
    new = P.adam_step(params, grads, st, lr=1e-2, eps=1e-8)
    for (W, b), (gW, gb), (nW, nb) in zip(params, grads, new):
        assert np.allclose(nW - W, -1e-2 * gW / (np.abs(gW) + 1e-8), rtol=1e-12, atol=1e-15)
        assert np.allclose(nb - b, -1e-2 * gb / (np.abs(gb) + 1e-8), rtol=1e-12, atol=1e-15)


def test_adam_training_separates_a_linearly_separable_set():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(256, 8))
    y = (X @ np.arange(1, 9) > 0).astype(np.float64)
    params = P.init_params(9)
    st = P.adam_init(params)
    losses = []
    for _ in range(300):
        z, cache = P.forward(params, X)
        losses.append(P.bce(z, y))
        params = P.adam_step(params, P.backward(params, cache, y), st, lr=3e-3)
    z, _ = P.forward(params, X)
    assert losses[-1] < 0.1 * losses[0]
    assert np.mean((z > 0) == (y > 0)) > 0.97


def test_features_closed_forms():
    X = P.features(np.array([[0, 0, 0], [3, 1, 2]]), np.array([1, 2]), np.array([0.5, 0.2]),
                   np.array([0.7, 0.1]), np.array([0.3, 0.05]), np.array([1, 2]))
    assert np.allclose(X[0], [-0.5, -0.5, -0.5, -1.0, 0.5, 0.2, 0.3, 1.0])
    assert np.allclose(X[1], [0.75, -0.25, 0.25, -2.0, 0.2, -0.1, 0.05, 2.0])


def test_forward_standardises_the_features():
    """x_norm = (x - mu) / sd: a single linear unit reading feature 0 returns (x_0 - mu_0) / sd_0."""
    W = np.zeros((1, 8))
    W[0, 0] = 1.0
    params = [(W, np.zeros(1))]
    mu = np.full(8, 1.0)
    sd = np.full(8, 4.0)
    z, _ = P.forward(params, np.array([[3.0] + [0.0] * 7, [-7.0] + [0.0] * 7]), mu, sd)
    assert np.allclose(z, [0.5, -2.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_subtree_labels_match_brute_force(level):
    L = 4
    rng = np.random.default_rng(level)
    codes = rng.integers(0, 1 << L, size=(40, 3))
    masks = rng.integers(1, 8, size=40)
    cells = np.array([[i, j, k] for i in range(1 << level) for j in range(1 << level) for k in range(1 << level)])
    got = P.subtree_labels(codes, masks, L, cells, level)
    s = 1 << (L - level)
    for c, g in zip(cells, got):
        want = 0
        for code, m in zip(codes, masks):
            if all(c[d] * s <= code[d] < (c[d] + 1) * s for d in range(3)):
                want |= int(m)
        assert g == want


def test_he_initialisation_scales_with_fan_in():
    """He-normal initialisation: weights of a layer with fan-in n have standard deviation
    sqrt(2 / n) and the biases start at 0.  The sample deviation of each layer of the proposer's
    shape (8 -> 64 -> 64 -> 64 -> 1) is checked against it (chi-square width: 4 / sqrt(2 N))."""
    params = P.init_params(123)
    assert [W.shape for W, _ in params] == [(64, 8), (64, 64), (64, 64), (1, 64)]
    for W, b in params:
        want = np.sqrt(2.0 / W.shape[1])
        sd = np.sqrt(np.mean(W * W))
        assert abs(sd / want - 1.0) < 4.0 / np.sqrt(2.0 * W.size)
        assert np.all(b == 0.0)
    a = P.init_params(123)
    assert all(np.array_equal(W, W2) for (W, _), (W2, _) in zip(params, a))
