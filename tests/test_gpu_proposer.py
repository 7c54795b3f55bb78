"""GPU parity of the proposer's hand-written BF16 kernels against the float64 oracle
(oracle/proposer.py), and the gating plumbing of the extraction.

Tolerances from the arithmetic: the GPU rounds the standardised inputs, the weights and every
hidden activation to bfloat16 (unit roundoff u_b = 2^-8) and accumulates in float32, so each of the
4 layers adds a relative error below 3 u_b of the layer's absolute-value propagation
|W| |a| + |b|; the logits must agree within 16 u_b of the absolute forward pass.  Gradients follow
the scope table's bar for BF16: cosine >= 0.999 and relative L2 <= 2e-2 against the FP64 gradient.
"""
import numpy as np
import pytest
import torch

from oracle import proposer as P
from synth import boxes, inr

pytestmark = pytest.mark.gpu
UB = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _packed(layers):
    from paper_2402_13861_gb300 import proposer as gp
    return gp.pack(layers)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 8)) * np.array([0.5, 0.5, 0.5, 2.0, 0.3, 0.4, 0.2, 0.8]) + \
        np.array([0, 0, 0, -6, 0.5, 0.0, 0.1, 1.5])
    y = (rng.uniform(size=n) < 0.35).astype(np.float64)
    return X, y


def _abs_forward(layers, Xn):
    a = np.abs(Xn)
    for l, (W, b) in enumerate(layers):
        a = a @ np.abs(W).T + np.abs(b)
    return a[:, 0]


def _oracle_layers(seed):
    layers = P.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    return [(W, rng.normal(0, 0.1, size=b.shape)) for W, b in layers]


def test_predict_matches_oracle(pkg):
    layers = _oracle_layers(1)
    X, _ = _batch(1000, 2)                       # > 7 tiles of 128 samples, ragged tail
    mu, sd = X.mean(0), X.std(0)
    prop = pkg.Proposer(_packed(layers), mu, sd)
    z = prop.predict(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
    zo, _ = P.forward(layers, X, mu, sd)
    tol = 16 * UB * _abs_forward(layers, (X - mu) / sd) + 1e-6
    print(f"max |dz| / tol = {(np.abs(z - zo) / tol).max():.3f}")
    assert np.all(np.abs(z - zo) <= tol)
    prop.close()


@pytest.mark.parametrize("n", [1, 128, 777])
def test_gradient_matches_oracle(pkg, n):
    layers = _oracle_layers(3)
    X, y = _batch(max(n, 2), 4)
    X, y = X[:n], y[:n]
    mu, sd = np.zeros(8), np.ones(8)
    prop = pkg.Proposer(_packed(layers), mu, sd)
    g, loss = prop.grad(torch.tensor(X, dtype=torch.float32, device="cuda"),
                        torch.tensor(y, dtype=torch.float32, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    zo, cache = P.forward(layers, X, mu, sd)
    go = np.concatenate([np.concatenate([gW.reshape(-1), gb.reshape(-1)]) for gW, gb in P.backward(layers, cache, y)])
    cos = g @ go / (np.linalg.norm(g) * np.linalg.norm(go))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"n={n}: cosine {cos:.6f}, relative L2 {rel:.3e}, loss {float(loss):.5f} vs {P.bce(zo, y):.5f}")
    assert cos >= 0.999 and rel <= 2e-2
    # the loss moves by |dL/dz| = |sigmoid(z) - y| per unit of logit error (first order)
    dz = 16 * UB * _abs_forward(layers, X)
    assert abs(float(loss) - P.bce(zo, y)) <= 1.5 * np.mean(np.abs(P.sigmoid(zo) - y) * dz) + 1e-6
    prop.close()


def test_adam_first_step_matches_closed_form(pkg):
    layers = _oracle_layers(5)
    X, y = _batch(512, 6)
    mu, sd = np.zeros(8), np.ones(8)
    p0 = _packed(layers)
    prop = pkg.Proposer(p0, mu, sd)
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    g, _ = prop.grad(Xt, yt)
    g = g.cpu().numpy()
    lr = 1e-3
    prop.train_step(Xt, yt, lr)
    p1 = prop.get_params()
    big = np.abs(g) > 1e-5 * np.abs(g).max()
    # first Adam step: -lr g / (|g| + eps) = -lr sign(g) wherever |g| >> eps
    step = p1 - p0
    assert np.allclose(step[big], -lr * np.sign(g[big]), rtol=2e-3, atol=1e-8)
    prop.close()


def test_training_reduces_loss_and_separates(pkg):
    rng = np.random.default_rng(7)
    X = rng.normal(size=(16384, 8))
    y = ((X @ np.arange(1, 9)) + 0.5 * X[:, 0] * X[:, 1] > 0).astype(np.float64)
    from paper_2402_13861_gb300 import proposer as gp
    prop = pkg.Proposer(gp.he_params(0), np.zeros(8), np.ones(8))
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, device="cuda")
    first = None
    for step in range(300):
        sel = torch.randint(0, X.shape[0], (2048,), device="cuda")
        prop.train_step(Xt[sel].contiguous(), yt[sel].contiguous(), 3e-3, loss=loss)
        if first is None:
            first = float(loss)
    z = prop.predict(Xt).cpu().numpy()
    acc = np.mean((z > 0) == (y > 0))
    print(f"loss {first:.4f} -> {float(loss):.4f}, accuracy {acc:.4f}")
    assert float(loss) < 0.25 * first and acc > 0.97
    prop.close()


def _constant_proposer(pkg, logit):
    params = np.zeros(8961, dtype=np.float32)
    params[-1] = logit                                   # b4: every pair gets this logit
    return pkg.Proposer(params, np.zeros(8), np.ones(8))


def test_gate_all_unsure_equals_plain_extraction(pkg):
    """tau_lo = 0, tau_hi = 1: every pair is undecided, every cell is bounded: plain extraction."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 31)
    net = pkg.Inr(layers)
    isos = np.array([-0.05, 0.02], dtype=np.float32)
    prop = _constant_proposer(pkg, 0.0)
    a = net.extract(6, isos, mode="clt", k=3.0, prec="bf16")
    b = net.extract(6, isos, mode="clt", k=3.0, prec="bf16", proposer=prop, proposer_level=2, tau_lo=0.0,
                    tau_hi=1.0)
    assert a["n_active"] == b["n_active"] and a["n_tris"] == b["n_tris"]
    assert a["cells_bounded"] == b["cells_bounded"] and b["cells_visited"] == a["cells_bounded"]
    assert torch.equal(a["codes"], b["codes"]) and torch.equal(a["masks"], b["masks"])
    net.close()
    prop.close()


def test_gate_all_keep_and_all_drop(pkg):
    layers = inr.random_inr([3, 128, 128, 128, 1], 32)
    net = pkg.Inr(layers)
    isos = np.array([0.0], dtype=np.float32)
    L, pl = 5, 3
    plain = net.extract(L, isos, mode="clt", k=3.0, prec="bf16")
    keep = _constant_proposer(pkg, 40.0)
    r = net.extract(L, isos, mode="clt", k=3.0, prec="bf16", proposer=keep, proposer_level=pl, tau_lo=0.1,
                    tau_hi=0.9)
    # levels >= pl are never bounded; every cell reaching pl keeps all its descendants
    assert all(r["cells_bounded"][l] == 0 for l in range(pl, L + 1))
    assert r["cells_bounded"][:pl] == plain["cells_bounded"][:pl]
    assert r["n_active"] == r["cells_visited"][pl] * 8 ** (L - pl)
    # the plain active set is contained in the kept set
    kept = set((r["codes"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF).tolist())
    assert set((plain["codes"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF).tolist()) <= kept
    drop = _constant_proposer(pkg, -40.0)
    r = net.extract(L, isos, mode="clt", k=3.0, prec="bf16", proposer=drop, proposer_level=pl, tau_lo=0.1,
                    tau_hi=0.9)
    assert r["n_active"] == 0 and r["n_tris"] == 0
    net.close()
    keep.close()
    drop.close()


def test_bad_thresholds_are_rejected(pkg):
    net = pkg.Inr(inr.random_inr([3, 128, 128, 1], 1))
    prop = _constant_proposer(pkg, 0.0)
    with pytest.raises(pkg.IsxError) as e:
        net.extract(3, [0.0], mode="clt", proposer=prop, tau_lo=0.6, tau_hi=0.4)
    assert e.value.status == 1
    net.close()
    prop.close()


def test_trained_proposer_on_held_out_field(pkg):
    """The committed proposer (trained on fields seeded 2000-2011) on the committed scientific INR
    (field seed 2, held out) at 128^3: fewer cells bounded than plain extraction, and no more
    crossing (cell, iso) pairs of the dense extraction missed than plain extraction misses plus 1 %."""
    import os
    from paper_2402_13861_gb300 import proposer as gp
    from paper_2402_13861_gb300.train_proposer import missed
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    layers, isos, _ = inr.load_inr("scientific")
    net = pkg.Inr(layers)
    prop, meta = gp.load(os.path.join(root, "synth", "data", "proposer.npz"))
    L = 7
    kw = dict(mode="clt", k=3.0, prec="bf16", active_cap=1 << 22, tri_cap=1 << 23)
    plain = net.extract(L, isos, **kw)
    assisted = net.extract(L, isos, proposer=prop, proposer_level=meta["proposer_level"], tau_lo=meta["tau_lo"],
                           tau_hi=meta["tau_hi"], **kw)
    cross = gp.crossing_cells(net, L, isos)
    mp, tot = missed(plain["codes"], plain["masks"], cross)
    ma, _ = missed(assisted["codes"], assisted["masks"], cross)
    bp, ba = sum(plain["cells_bounded"]), sum(assisted["cells_bounded"])
    print(f"bounded {bp} -> {ba}; missed pairs plain {mp}, proposer {ma} of {tot}")
    assert ba < bp and ma <= mp + 0.01 * tot
    net.close()
    prop.close()
