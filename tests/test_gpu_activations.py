"""GPU parity of ELU and sine (SIREN) networks against the float64 oracle: evaluation on the CUDA
and tensor cores, uncertainty-propagation bounds with the ELU / sine rows of Table VII on the
float32 and tensor-core paths, and hierarchical extraction.

Tolerances from the arithmetic.  Evaluation: a K-term float32 dot product errs by at most
~K u |terms| (u = 2^-24) and both activations are 1-Lipschitz, so the output stays within
8 H w u of the absolute-value propagation |W| |a| + |b| (the two-term BF16 tensor-core products:
2^-12 of it, as for ReLU).  Bounds: the same rounding enters the centre and sigma of every neuron,
and the test holds both paths to the ReLU allowances: 8 H w u (|x0| + sigma) for float32 and
3 H u_b (|x0| + sigma) for the bfloat16 coefficients of the tensor-core path (u_b = 2^-8).  The
sine row can amplify a centre error by up to 1 + |mu| (d beta / d mu = a mu sin mu), a factor the
allowance leaves out; the printed ratios show how far inside it the measured errors stay even so.
"""
import numpy as np
import pytest
import torch

from oracle import affine, mlp, octree
from synth import boxes, inr

from _helpers import to_np

pytestmark = pytest.mark.gpu
U, UB = 2.0 ** -24, 2.0 ** -8
NETS = [("sine", [3, 64, 64, 1]), ("sine", [3, 128, 128, 128, 1]), ("sine", [3] + [256] * 3 + [1]),
        ("elu", [3, 48, 48, 1]), ("elu", [3, 128, 128, 128, 1]), ("elu", [3] + [256] * 4 + [1])]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _abs_prop(layers, x, act):
    from oracle import activations
    a = np.asarray(x, dtype=np.float64)
    m = np.abs(a)
    for l, (W, b) in enumerate(layers):
        W = np.asarray(W, np.float64)
        b = np.asarray(b, np.float64)
        m = m @ np.abs(W).T + np.abs(b)
        a = a @ W.T + b
        if l < len(layers) - 1:
            a = activations.forward(act, a)
            m = np.maximum(m, 0) if act == "elu" else np.minimum(m, 1.0)
    return m[:, 0]


def _max_mu(layers, lo, hi, act):
    """Largest |pre-activation| met by the boxes' centre points: the size of the centres mu the
    linearisation sees, the conditioning factor of the bound."""
    from oracle import activations
    a = (np.asarray(lo, np.float64) + np.asarray(hi, np.float64)) / 2
    worst = 0.0
    for W, b in layers[:-1]:
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        worst = max(worst, float(np.abs(z).max()))
        a = activations.forward(act, z)
    return worst


def _net(act, dims, seed=31):
    layers = inr.random_inr(dims, seed, act=act)
    if act == "elu":
        rng = np.random.default_rng(seed)
        layers = [(W, rng.normal(0, 0.1, size=b.shape).astype(np.float32)) for W, b in layers]
    return layers


@pytest.mark.parametrize("act,dims", NETS, ids=lambda v: v if isinstance(v, str) else "x".join(map(str, v[1:-1])))
def test_eval_matches_oracle(pkg, act, dims):
    layers = _net(act, dims)
    net = pkg.Inr(layers, act=act)
    x = np.random.default_rng(4).uniform(-1, 1, size=(1000, 3)).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    vo = mlp.mlp_forward(layers, x, act=act)
    scale = _abs_prop(layers, x, act)
    H, w = len(dims) - 2, dims[1]
    v32 = to_np(net.eval_points(xt, prec="fp32")).astype(np.float64)
    r32 = np.abs(v32 - vo) / scale
    msg = f"{act} {dims[1:-1]}: fp32 max err / |W||a| {r32.max():.2e}"
    assert np.all(r32 <= 8 * H * w * U)
    if w in (128, 256):
        vtc = to_np(net.eval_points(xt, prec="bf16")).astype(np.float64)
        rtc = np.abs(vtc - vo) / scale
        msg += f", tensor cores {rtc.max():.2e}"
        assert np.all(rtc <= 2.0 ** -12)
    print(msg)
    net.close()


@pytest.mark.parametrize("act,dims", NETS, ids=lambda v: v if isinstance(v, str) else "x".join(map(str, v[1:-1])))
def test_clt_bounds_match_oracle(pkg, act, dims):
    layers = _net(act, dims)
    net = pkg.Inr(layers, act=act)
    lo, hi = boxes.random_boxes(613, 17, -9, -1)
    H, w = len(dims) - 2, dims[1]
    m = 97 if w >= 256 else 613
    oc, os_ = affine.bound(layers, lo[:m], hi[:m], affine.CLT, batch=64, act=act)
    cond = 1.0 + _max_mu(layers, lo[:m], hi[:m], act)
    for prec in ("fp32", "bf16"):
        if prec == "bf16" and w not in (128, 256):
            continue
        c, s = net.bound_cells(torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), mode="clt",
                               prec=prec)
        c, s = to_np(c).astype(np.float64)[:m], to_np(s).astype(np.float64)[:m]
        tol = (8 * H * w * U if prec == "fp32" else 3 * H * UB) * (np.abs(oc) + os_) + 1e-7
        rc, rs = np.max(np.abs(c - oc) / tol), np.max(np.abs(s - os_) / tol)
        print(f"{act} {dims[1:-1]} {prec}: max |dc| / tol {rc:.4f}, max |ds| / tol {rs:.4f} "
              f"(1 + max |mu| = {cond:.1f})")
        assert rc <= 1 and rs <= 1
    net.close()


def test_sound_modes_reject_elu_and_sine(pkg):
    for act in ("elu", "sine"):
        net = pkg.Inr(_net(act, [3, 128, 128, 1]), act=act)
        box = torch.zeros((4, 3), device="cuda"), torch.ones((4, 3), device="cuda") * 0.1
        for mode in ("sound", "raua", "rafixed"):
            with pytest.raises(pkg.IsxError) as e:
                net.bound_cells(*box, mode=mode)
            assert e.value.status == 5
        with pytest.raises(pkg.IsxError) as e:
            net.extract(3, [0.0], mode="sound")
        assert e.value.status == 5
        net.close()


@pytest.mark.parametrize("act", ["sine", "elu"])
def test_clt_extraction_matches_oracle(pkg, act):
    """Hierarchical CLT extraction of an ELU / SIREN network: active sets equal the oracle's up to
    cells near an iso-value, triangles of clean common cells identical."""
    from test_gpu_extract import _check_extraction
    dims = [3, 64, 64, 1]
    layers = _net(act, dims, seed=8)
    if act == "sine":                                   # a smoother SIREN: omega0 = 30 only in layer 0
        layers = [layers[0]] + [(W / 6.0, b / 6.0) for W, b in layers[1:-1]] + [layers[-1]]
    net = pkg.Inr(layers, act=act)
    L = 5
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L), act=act)
    isos = np.quantile(vals, [0.35, 0.65]).astype(np.float32)
    res = net.extract(L, isos, mode="clt", k=3.0, prec="fp32")
    _check_extraction(layers, isos, L, vals, res, affine.CLT, 3.0, act=act)
    d = net.extract(L, isos, prec="fp32", dense=True)
    print(f"{act}: active {res['n_active']}, triangles {res['n_tris']} (dense {d['n_tris']})")
    assert res["n_tris"] > 0.9 * d["n_tris"]
    net.close()
