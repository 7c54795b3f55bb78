"""GPU parity of the tensor-core MLP evaluation (two-term BF16 operands, tcgen05) against the float64
oracle, and of extractions that use it for their corner values.

Tolerance from the arithmetic: every operand x is carried as x_hi + x_lo (two BF16 terms, within
2^-17 |x| of x) and products as a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is below
2^-18 |a b|), accumulated in FP32; per layer the error stays below a few 2^-16 of the layer's
absolute-value propagation |W| |a| + |b|.  The test allows 2^-12 of that propagation at the output
(16x tighter than single-term BF16 products could meet) and prints the measured ratio.
"""
import numpy as np
import pytest
import torch

from oracle import mlp, octree
from synth import inr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _abs_prop(layers, x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    for l, (W, b) in enumerate(layers):
        a = a @ np.abs(np.asarray(W, np.float64)).T + np.abs(np.asarray(b, np.float64))
    return a[:, 0]


@pytest.mark.parametrize("dims", [[3, 128, 128, 1], [3, 128, 128, 128, 128, 1], [3] + [256] * 5 + [1], "scientific"])
def test_tc_eval_matches_oracle(pkg, dims):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 9)
    if not isinstance(dims, str):
        rng = np.random.default_rng(3)
        layers = [(W, rng.normal(0, 0.05, size=b.shape).astype(np.float32)) for W, b in layers]
    net = pkg.Inr(layers)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, size=(1000, 3)).astype(np.float32)        # 7 full tiles and a ragged one
    xt = torch.tensor(x, device="cuda")
    v = net.eval_points(xt, prec="bf16").cpu().numpy().astype(np.float64)
    v32 = net.eval_points(xt, prec="fp32").cpu().numpy().astype(np.float64)
    vo = mlp.mlp_forward(layers, x.astype(np.float64))
    scale = _abs_prop(layers, x)
    r = np.abs(v - vo) / scale
    r32 = np.abs(v32 - vo) / scale
    print(f"{dims if isinstance(dims, str) else dims[1:-1]}: max err / |W||a| tensor cores {r.max():.2e}, "
          f"fp32 cores {r32.max():.2e}")
    assert np.all(np.isfinite(v)) and np.all(r <= 2.0 ** -12)
    net.close()


def test_tc_eval_lattice_and_unsupported_width(pkg):
    layers = inr.random_inr([3, 64, 64, 1], 2)
    net = pkg.Inr(layers)
    with pytest.raises(pkg.IsxError) as e:
        net.eval_points(torch.zeros((4, 3), device="cuda"), prec="bf16")
    assert e.value.status == 5
    net.close()


@pytest.mark.parametrize("dense", [False, True])
def test_extraction_with_tc_corner_values(pkg, dense):
    """Corner values from the tensor cores give the FP32-evaluated mesh except in cells with a corner
    value within the evaluation band of an iso-value; shared vertices agree to 1e-4."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 31)
    net = pkg.Inr(layers)
    L = 5
    R = 1 << L
    pts = octree.lattice_points(R)
    vals = mlp.mlp_forward(layers, pts)
    isos = np.quantile(vals, [0.3, 0.6]).astype(np.float32)
    kw = dict(mode="clt", k=3.0, prec="bf16", dense=dense)
    a = net.extract(L, isos, eval_prec="fp32", **kw)
    b = net.extract(L, isos, eval_prec="bf16", **kw)
    band = 2.0 ** -12 * _abs_prop(layers, pts).reshape(R + 1, R + 1, R + 1)
    v3 = vals.reshape(R + 1, R + 1, R + 1)                  # [k][j][i]

    def tris(res):
        e = res["tri_edge"].cpu().numpy()
        c = res["tri_cell"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        q = res["tri_iso"].cpu().numpy()
        return {(int(cc), int(qq), tuple(sorted(ee.tolist()))): i for i, (cc, qq, ee) in enumerate(zip(c, q, e))}

    ta, tb = tris(a), tris(b)
    for key in set(ta) ^ set(tb):
        code, q = key[0], key[1]
        i, j, k = code & 1023, (code >> 10) & 1023, (code >> 20) & 1023
        corner = v3[k:k + 2, j:j + 2, i:i + 2]
        assert np.any(np.abs(corner - isos[q]) <= band[k:k + 2, j:j + 2, i:i + 2] + 1e-6), key
    va, vb = a["tri_vert"].cpu().numpy(), b["tri_vert"].cpu().numpy()
    ea = a["tri_edge"].cpu().numpy()
    common = set(ta) & set(tb)
    assert len(common) > 0.99 * max(len(ta), 1)
    # a vertex moves along its edge by h |dt| with |dt| <= (|dv_a| + |dv_b|) / |v_b - v_a| (first order):
    # the allowance comes from the two evaluations' measured difference at the edge's end points
    xyz = torch.tensor(pts, dtype=torch.float32, device="cuda")
    v32 = net.eval_points(xyz, prec="fp32").cpu().numpy().astype(np.float64)
    vtc = net.eval_points(xyz, prec="bf16").cpu().numpy().astype(np.float64)
    dv = np.abs(vtc - v32)
    n1, h = R + 1, 2.0 / R
    step = np.array([1, n1, n1 * n1])
    worst = 0.0
    for key in common:
        ia, ib = ta[key], tb[key]
        for e3 in range(3):
            eid = int(ea[ia, e3])
            lid, ax = eid // 3, eid % 3
            lid2 = lid + int(step[ax])
            allow = 1.5 * h * (dv[lid] + dv[lid2]) / max(abs(v32[lid2] - v32[lid]), 1e-30) + 1e-6
            shift = float(np.abs(va[ia, e3] - vb[ib, e3]).max())
            worst = max(worst, shift / allow)
            assert shift <= allow, (key, e3, shift, allow)
    print(f"dense={dense}: {len(set(ta) ^ set(tb))} differing triangles of {len(ta)}, max vertex shift / "
          f"allowance {worst:.3f}, max |dv| {dv.max():.2e}")
    net.close()
