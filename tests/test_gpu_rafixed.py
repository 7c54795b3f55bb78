"""GPU parity of the RA-Fixed bound kernel (mode "rafixed": input symbols kept, all other
coefficients condensed into one radius per neuron) against the float64 oracle, through the C
interface.

Tolerance from the rounding model, as for the float32 affine path: a K-term float32 dot product
errs by at most ~K u |terms| (u = 2^-24) and the forms pass through H layers, so every bound
endpoint stays within 8 H w u (|x0| + spread) of the oracle's.  With inflation the bound encloses
every value sampled in the box (evaluated in float64), down to boxes of width 2^-20.
"""
import numpy as np
import pytest
import torch

from oracle import affine, mlp, octree
from synth import boxes, inr

from _helpers import to_np

pytestmark = pytest.mark.gpu

DIMS = [[3, 16, 16, 1], [3, 48, 48, 48, 1], [3, 128, 128, 128, 1], [3] + [256] * 5 + [1], [3, 512, 512, 1]]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _gpu_bounds(net, lo, hi, mode="rafixed", inflate=False):
    c, s = net.bound_cells(torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), mode=mode, prec="fp32",
                           inflate=inflate)
    torch.cuda.synchronize()
    return to_np(c).astype(np.float64), to_np(s).astype(np.float64)


@pytest.mark.parametrize("dims", DIMS, ids=lambda d: "x".join(map(str, d[1:-1])))
def test_rafixed_matches_oracle(pkg, dims):
    layers = inr.random_inr(dims, 21)
    net = pkg.Inr(layers)
    n = 1000 if dims[1] >= 256 else 3001          # many tiles of cells and a ragged last tile
    lo, hi = boxes.random_boxes(n, 22, -10, -1)
    c, s = _gpu_bounds(net, lo, hi)
    oc, os_ = affine.bound(layers, lo, hi, affine.RAFIXED, batch=256)
    H, w = len(dims) - 2, dims[1]
    tol = 8 * H * w * 2.0 ** -24 * (np.abs(oc) + os_) + 1e-7
    print(f"{dims[1:-1]}: max |dc| / tol {np.max(np.abs(c - oc) / tol):.3f}, max |ds| / tol "
          f"{np.max(np.abs(s - os_) / tol):.3f}")
    assert np.all(np.abs(c - oc) <= tol) and np.all(np.abs(s - os_) <= tol)
    net.close()


def test_rafixed_against_full_affine_on_gpu(pkg):
    """One hidden layer: RA-Fixed equals full affine arithmetic; two: never tighter."""
    for dims, equal in (([3, 64, 1], True), ([3, 64, 64, 1], False)):
        layers = inr.random_inr(dims, 5)
        net = pkg.Inr(layers)
        lo, hi = boxes.random_boxes(500, 6, -8, -1)
        c0, s0 = _gpu_bounds(net, lo, hi, mode="sound")
        c1, s1 = _gpu_bounds(net, lo, hi)
        tol = 1e-5 * (np.abs(c0) + s0) + 1e-7
        assert np.all(np.abs(c1 - c0) <= tol)
        if equal:
            assert np.all(np.abs(s1 - s0) <= tol)
        else:
            assert np.all(s1 >= s0 - tol) and np.mean(s1 > s0 + tol) > 0.5
        net.close()


@pytest.mark.parametrize("dims", [[3, 64, 64, 1], [3, 128, 128, 128, 1], [3, 48, 48, 48, 48, 1]])
def test_inflated_rafixed_contains_samples(pkg, dims):
    layers = inr.load_inr("small")[0] if dims == [3, 64, 64, 1] else inr.random_inr(dims, 3)
    net = pkg.Inr(layers)
    rng = np.random.default_rng(4)
    for lg in (-20, -12, -6, -2):
        lo, hi = boxes.random_boxes(200, 70 + lg, lg - 1, lg)
        c, s = _gpu_bounds(net, lo, hi, inflate=True)
        u = rng.uniform(size=(200, 400, 3))
        corners = np.array([[(q >> d) & 1 for d in range(3)] for q in range(8)], dtype=np.float64)
        u = np.concatenate([u, np.broadcast_to(corners, (200, 8, 3))], axis=1)
        lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
        pts = lo64[:, None, :] + u * (hi64 - lo64)[:, None, :]
        v = mlp.mlp_forward(layers, pts.reshape(-1, 3)).reshape(200, -1)
        lower = np.float32(c) - np.float32(s)
        upper = np.float32(c) + np.float32(s)
        assert np.all(v.min(1) >= lower.astype(np.float64))
        assert np.all(v.max(1) <= upper.astype(np.float64))
    net.close()


def test_rafixed_degenerate_boxes_and_errors(pkg):
    layers = inr.load_inr("small")[0]
    net = pkg.Inr(layers)
    x = np.random.default_rng(9).uniform(-1, 1, size=(100, 3)).astype(np.float32)
    c, s = _gpu_bounds(net, x, x)
    assert np.all(s == 0)
    np.testing.assert_allclose(c, mlp.mlp_forward(layers, x), atol=1e-5)
    e = torch.empty((0, 3), device="cuda")
    c, s = net.bound_cells(e, e, mode="rafixed")
    assert c.shape[0] == 0
    with pytest.raises(pkg.IsxError) as err:
        net.bound_cells(torch.zeros((4, 3), device="cuda"), torch.ones((4, 3), device="cuda"), mode="rafixed",
                        prec="bf16")
    assert err.value.status == 5
    with pytest.raises(pkg.IsxError) as err:
        net.extract(4, [0.5], mode="rafixed", prec="bf16")
    assert err.value.status == 5
    net.close()


def test_rafixed_extraction_matches_oracle(pkg):
    """Hierarchical extraction with RA-Fixed culling: the active set equals the oracle's except for
    cells whose ancestor bound endpoint lies within 1e-5 of the iso-value; sound RA-Fixed with
    inflation keeps every triangle of the dense extraction."""
    from test_gpu_extract import _check_extraction
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    L = wl.max_level
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
    res = net.extract(L, isos, mode="rafixed", prec="fp32")
    _check_extraction(layers, isos, L, vals, res, affine.RAFIXED, 0.0)
    full = net.extract(L, isos, mode="sound", prec="fp32")
    assert res["n_active"] >= full["n_active"] and sum(res["cells_bounded"]) >= sum(full["cells_bounded"])
    h = net.extract(L, isos, mode="rafixed", prec="fp32", inflate=True)
    d = net.extract(L, isos, prec="fp32", dense=True)
    gh = set(zip((to_np(h["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(h["tri_iso"]).tolist()))
    gd = set(zip((to_np(d["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(d["tri_iso"]).tolist()))
    assert gd <= gh and h["n_tris"] == d["n_tris"]
    print(f"RA-Fixed active {res['n_active']} bounded {sum(res['cells_bounded'])}; full AA active "
          f"{full['n_active']} bounded {sum(full['cells_bounded'])}")
    net.close()
