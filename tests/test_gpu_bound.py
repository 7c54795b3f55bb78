"""GPU parity of isx_bound_cells and isx_eval_points against the float64 oracle (called through
the C interface).

Tolerances.  The float32 path evaluates the same formulas as the oracle; its error is rounding
only: a K-term float32 dot product errs by at most ~K u |terms| (u = 2^-24), and the forms pass
through H layers.  For the 3->64->64->1 network that keeps every bound endpoint within 1e-5 of the
oracle (the band the active-set comparison allows).  For wider and deeper networks the test
scales the allowance with the rounding model: 8 * H * w * u * (|x0| + spread).
"""
import numpy as np
import pytest
import torch

from oracle import affine, mlp
from synth import boxes, inr

from _helpers import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


@pytest.fixture(scope="module")
def small(pkg):
    layers, isos, wl = inr.load_inr("small")
    return layers, pkg.Inr(layers)


def _gpu_bounds(net, lo, hi, mode, prec="fp32", inflate=False):
    c, s = net.bound_cells(torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), mode=mode, prec=prec,
                           inflate=inflate)
    torch.cuda.synchronize()
    return to_np(c).astype(np.float64), to_np(s).astype(np.float64)


@pytest.mark.parametrize("mode", ["sound", "clt", "raua"])
def test_fp32_bounds_match_oracle_small(small, mode):
    layers, net = small
    lo, hi = boxes.random_boxes(3000, 31, -10, 0)   # several chunks' worth of tiles, ragged count
    c, s = _gpu_bounds(net, lo, hi, mode)
    oc, os_ = affine.bound(layers, lo, hi, mode, batch=512)
    k = 0.0 if mode == "sound" else 3.0
    assert np.abs(c - oc).max() <= 1e-5
    assert np.abs(s - os_).max() <= 1e-5
    if mode != "sound":
        assert np.abs((c + k * s) - (oc + k * os_)).max() <= 1e-5


@pytest.mark.parametrize("dims", [[3, 128, 128, 128, 1], [3, 256] + [256] * 4 + [1]])
@pytest.mark.parametrize("mode", ["sound", "clt"])
def test_fp32_bounds_match_oracle_wide(pkg, dims, mode):
    layers = inr.random_inr(dims, 7)
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(67, 8, -9, -2)
    c, s = _gpu_bounds(net, lo, hi, mode)
    oc, os_ = affine.bound(layers, lo, hi, mode, batch=16)
    H, w = len(dims) - 2, dims[1]
    tol = 8 * H * w * 2.0 ** -24 * (np.abs(oc) + os_) + 1e-7
    assert np.all(np.abs(c - oc) <= tol)
    assert np.all(np.abs(s - os_) <= tol)
    net.close()


@pytest.mark.parametrize("dims", [[3, 64, 64, 1], [3, 128, 128, 128, 1]])
def test_inflated_sound_bounds_contain_samples(pkg, dims):
    """With rounding-error inflation the float32 bound encloses every sampled value (evaluated in
    float64 by the oracle), including boxes of width 2^-20 where rounding dominates."""
    layers = inr.load_inr("small")[0] if dims == [3, 64, 64, 1] else inr.random_inr(dims, 3)
    net = pkg.Inr(layers)
    rng = np.random.default_rng(4)
    for lg in (-20, -12, -6, -2):
        lo, hi = boxes.random_boxes(200, 50 + lg, lg - 1, lg)
        c, s = _gpu_bounds(net, lo, hi, "sound", inflate=True)
        u = rng.uniform(size=(200, 400, 3))
        corners = np.array([[(q >> d) & 1 for d in range(3)] for q in range(8)], dtype=np.float64)
        u = np.concatenate([u, np.broadcast_to(corners, (200, 8, 3))], axis=1)
        lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
        pts = lo64[:, None, :] + u * (hi64 - lo64)[:, None, :]
        v = mlp.mlp_forward(layers, pts.reshape(-1, 3)).reshape(200, -1)
        lower = np.float32(c) - np.float32(s)
        upper = np.float32(c) + np.float32(s)
        assert np.all(v.min(1) >= lower.astype(np.float64) - 0.0)
        assert np.all(v.max(1) <= upper.astype(np.float64) + 0.0)
    net.close()


def test_degenerate_boxes_and_empty_batch(small):
    layers, net = small
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(100, 3)).astype(np.float32)
    c, s = _gpu_bounds(net, x, x, "sound")
    assert np.all(s == 0)
    np.testing.assert_allclose(c, mlp.mlp_forward(layers, x), atol=1e-5)
    c, s = _gpu_bounds(net, x, x, "clt")
    assert np.all(s == 0)
    np.testing.assert_allclose(c, mlp.mlp_forward(layers, x), atol=1e-5)
    e = torch.empty((0, 3), device="cuda")
    c, s = net.bound_cells(e, e, mode="sound")
    assert c.shape[0] == 0


def test_eval_points_matches_oracle(small, pkg):
    layers, net = small
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, size=(10007, 3)).astype(np.float32)
    v = to_np(net.eval_points(torch.tensor(x, device="cuda")))
    np.testing.assert_allclose(v, mlp.mlp_forward(layers, x), atol=1e-5, rtol=0)
    wide = inr.random_inr([3] + [256] * 5 + [1], 2)
    net2 = pkg.Inr(wide)
    x = x[:2049]
    v = to_np(net2.eval_points(torch.tensor(x, device="cuda"))).astype(np.float64)
    ref = mlp.mlp_forward(wide, x)
    assert np.all(np.abs(v - ref) <= 1e-5 * (1 + np.abs(ref)) * 10)
    net2.close()


def test_fp32_gemm_autotuner_picks_a_shape_and_keeps_results(pkg):
    """The autotuner times the FP32 GEMM tile shapes on first use of a (width, rows) key and caches
    one; bounds computed with the cached shape equal the first (tuning) call bit for bit and the
    float64 oracle within the FP32 band."""
    pkg.tune_reset()
    layers = inr.random_inr([3, 64, 64, 64, 1], 12)
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(300, 13, -8, -2)
    dlo, dhi = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    c1, s1 = [x.clone() for x in net.bound_cells(dlo, dhi, mode="clt", prec="fp32")]
    table = pkg.tune_read()
    keys = [k for k in table if k.startswith("gemm_fp32 w=64")]
    print({k: (table[k]["choice"], round(table[k]["ms_best"], 4), round(table[k]["ms_first"], 4)) for k in keys})
    assert keys and all(0 <= table[k]["variant"] < table[k]["n_variants"] == 5 for k in keys)
    c2, s2 = net.bound_cells(dlo, dhi, mode="clt", prec="fp32")
    assert torch.equal(c1, c2) and torch.equal(s1, s2)
    oc, os_ = affine.bound(layers, lo[:50], hi[:50], "clt", batch=25)
    s = s2.cpu().numpy()[:50].astype(np.float64)
    assert np.all(np.abs(s - os_) <= 1e-4 * os_ + 1e-7)
    net.close()


@pytest.mark.parametrize("mode", ["sound", "clt"])
def test_fp32_bounds_large_network_shape(pkg, mode):
    """The large configuration's network shape (3 -> 512 x 8 -> 1: up to 4099 noise symbols per
    neuron) on the float32 path against the oracle, a few boxes from level 2 to level 10 size."""
    dims = [3] + [512] * 8 + [1]
    layers = inr.random_inr(dims, 77)
    rng = np.random.default_rng(78)
    layers = [(W, rng.normal(0, 0.05, size=b.shape).astype(np.float32)) for W, b in layers]
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(9, 79, -10, -2)
    c, s = _gpu_bounds(net, lo, hi, mode)
    oc, os_ = affine.bound(layers, lo, hi, mode, batch=3)
    H, w = len(dims) - 2, dims[1]
    tol = 8 * H * w * 2.0 ** -24 * (np.abs(oc) + os_) + 1e-7
    print(f"large {mode}: max |dc| / tol {np.max(np.abs(c - oc) / tol):.3f}, max |ds| / tol "
          f"{np.max(np.abs(s - os_) / tol):.3f}")
    assert np.all(np.abs(c - oc) <= tol) and np.all(np.abs(s - os_) <= tol)
    net.close()
