"""GPU parity of the bfloat16 tensor-core path (tcgen05) against the float64 oracle.

Tolerance derived from the arithmetic: every coefficient passes through at most 3 bfloat16
roundings per layer (stored coefficient, W, alpha * W; unit roundoff u_b = 2^-8) plus float32
accumulation, so after H hidden layers a coefficient carries a relative error below
(1 + u_b)^(3 H) - 1 < 3 H u_b (1.1 at most for the shapes here).  The bounds are sums of such
coefficients through data-dependent linearisations, so the test allows |delta spread| <=
3 H u_b * spread and |delta centre| <= 3 H u_b * (|x0| + spread); the measured errors are printed
(they sit two orders of magnitude below the allowance).  Soundness with inflation is exact: the
inflated bf16 bound must contain every sampled value.
"""
import numpy as np
import pytest
import torch

from oracle import affine, mc, mlp, octree
from synth import boxes, inr

from _helpers import band_codes, excused, pack, to_np

pytestmark = pytest.mark.gpu
UB = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _bounds(net, lo, hi, mode, prec, inflate=False):
    c, s = net.bound_cells(torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), mode=mode, prec=prec,
                           inflate=inflate)
    torch.cuda.synchronize()
    return to_np(c).astype(np.float64), to_np(s).astype(np.float64)


@pytest.mark.parametrize("dims", [[3, 64, 64, 64, 1], [3, 128, 128, 1], [3, 128, 128, 128, 1],
                                  [3, 128] * 1 + [128] * 4 + [1], [3] + [256] * 5 + [1], "scientific"])
@pytest.mark.parametrize("mode", ["sound", "clt", "raua"])
def test_bf16_bounds_match_oracle(pkg, dims, mode):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 21)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(613, 17, -9, -1)       # > 4 cells per CTA, ragged
    c, s = _bounds(net, lo, hi, mode, "bf16")
    m = 97
    oc, os_ = affine.bound(layers, lo[:m], hi[:m], mode, batch=32)
    tol = 3 * H * UB
    dc = np.abs(c[:m] - oc)
    ds = np.abs(s[:m] - os_)
    print(f"{dims} {mode}: max |dc|/(|x0|+s) = {(dc / (np.abs(oc) + os_)).max():.2e}, "
          f"max |ds|/s = {(ds / np.maximum(os_, 1e-30)).max():.2e}")
    assert np.all(ds <= tol * os_ + 1e-6)
    assert np.all(dc <= tol * (np.abs(oc) + os_) + 1e-6)
    # the tail of the batch (processed by other CTAs) agrees with the float32 path
    c32, s32 = _bounds(net, lo, hi, mode, "fp32")
    assert np.all(np.abs(s - s32) <= tol * s32 + 1e-6)
    net.close()


@pytest.mark.parametrize("dims", [[3, 128, 128, 128, 1], "scientific"])
def test_bf16_inflated_sound_bounds_contain_samples(pkg, dims):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 5)
    net = pkg.Inr(layers)
    rng = np.random.default_rng(8)
    for lg in (-16, -10, -5, -2):
        n = 150
        lo, hi = boxes.random_boxes(n, 90 + lg, lg - 1, lg)
        c, s = _bounds(net, lo, hi, "sound", "bf16", inflate=True)
        u = rng.uniform(size=(n, 300, 3))
        corners = np.array([[(q >> d) & 1 for d in range(3)] for q in range(8)], dtype=np.float64)
        u = np.concatenate([u, np.broadcast_to(corners, (n, 8, 3))], axis=1)
        pts = lo.astype(np.float64)[:, None, :] + u * (hi.astype(np.float64) - lo.astype(np.float64))[:, None, :]
        v = mlp.mlp_forward(layers, pts.reshape(-1, 3)).reshape(n, -1)
        lower = (np.float32(c) - np.float32(s)).astype(np.float64)
        upper = (np.float32(c) + np.float32(s)).astype(np.float64)
        assert np.all(v.min(1) >= lower) and np.all(v.max(1) <= upper)
        # and it encloses the uninflated float64 affine bound up to the stated bf16 error
        oc, os_ = affine.bound(layers, lo[:40], hi[:40], "sound", batch=20)
        assert np.all(s[:40] >= os_ * (1 - 3 * (len(layers) - 1) * UB))
    net.close()


def test_bf16_unsupported_width_is_reported(pkg):
    """Width 64 is bounded on the row-batched path (UP, RA-UA, sound without inflation); sound bounds
    with inflation need the per-cell kernel (widths 128 and 256) and width 48 has no BF16 path."""
    net = pkg.Inr(inr.random_inr([3, 64, 64, 1], 1))
    lo = torch.zeros((4, 3), device="cuda")
    c, s = net.bound_cells(lo, lo + 0.1, mode="clt", prec="bf16")
    assert torch.isfinite(c).all() and torch.isfinite(s).all()
    with pytest.raises(pkg.IsxError) as e:
        net.bound_cells(lo, lo + 0.1, mode="sound", prec="bf16", inflate=True)
    assert e.value.status == 5
    net.close()
    net = pkg.Inr(inr.random_inr([3, 48, 48, 1], 1))
    with pytest.raises(pkg.IsxError) as e:
        net.bound_cells(lo, lo + 0.1, mode="clt", prec="bf16")
    assert e.value.status == 5
    net.close()


def test_bf16_extraction_clt_matches_oracle(pkg):
    """CLT k = 3 extraction of a 3->128x3->1 network at 32^3: active sets equal the oracle's up to
    the bf16 band (bound endpoints within 3 H u_b (|mu| + k sigma) of an iso-value)."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 31)
    net = pkg.Inr(layers)
    L = 5
    R = 1 << L
    vals = mlp.mlp_forward(layers, octree.lattice_points(R))
    isos = np.quantile(vals, [0.3, 0.6]).astype(np.float32)
    res = net.extract(L, isos, mode="clt", k=3.0, prec="bf16")
    levels = octree.extract_active(layers, L, isos, affine.CLT, k=3.0, batch=256)
    H = 3
    band = 3 * H * UB * max(np.abs(lv["centre"]).max() + 3 * lv["spread"].max() for lv in levels if lv["ijk"].size)
    bands = band_codes(levels, isos, band, L)
    o_cells, o_masks = octree.active_cells(levels)
    o = dict(zip(pack(o_cells).tolist(), o_masks.tolist()))
    g = dict(zip((to_np(res["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist(),
                 (to_np(res["masks"]).astype(np.int64) & 0xFFFFFFFF).tolist()))
    diff = (set(o) ^ set(g)) | {c for c in set(o) & set(g) if o[c] != g[c]}
    assert all(excused(c, bands, L) for c in diff)
    print(f"bf16 CLT: {len(diff)} differing cells of {len(o)} (band {band:.2e})")
    net.close()


def test_bf16_sound_inflated_extraction_misses_nothing(pkg):
    """Sound bf16 bounds with inflation keep every cell whose float32 corner values straddle the
    iso-value: hierarchical triangles equal the dense ones."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 32)
    net = pkg.Inr(layers)
    L = 5
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
    isos = np.quantile(vals, [0.4, 0.7]).astype(np.float32)
    h = net.extract(L, isos, mode="sound", prec="bf16", inflate=True)
    d = net.extract(L, isos, prec="fp32", dense=True)
    assert h["n_tris"] == d["n_tris"] and d["n_tris"] > 0
    net.close()
