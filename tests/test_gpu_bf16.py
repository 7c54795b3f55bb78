"""GPU parity of the bfloat16 tensor-core bounds (tcgen05) against the float64 oracle, result by
result.

Band: each result's own band from the rounding-noise model of tests/_rounding_model.py (every
bfloat16 rounding of the row-batched path as an independent relative error of at most 2^-8, twelve
draws through the float64 layer loop, band = 10 x RMS deviation + a float32 floor).  Every test
prints the measured error next to the band it is checked against.  Extraction: the active (cell,
iso) pairs equal the oracle's except pairs with an ancestor-or-self whose oracle endpoint lies
within its own band of that iso-value, and the fraction of such excused pairs is printed and
asserted small.  Soundness with inflation is exact: the inflated bound must contain every sampled
value.
"""
import numpy as np
import pytest
import torch

from oracle import affine, mlp, octree
from synth import boxes, inr

import _rounding_model as rm
from _helpers import compare_active_pairs, near_maps, pack, to_np

pytestmark = pytest.mark.gpu


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


def check_against_bands(c, s, b, label):
    """|GPU - oracle| <= the result's band, for centre and spread; prints the worst ratio."""
    dc = np.abs(c - b["centre"])
    ds = np.abs(s - b["spread"])
    rc, rs = dc / b["band_c"], ds / b["band_s"]
    print(f"{label}: max |d x0| {dc.max():.2e} = {rc.max():.3f} of its band, max |d spread| {ds.max():.2e} = "
          f"{rs.max():.3f} of its band; median relative |d spread|/spread "
          f"{np.median(ds / np.maximum(b['spread'], 1e-30)):.1e}")
    assert np.all(dc <= b["band_c"]), f"{int((dc > b['band_c']).sum())} centres outside their band"
    assert np.all(ds <= b["band_s"]), f"{int((ds > b['band_s']).sum())} spreads outside their band"
    return rc.max(), rs.max()


@pytest.mark.parametrize("dims", [[3, 64, 64, 64, 1], [3, 128, 128, 1], [3, 128, 128, 128, 1],
                                  [3, 128] * 1 + [128] * 4 + [1], [3] + [256] * 5 + [1], "scientific"])
@pytest.mark.parametrize("mode", ["sound", "clt", "raua"])
def test_bf16_bounds_match_oracle(pkg, dims, mode):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 21)
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(613, 17, -9, -1)       # > 4 cells per CTA, ragged
    c, s = _bounds(net, lo, hi, mode, "bf16")
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(s))
    m = 24 if dims[1] == 256 or isinstance(dims, str) else 64
    idx = np.concatenate([np.arange(m), np.arange(613 - m, 613)])    # head and ragged tail
    b = rm.bound_bands(layers, lo[idx], hi[idx], mode, batch=16)
    check_against_bands(c[idx], s[idx], b, f"{dims if isinstance(dims, str) else dims[1:-1]} {mode}")
    net.close()


@pytest.mark.parametrize("dims,mode,m", [([3, 512, 512, 512, 1], "clt", 16), ([3, 512, 512, 512, 1], "sound", 16),
                                         ([3] + [512] * 8 + [1], "clt", 6)])
def test_bf16_width512_bounds_match_oracle(pkg, dims, mode, m):
    """Width 512 (the large configuration's width): the row GEMM holds a 128-row quarter of W_j per
    CTA and the split GEMM a 256-column half; head and ragged tail of 613 boxes against the oracle."""
    layers = inr.random_inr(dims, 23)
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(613, 19, -9, -1)
    c, s = _bounds(net, lo, hi, mode, "bf16")
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(s))
    idx = np.concatenate([np.arange(m), np.arange(613 - m, 613)])
    b = rm.bound_bands(layers, lo[idx], hi[idx], mode, batch=4)
    check_against_bands(c[idx], s[idx], b, f"w512 x {len(dims) - 2} {mode}")
    net.close()


@pytest.mark.parametrize("dims", [[3, 64, 64, 64, 64, 1], [3, 128, 128, 128, 1], [3] + [256] * 5 + [1],
                                  [3, 512, 512, 512, 1], "scientific"])
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
        # it also encloses the uninflated float64 affine bound, up to that bound's own rounding band
        b = rm.bound_bands(layers, lo[:16], hi[:16], "sound", batch=16)
        assert np.all(c[:16] - s[:16] <= b["centre"] - b["spread"] + b["band_lo"])
        assert np.all(c[:16] + s[:16] >= b["centre"] + b["spread"] - b["band_hi"])
        print(f"2^{lg} boxes: inflated radius / oracle radius median {np.median(s[:16] / b['spread']):.4f}")
    net.close()


def test_bf16_unsupported_width_is_reported(pkg):
    """Width 64 is bounded on the row-batched path; width 48 has no BF16 path."""
    net = pkg.Inr(inr.random_inr([3, 64, 64, 1], 1))
    lo = torch.zeros((4, 3), device="cuda")
    c, s = net.bound_cells(lo, lo + 0.1, mode="clt", prec="bf16")
    assert torch.isfinite(c).all() and torch.isfinite(s).all()
    net.close()
    net = pkg.Inr(inr.random_inr([3, 48, 48, 1], 1))
    with pytest.raises(pkg.IsxError) as e:
        net.bound_cells(lo, lo + 0.1, mode="clt", prec="bf16")
    assert e.value.status == 5
    net.close()


def check_extraction_pairs(layers, isos, L, res, mode, k, label, max_excused=0.01, act="relu", batch=256):
    """Active (cell, iso) pairs of a BF16 extraction against the oracle's hierarchy, with the
    per-result bands of the rounding model on every oracle node near an iso-value."""
    levels = octree.extract_active(layers, L, isos, mode, k=k, batch=batch, act=act)
    near, n_drawn = rm.near_iso_bits(levels, isos, layers, mode, k, coarse=0.05, act=act)
    maps = near_maps(levels, near)
    o_cells, o_masks = octree.active_cells(levels)
    o = dict(zip(pack(o_cells).tolist(), o_masks.tolist()))
    g = dict(zip((to_np(res["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist(),
                 (to_np(res["masks"]).astype(np.int64) & 0xFFFFFFFF).tolist()))
    n_pairs, n_diff, n_exc, bad = compare_active_pairs(o, g, maps, L)
    print(f"{label}: {n_pairs} active (cell, iso) pairs, {n_diff} differ from the oracle, {n_exc} "
          f"({n_exc / max(n_pairs, 1):.2%}) excused by their per-result bands; {n_drawn} oracle nodes given "
          f"model draws")
    assert not bad, f"{len(bad)} cells differ outside the band, e.g. {bad[:3]}"
    assert n_exc <= max_excused * n_pairs
    return levels, n_pairs, n_diff


def test_bf16_extraction_clt_matches_oracle(pkg):
    """UP k = 3 extraction of a 3->128x3->1 network at 32^3 on the row-batched path."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 31)
    net = pkg.Inr(layers)
    L = 5
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
    isos = np.quantile(vals, [0.3, 0.6]).astype(np.float32)
    res = net.extract(L, isos, mode="clt", k=3.0, prec="bf16")
    check_extraction_pairs(layers, isos, L, res, "clt", 3.0, "bf16 UP 128x3 32^3")
    net.close()


def test_bf16_extraction_width512_matches_oracle(pkg):
    """UP k = 3 extraction of a 3->512x3->1 network at 16^3 on the row-batched path."""
    layers = inr.random_inr([3, 512, 512, 512, 1], 33)
    net = pkg.Inr(layers)
    L = 4
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
    isos = np.quantile(vals, [0.35, 0.65]).astype(np.float32)
    res = net.extract(L, isos, mode="clt", k=3.0, prec="bf16")
    check_extraction_pairs(layers, isos, L, res, "clt", 3.0, "bf16 UP 512x3 16^3", batch=16)
    net.close()


@pytest.mark.parametrize("mode", ["sound", "raua"])
def test_bf16_extraction_small_matches_oracle(pkg, mode):
    """Sound and RA-UA extraction of the 3->64->64->1 fixture to 64^3 on the row-batched path."""
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    k = 3.0
    res = net.extract(wl.max_level, isos, mode=mode, k=k, prec="bf16")
    check_extraction_pairs(layers, isos, wl.max_level, res, mode, k, f"bf16 {mode} small 64^3", batch=512)
    net.close()


@pytest.mark.parametrize("name,L", [("random128x3", 5), ("small", 6), ("scientific", 6), ("scientific", 7)])
def test_bf16_sound_inflated_extraction_misses_nothing(pkg, name, L):
    """Sound bf16 bounds with inflation (row-batched path) keep every cell whose float32 corner values
    straddle an iso-value: the hierarchical triangles are exactly the dense ones (FNR = 0)."""
    if name == "random128x3":
        layers = inr.random_inr([3, 128, 128, 128, 1], 32)
        vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
        isos = np.quantile(vals, [0.4, 0.7]).astype(np.float32)
    else:
        layers, isos, _ = inr.load_inr(name)
    net = pkg.Inr(layers)
    from paper_2402_13861_gb300 import _lib
    _lib.profile_reset()
    h = net.extract(L, isos, mode="sound", prec="bf16", inflate=True, active_cap=1 << 20, tri_cap=1 << 22)
    launches = _lib.profile_read()
    d = net.extract(L, isos, prec="fp32", dense=True, active_cap=1 << 20, tri_cap=1 << 22)
    assert launches.get("rows_gemm", {"launches": 0})["launches"] > 0 or len(layers) < 4
    assert launches.get("bound_tc", {"launches": 0})["launches"] == 0
    gh = set(zip((to_np(h["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(h["tri_iso"]).tolist()))
    gd = set(zip((to_np(d["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(d["tri_iso"]).tolist()))
    print(f"{name} {1 << L}^3: {h['n_tris']} hierarchical vs {d['n_tris']} dense triangles, "
          f"{sum(h['cells_bounded'])} cells bounded, {h['n_active']} active")
    assert gd <= gh and h["n_tris"] == d["n_tris"] and d["n_tris"] > 0
    assert torch.equal(torch.sort(h["tri_edge"].reshape(-1))[0], torch.sort(d["tri_edge"].reshape(-1))[0])
    net.close()
