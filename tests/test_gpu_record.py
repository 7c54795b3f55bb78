"""The level record of a hierarchical extraction (isx_level_record), the dense extraction's list of
crossing cells, and the bounded device-side wait, through the C interface.

- The record lists, level by level, exactly the cells Algorithm 1 visits: checked against the
  float64 oracle's level loop (float32 bounds; cells equal up to descendants of a node whose oracle
  endpoint lies within 1e-5 of an iso-value), and against the extraction's own output: the record's
  finest cells culled with their recorded bounds are the active list, and each level's cells are
  the children of the previous level's survivors.
- A record that does not fit returns ISX_ERR_CAPACITY with the required size.
- Dense extraction lists the cells with a triangle of each iso-value: the oracle's crossing cells
  on the same float32 lattice values, up to cells with a corner value within 1e-5 of the iso-value.
- isx_check_bounded_wait: a wait on an mbarrier that nothing completes expires after its limit and
  reports ISX_ERR_TIMEOUT; the next bound call on the same context succeeds.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import affine, mc, mlp, octree
from synth import boxes, inr

from _helpers import band_codes, excused, pack, to_np, unpack

pytestmark = pytest.mark.gpu
BAND = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _np64(t):
    return to_np(t).astype(np.int64) & 0xFFFFFFFF


@pytest.mark.parametrize("mode,k", [("sound", 0.0), ("clt", 3.0)])
def test_record_equals_oracle_level_loop(pkg, mode, k):
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    L = 5
    res = net.extract(L, isos, mode=mode, k=k, prec="fp32", record=True)
    levels = octree.extract_active(layers, L, isos, mode, k=k, batch=512)
    bands = band_codes(levels, isos, BAND, L)
    full = (1 << len(isos)) - 1
    for l, (rec, lv) in enumerate(zip(res["levels"], levels)):
        g = dict(zip(_np64(rec["codes"]).tolist(), _np64(rec["masks"]).tolist()))
        assert len(g) == rec["codes"].numel()                          # each cell once
        o = dict(zip(pack(lv["ijk"]).tolist(), lv["mask_in"].tolist()))
        diff = (set(g) ^ set(o)) | {c for c in set(g) & set(o) if g[c] != o[c]}
        # a cell that differs descends from a node (strictly above this level) near an iso-value
        for c in diff:
            ijk = unpack([c])[0]
            assert any(int(pack((ijk >> (l - a))[None])[0]) in bands[a] for a in range(l)), (l, c)
        # bounds of common cells within the float32 band of the oracle's
        common = sorted(set(g) & set(o))
        gi = {c: i for i, c in enumerate(_np64(rec["codes"]).tolist())}
        oi = {c: i for i, c in enumerate(pack(lv["ijk"]).tolist())}
        gc = to_np(rec["centre"]).astype(np.float64)[[gi[c] for c in common]]
        gs = to_np(rec["spread"]).astype(np.float64)[[gi[c] for c in common]]
        oc, os_ = lv["centre"][[oi[c] for c in common]], lv["spread"][[oi[c] for c in common]]
        tol = 8 * 3 * 64 * 2.0 ** -24 * (np.abs(oc) + os_) + 1e-6
        assert np.all(np.abs(gc - oc) <= tol) and np.all(np.abs(gs - os_) <= tol), l
        if l == 0:
            assert g == {0: full}
    # the record is the extraction's own level loop: children of the survivors, and the finest
    # cells' cull test on their recorded bounds is the active list
    # (an endpoint within a few float32 roundings of an iso-value may fall either way: k sigma is
    # subtracted with one rounding or two; such cells are left out of the exact comparison)
    iso = torch.tensor(np.asarray(isos, np.float64), device="cuda")
    for l, rec in enumerate(res["levels"]):
        c, s = rec["centre"].double(), rec["spread"].double()
        kk = 1.0 if mode == "sound" else k
        lo, hi = c - kk * s, c + kk * s
        bits = ((lo[:, None] <= iso[None, :]) & (iso[None, :] <= hi[:, None])).to(torch.int64)
        tie = (((lo[:, None] - iso[None, :]).abs() <= 2.0 ** -20 * (c.abs() + kk * s)[:, None]) |
               ((hi[:, None] - iso[None, :]).abs() <= 2.0 ** -20 * (c.abs() + kk * s)[:, None])).any(1)
        keep = (rec["masks"].to(torch.int64) & 0xFFFFFFFF) & (bits << torch.arange(len(isos), device="cuda")).sum(1)
        alive = keep != 0
        n_tie = int(tie.sum())
        if l < L:
            nxt = res["levels"][l + 1]
            assert abs(nxt["codes"].numel() - 8 * int(alive.sum())) <= 8 * n_tie, l
            assert abs(res["cells_kept"][l] - int(alive.sum())) <= n_tie
        else:
            a = dict(zip(_np64(rec["codes"][alive & ~tie]).tolist(), to_np(keep[alive & ~tie]).tolist()))
            got = dict(zip(_np64(res["codes"]).tolist(), _np64(res["masks"]).tolist()))
            ties = set(_np64(rec["codes"][tie]).tolist())
            assert a == {c_: m_ for c_, m_ in got.items() if c_ not in ties}
    print(f"{mode}: visited per level {[r['codes'].numel() for r in res['levels']]}")
    net.close()


def test_record_capacity_and_unsupported(pkg):
    from paper_2402_13861_gb300 import _lib
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    L = 4
    full = net.extract(L, isos, mode="clt", k=3.0, prec="fp32", record=True)
    need = sum(r["codes"].numel() for r in full["levels"])
    # a record of 10 entries: capacity error with the required size, nothing written past it
    p = net.params(L, isos, mode="clt", k=3.0, prec="fp32")
    bufs = {n: torch.full((need,), -7, dtype=torch.int32, device="cuda") for n in ("code", "mask")}
    fl = {n: torch.full((need,), -7.0, device="cuda") for n in ("c", "s")}
    rec = _lib.LevelRecord()
    rec.d_code, rec.d_mask = bufs["code"].data_ptr(), bufs["mask"].data_ptr()
    rec.d_center, rec.d_spread = fl["c"].data_ptr(), fl["s"].data_ptr()
    rec.cap = 10
    p.record = C.cast(C.pointer(rec), C.c_void_p)
    ac = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    tv = torch.empty((1 << 18, 3, 3), device="cuda")
    te = torch.empty((1 << 18, 3), dtype=torch.int64, device="cuda")
    ti = torch.empty(1 << 18, dtype=torch.int32, device="cuda")
    m = _lib.Mesh()
    m.d_active_code, m.d_active_mask, m.active_cap = ac.data_ptr(), ac.data_ptr(), 1 << 16
    m.d_tri_vert, m.d_tri_edge, m.d_tri_iso, m.d_tri_cell, m.tri_cap = (tv.data_ptr(), te.data_ptr(), ti.data_ptr(),
                                                                          ti.data_ptr(), 1 << 18)
    st = _lib.load().isx_extract_isosurface(net.handle, C.byref(p), C.byref(m),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 3 and rec.level_off[L + 1] == need
    assert bool((bufs["code"][10:] == -7).all()) and bool((fl["s"][10:] == -7.0).all())
    # k-d trees and proposers are not recorded
    with pytest.raises(pkg.IsxError) as e:
        net.extract(L, isos, mode="clt", k=3.0, prec="fp32", record=True, kd_tree=True)
    assert e.value.status == 5
    net.close()


def test_dense_lists_crossing_cells(pkg):
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    L = 5
    R = 1 << L
    more = np.asarray(list(isos) + [0.3], dtype=np.float32)
    res = net.extract(L, more, prec="fp32", dense=True)
    g = dict(zip(_np64(res["codes"]).tolist(), _np64(res["masks"]).tolist()))
    assert len(g) == res["n_active"] > 0
    vals32 = to_np(net.eval_points(torch.tensor(octree.lattice_points(R), dtype=torch.float32, device="cuda")))
    vals32 = vals32.astype(np.float64)
    o = {}
    for q, c in enumerate(more.astype(np.float64)):
        for code in pack(mc.crossing_cells(vals32, R, c)).tolist():
            o[code] = o.get(code, 0) | (1 << q)
    diff = (set(g) ^ set(o)) | {c for c in set(g) & set(o) if g[c] != o[c]}
    for code in diff:
        cv = mc.corner_values(vals32, unpack([code]), R)[0]
        assert np.any(np.abs(cv[:, None] - more[None, :].astype(np.float64)) <= BAND), code
    print(f"dense: {len(g)} cells with triangles, {len(diff)} differ from the oracle's crossing cells")
    # the cells are in cell order (i fastest, then j, then k)
    ijk = unpack(_np64(res["codes"]))
    lin = (ijk[:, 2] * R + ijk[:, 1]) * R + ijk[:, 0]
    assert np.all(np.diff(lin) > 0)
    net.close()


def test_bounded_wait_expires_and_the_context_stays_usable(pkg):
    from paper_2402_13861_gb300 import _lib
    assert _lib.check_bounded_wait(20000) == 4                 # 20 us: ISX_ERR_TIMEOUT
    assert b"expired" in _lib.load().isx_last_error()
    assert _lib.check_bounded_wait(10) == 1                    # limit below 1 us: argument error
    net = pkg.Inr(inr.random_inr([3, 128, 128, 128, 1], 3))
    lo, hi = boxes.random_boxes(300, 3, -7, -2)
    c, s = net.bound_cells(torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda"), mode="clt", prec="bf16")
    torch.cuda.synchronize()
    oc, os_ = affine.bound(inr.random_inr([3, 128, 128, 128, 1], 3), lo[:8], hi[:8], "clt")
    assert np.allclose(to_np(s)[:8], os_, rtol=0.02)
    net.close()
