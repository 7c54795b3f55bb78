"""GPU parity of the k-d form of Algorithm 1 (widest-side bisection, kd_tree = 1) against the float64
oracle (octree.kd_extract_active), through the C interface.

Acceptance as for the octree (float32 path): the active sets agree except for cells with an
ancestor-or-self box (at any depth of the k-d tree) whose oracle bound endpoint lies within 1e-5 of
an iso-value; triangles of clean common cells are identical.  Sound bounds with inflation keep every
cell the dense GPU extraction marches.
"""
import numpy as np
import pytest
import torch

from oracle import mc, mlp, octree
from synth import inr

from _helpers import pack, to_np, unpack

pytestmark = pytest.mark.gpu

BAND = 1e-5


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
    return layers, isos, wl, pkg.Inr(layers)


def _splits(depth):
    return np.array([(depth + 2 - a) // 3 for a in range(3)])


def _band_sets(depths, isos):
    out = []
    for dv in depths:
        near = np.zeros(dv["ijk"].shape[0], dtype=bool)
        for c in isos:
            near |= (np.abs(dv["lower"] - c) <= BAND) | (np.abs(dv["upper"] - c) <= BAND)
        out.append(set(map(tuple, dv["ijk"][near].tolist())))
    return out


def _excused(code, bands, L):
    ijk = unpack([code])[0]
    for d, s in enumerate(bands):
        if tuple((ijk >> (L - _splits(d))).tolist()) in s:
            return True
    return False


@pytest.mark.parametrize("mode,k", [("sound", 0.0), ("clt", 3.0)])
def test_kd_extraction_matches_oracle(small, mode, k):
    layers, isos, wl, net = small
    L = min(wl.max_level, 6)
    R = 1 << L
    vals = mlp.mlp_forward(layers, octree.lattice_points(R))
    res = net.extract(L, isos, mode=mode, k=k, prec="fp32", kd_tree=True)
    depths = octree.kd_extract_active(layers, L, isos, mode, k=k, batch=512)
    o_cells, o_masks = octree.active_cells(depths)
    o_map = dict(zip(pack(o_cells).tolist(), o_masks.tolist()))
    g_codes = to_np(res["codes"]).astype(np.int64) & 0xFFFFFFFF
    g_masks = to_np(res["masks"]).astype(np.int64) & 0xFFFFFFFF
    g_map = dict(zip(g_codes.tolist(), g_masks.tolist()))
    assert len(g_map) == len(g_codes)
    diff = list(set(o_map) ^ set(g_map)) + [c for c in set(o_map) & set(g_map) if o_map[c] != g_map[c]]
    bands = _band_sets(depths, isos)
    bad = [c for c in diff if not _excused(c, bands, L)]
    assert not bad, f"{len(bad)} active-set differences outside the 1e-5 band"
    # boxes bounded per octree level: depths 3l-2 .. 3l are filed under level l
    want = [0] * (L + 1)
    for dv in depths:
        want[(dv["depth"] + 2) // 3] += dv["ijk"].shape[0]
    for l in range(L + 1):
        assert abs(res["cells_bounded"][l] - want[l]) <= 8 * len(diff)
    # the k-d tree never keeps a cell the octree culls (same bound on the same cube, nested masks)
    oc = net.extract(L, isos, mode=mode, k=k, prec="fp32")
    oc_codes = set((to_np(oc["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist())
    assert len(set(g_map) - oc_codes) <= len(diff)
    # triangles of clean common cells
    checked = 0
    g_tri = {}
    tc = to_np(res["tri_cell"]).astype(np.int64) & 0xFFFFFFFF
    tq, te, tv = to_np(res["tri_iso"]), to_np(res["tri_edge"]), to_np(res["tri_vert"]).astype(np.float64)
    for t in range(tc.shape[0]):
        g_tri.setdefault((int(tc[t]), int(tq[t])), []).append((tuple(te[t]), tv[t]))
    for q, c in enumerate(isos):
        codes = [cc for cc in set(o_map) & set(g_map) if (o_map[cc] >> q) & 1 and (g_map[cc] >> q) & 1]
        if not codes:
            continue
        ijk = unpack(codes)
        cv = mc.corner_values(vals, ijk, R)
        clean = np.all(np.abs(cv - c) > BAND, axis=1)
        e, p, cell = mc.march(vals, ijk[clean], R, c)
        ccodes = np.asarray(codes)[clean]
        o_tri = {}
        for t in range(e.shape[0]):
            o_tri.setdefault(int(ccodes[cell[t]]), []).append((tuple(e[t]), p[t]))
        for code, tris in o_tri.items():
            got = g_tri.get((code, q), [])
            assert [t[0] for t in tris] == [t[0] for t in got], (code, q)
            for (_, pa), (_, pb) in zip(tris, got):
                assert np.abs(pa - pb).max() <= 1e-4
            checked += len(tris)
    assert checked > 1000
    print(f"{mode}: active {res['n_active']} (octree {oc['n_active']}), bounded {sum(res['cells_bounded'])} "
          f"(octree {sum(oc['cells_bounded'])}), {len(diff)} band differences")


def test_kd_sound_inflated_keeps_every_dense_triangle(small):
    layers, isos, wl, net = small
    L = wl.max_level
    h = net.extract(L, isos, mode="sound", prec="fp32", inflate=True, kd_tree=True)
    d = net.extract(L, isos, prec="fp32", dense=True)
    assert h["n_tris"] == d["n_tris"]
    gh = set(zip((to_np(h["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(h["tri_iso"]).tolist()))
    gd = set(zip((to_np(d["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(d["tri_iso"]).tolist()))
    assert gd <= gh


def test_kd_bf16_tensor_core_bounds(pkg):
    """The tensor-core bound kernel takes the k-d boxes too: sound BF16 with inflation still keeps
    every dense triangle, and CLT BF16 gives the FP32 active set up to cells near the iso-value."""
    layers = inr.random_inr([3, 128, 128, 128, 1], 31)
    net = pkg.Inr(layers)
    L = 6
    vals = mlp.mlp_forward(layers, octree.lattice_points(16))
    isos = np.quantile(vals, [0.3, 0.6]).astype(np.float32)
    h = net.extract(L, isos, mode="sound", prec="bf16", inflate=True, kd_tree=True, active_cap=1 << 18,
                    tri_cap=1 << 20)
    d = net.extract(L, isos, prec="fp32", dense=True, active_cap=1 << 18, tri_cap=1 << 20)
    gh = set(zip((to_np(h["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(h["tri_iso"]).tolist()))
    gd = set(zip((to_np(d["tri_cell"]).astype(np.int64) & 0xFFFFFFFF).tolist(), to_np(d["tri_iso"]).tolist()))
    assert gd <= gh and h["n_tris"] == d["n_tris"]
    a = net.extract(L, isos, mode="clt", k=3.0, prec="bf16", kd_tree=True)
    b = net.extract(L, isos, mode="clt", k=3.0, prec="fp32", kd_tree=True)
    sa = set((to_np(a["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist())
    sb = set((to_np(b["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist())
    print(f"bf16 vs fp32 k-d active: {len(sa)} vs {len(sb)}, symmetric difference {len(sa ^ sb)}")
    assert len(sa ^ sb) <= 0.01 * max(len(sb), 1)
    net.close()


def test_kd_rejects_proposer(small, pkg):
    layers, isos, wl, net = small
    params = np.zeros(8961, dtype=np.float32)
    prop = pkg.Proposer(params, np.zeros(8), np.ones(8))
    with pytest.raises(pkg.IsxError) as e:
        net.extract(4, isos, mode="clt", proposer=prop, kd_tree=True)
    assert e.value.status == 5
    prop.close()
