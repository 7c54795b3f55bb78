"""Batched extraction (isx_batch_*): many extractions in flight on worker streams.
- Every entry equals its own single extraction bit for bit (active cells, masks, triangles, edge
  ids, vertices), for entries of mixed width, depth, mode, precision, k, iso count and level, with
  an INR shared by two entries, over repeated runs and for several worker counts.
- One entry is checked against the float64 oracle's extraction with per-result bands
  (tests/_rounding_model.py).
- A capacity shortfall in one entry reports that entry's required counts; the others complete.
- Malformed batches are rejected.
"""
import numpy as np
import pytest
import torch

from oracle import mlp, octree
from synth import inr

from test_gpu_bf16 import check_extraction_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _entries():
    specs = [([3, 128, 128, 128, 1], 41, 5, 2, dict(mode="clt", k=3.0, prec="bf16")),
             ([3] + [256] * 4 + [1], 42, 6, 3, dict(mode="clt", k=2.0, prec="bf16")),
             ([3] + [128] * 5 + [1], 43, 4, 1, dict(mode="sound", prec="bf16", inflate=True)),
             ([3, 256, 256, 1], 44, 5, 4, dict(mode="raua", k=3.0, prec="bf16")),
             ([3, 64, 64, 64, 1], 45, 5, 2, dict(mode="sound", prec="fp32")),
             ([3, 64, 64, 1], 46, 6, 16, dict(mode="clt", k=3.0, prec="bf16", eval_prec="fp32"))]
    out = []
    for dims, seed, L, niso, kw in specs:
        layers = inr.random_inr(dims, seed)
        vals = mlp.mlp_forward(layers, octree.lattice_points(16))
        isos = np.quantile(vals, np.linspace(0.3, 0.7, niso)).astype(np.float32)
        out.append((layers, dict(max_level=L, isos=isos, **kw)))
    return out


def _same(a, b):
    assert a["n_active"] == b["n_active"] and a["n_tris"] == b["n_tris"]
    assert torch.equal(a["codes"], b["codes"]) and torch.equal(a["masks"], b["masks"])
    assert torch.equal(a["tri_edge"], b["tri_edge"]) and torch.equal(a["tri_iso"], b["tri_iso"])
    assert torch.equal(a["tri_vert"], b["tri_vert"])


@pytest.mark.parametrize("workers", [1, 3, 8])
def test_batch_equals_single_extractions(pkg, workers):
    ents = _entries()
    nets = [pkg.Inr(layers) for layers, _ in ents]
    # entry 6 reuses entry 0's INR with other isos: the two run on one worker, in order
    ents.append((ents[0][0], dict(ents[0][1], isos=ents[0][1]["isos"][::-1].copy(), k=2.5)))
    nets.append(nets[0])
    singles = [net.extract(**p) for net, (_, p) in zip(nets, ents)]
    singles = [dict(s, codes=s["codes"].clone(), masks=s["masks"].clone(), tri_edge=s["tri_edge"].clone(),
                    tri_iso=s["tri_iso"].clone(), tri_vert=s["tri_vert"].clone()) for s in singles]
    batch = pkg.Batch(nets, [p for _, p in ents], workers=workers)
    for rep in range(2):
        res = batch.run()
        for r, s in zip(res, singles):
            _same(r, s)
    print(f"{workers} workers: active cells per entry", [r["n_active"] for r in res])
    if workers == 3:
        layers, p = ents[0]
        check_extraction_pairs(layers, p["isos"], p["max_level"], res[0], "clt", p["k"], "batch entry 0")
    batch.close()
    for net in nets[:-1]:
        net.close()


def test_batch_capacity_is_per_entry(pkg):
    from paper_2402_13861_gb300 import _lib
    import ctypes as C
    ents = _entries()[:3]
    nets = [pkg.Inr(layers) for layers, _ in ents]
    singles = [net.extract(**p) for net, (_, p) in zip(nets, ents)]
    batch = pkg.Batch(nets, [p for _, p in ents], workers=3)
    n = len(ents)
    meshes = (_lib.Mesh * n)()
    keep = []
    for i in range(n):
        cap_a = 4 if i == 1 else 1 << 18
        ca = torch.empty(max(cap_a, 1), dtype=torch.int32, device="cuda")
        ma = torch.empty_like(ca)
        tv = torch.empty((1 << 20, 3, 3), device="cuda")
        te = torch.empty((1 << 20, 3), dtype=torch.int64, device="cuda")
        ti = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
        keep += [ca, ma, tv, te, ti]
        m = meshes[i]
        m.d_active_code, m.d_active_mask, m.active_cap = ca.data_ptr(), ma.data_ptr(), cap_a
        m.d_tri_vert, m.d_tri_edge, m.d_tri_iso, m.d_tri_cell, m.tri_cap = (tv.data_ptr(), te.data_ptr(), ti.data_ptr(),
                                                                              ti.data_ptr(), 1 << 20)
    st = _lib.load().isx_batch_run(batch._h, meshes, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 3 and b"entry 1" in _lib.load().isx_last_error()
    assert meshes[1].n_active == singles[1]["n_active"]
    for i in (0, 2):
        assert meshes[i].n_active == singles[i]["n_active"] and meshes[i].n_tris == singles[i]["n_tris"]
    batch.close()
    for net in nets:
        net.close()


def test_batch_rejects_malformed(pkg):
    ents = _entries()[:2]
    nets = [pkg.Inr(layers) for layers, _ in ents]
    ps = [dict(p) for _, p in ents]
    ps[1]["max_level"] = 11
    with pytest.raises(pkg.IsxError) as e:
        pkg.Batch(nets, ps)
    assert e.value.status == 1
    with pytest.raises(pkg.IsxError) as e:
        pkg.Batch(nets, [p for _, p in ents], workers=65)
    assert e.value.status == 1
    for net in nets:
        net.close()
