"""Batched extraction (isx_batch_*): a level-synchronous batch of mixed INRs bounded by the
per-cell tensor-core kernel.
- Runs are reproducible: the sized run, the graph capture and every replay give identical outputs.
- One entry is checked against the float64 oracle's extraction with per-result bands
  (tests/_rounding_model.py): its active (cell, iso) pairs equal the oracle's up to pairs with an
  ancestor-or-self endpoint within its own band of the iso-value.
- Every entry agrees with its own single extraction (the row-batched kernel) up to a small number
  of (cell, iso) pairs.
- Unsupported batches are rejected.
"""
import numpy as np
import pytest
import torch

from oracle import mlp, octree
from synth import inr

from _helpers import to_np
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
    specs = [([3, 128, 128, 128, 1], 41, 5, 2, 3.0), ([3] + [256] * 4 + [1], 42, 6, 3, 2.0),
             ([3] + [128] * 5 + [1], 43, 4, 1, 3.0), ([3, 256, 256, 1], 44, 5, 4, 3.0)]
    out = []
    for dims, seed, L, niso, k in specs:
        layers = inr.random_inr(dims, seed)
        vals = mlp.mlp_forward(layers, octree.lattice_points(16))
        isos = np.quantile(vals, np.linspace(0.3, 0.7, niso)).astype(np.float32)
        out.append((layers, dict(max_level=L, isos=isos, mode="clt", k=k, prec="bf16")))
    return out


def _same(a, b):
    assert a["n_active"] == b["n_active"] and a["n_tris"] == b["n_tris"]
    assert torch.equal(a["codes"], b["codes"]) and torch.equal(a["masks"], b["masks"])
    assert torch.equal(a["tri_edge"], b["tri_edge"]) and torch.equal(a["tri_iso"], b["tri_iso"])


def _pairs(res):
    codes = to_np(res["codes"]).astype(np.int64) & 0xFFFFFFFF
    masks = to_np(res["masks"]).astype(np.int64) & 0xFFFFFFFF
    return dict(zip(codes.tolist(), masks.tolist()))


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle_and_single_extractions(pkg, use_graph):
    ents = _entries()
    nets = [pkg.Inr(layers) for layers, _ in ents]
    singles = [net.extract(**p) for net, (_, p) in zip(nets, ents)]
    batch = pkg.Batch(nets, [p for _, p in ents], use_graph=use_graph)
    first = None
    for rep in range(3):                       # sized run, then (graph) capture + replay, then replay
        res = batch.run()
        if first is None:
            first = [dict(r, codes=r["codes"].clone(), masks=r["masks"].clone(), tri_edge=r["tri_edge"].clone(),
                          tri_iso=r["tri_iso"].clone()) for r in res]
        else:
            for r, f in zip(res, first):
                _same(r, f)
    for i, (r, s) in enumerate(zip(res, singles)):
        a, b = _pairs(r), _pairs(s)
        n = sum(bin(m).count("1") for m in a.values())
        d = sum(bin(a.get(c, 0) ^ b.get(c, 0)).count("1") for c in set(a) | set(b))
        print(f"entry {i}: {r['n_active']} active cells, {d} of {n} (cell, iso) pairs differ from the single "
              f"extraction")
        assert d <= max(4, 0.01 * n)
    if use_graph:
        # entry 0 (3 -> 128 x 3 -> 1, 32^3, 2 isos, UP k = 3) against the oracle
        layers, p = ents[0]
        check_extraction_pairs(layers, p["isos"], p["max_level"], res[0], "clt", p["k"], "batch entry 0")
    print("active cells per entry:", [r["n_active"] for r in res], "level loop ms", res[0]["ms_acp"])
    batch.close()
    for net in nets:
        net.close()


def test_batch_rejects_unsupported(pkg):
    ents = _entries()[:2]
    nets = [pkg.Inr(layers) for layers, _ in ents]
    ps = [dict(p) for _, p in ents]
    ps[1]["mode"] = "sound"
    with pytest.raises(pkg.IsxError) as e:
        pkg.Batch(nets, ps)
    assert e.value.status == 1
    ps = [dict(p) for _, p in ents]
    ps[0]["prec"] = "fp32"
    with pytest.raises(pkg.IsxError) as e:
        pkg.Batch(nets, ps)
    assert e.value.status == 5
    small = pkg.Inr(inr.random_inr([3, 64, 64, 1], 1))
    with pytest.raises(pkg.IsxError) as e:
        pkg.Batch([small], [dict(max_level=3, isos=[0.0], mode="clt", prec="bf16")])
    assert e.value.status == 5
    for net in nets + [small]:
        net.close()
