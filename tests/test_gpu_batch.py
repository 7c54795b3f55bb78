"""Batched extraction (isx_batch_*): every entry of a level-synchronous batch gives exactly the
active cells and triangles of its own single extraction with the per-cell tensor-core bound
kernel (the same bound kernel and cull test, the same stable order), with and without CUDA-graph
replay; unsupported batches are rejected."""
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


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_extractions(pkg, use_graph, monkeypatch):
    ents = _entries()
    nets = [pkg.Inr(layers) for layers, _ in ents]
    # the batch runs the per-cell tensor-core bound kernel; single extractions take it too
    monkeypatch.setenv("ISX_BF16_ROWS", "0")
    singles = [net.extract(**p) for net, (_, p) in zip(nets, ents)]
    monkeypatch.delenv("ISX_BF16_ROWS")
    batch = pkg.Batch(nets, [p for _, p in ents], use_graph=use_graph)
    for rep in range(3):                       # sized run, then (graph) capture + replay, then replay
        res = batch.run()
        for r, s in zip(res, singles):
            _same(r, s)
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
