"""Training data, training loop and decision thresholds of the cell-subdivision proposer.

The proposer (``Proposer``, C interface ``isx_proposer_*``) is an addition to the paper's method,
whose Algorithm 1 decides by range analysis alone.  Its labels are produced by the method itself:
- dense extraction (``isx_extract_dense``) gives the finest cells crossed by each iso-surface (the
  cells where marching cubes emits a triangle);
- a (cell, iso) pair is positive iff the cell's subtree holds such a cell.
Its features use the bounds of the plain level loop, read from the library's record of it
(``isx_level_record``: visited cells, inherited masks and bounds per level).  Training runs the library's forward, backward
and Adam kernels (``isx_proposer_train_step``).  Everything here is data plumbing in PyTorch:
index arithmetic on cell codes (ancestor lookups), sampling and bookkeeping; the cull test and
the subdivision run in the library only.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib

NPARAM = _lib.PROPOSER_NPARAM
DIMS = (8, 64, 64, 64, 1)


def he_params(seed):
    """Packed He-normal initial parameters (std sqrt(2 / fan_in), zero biases)."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in zip(DIMS[:-1], DIMS[1:]):
        out.append(rng.normal(0.0, math.sqrt(2.0 / fi), size=fo * fi))
        out.append(np.zeros(fo))
    return np.concatenate(out).astype(np.float32)


def unpack(params):
    """Packed vector -> [(W, b)] with W row-major [out][in]."""
    params = np.asarray(params, dtype=np.float64)
    layers, o = [], 0
    for fi, fo in zip(DIMS[:-1], DIMS[1:]):
        W = params[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = params[o:o + fo]
        o += fo
        layers.append((W, b))
    return layers


def pack(layers):
    return np.concatenate([np.concatenate([np.asarray(W).reshape(-1), np.asarray(b).reshape(-1)])
                           for W, b in layers]).astype(np.float32)


# ---- cell codes (i | j << 10 | k << 20) -------------------------------------------------------------
def split_codes(codes):
    return codes & 1023, (codes >> 10) & 1023, (codes >> 20) & 1023


def join_codes(i, j, k):
    return i | (j << 10) | (k << 20)


def plain_levels(net, L, isos, mode="clt", k=3.0, prec="bf16"):
    """The plain level loop of Algorithm 1 as the library runs it (isx_extract_isosurface with its
    level record): per level a dict with the visited cells' codes (sorted), the iso masks they
    inherited from their parents, and their bounds (centre, spread)."""
    import torch
    res = net.extract(L, isos, mode=mode, k=k, prec=prec, record=True, active_cap=1 << 22, tri_cap=1 << 24,
                      record_cap=1 << 24)
    out = []
    for lv in res["levels"]:
        codes = lv["codes"].to(torch.int64) & 0xFFFFFFFF
        order = torch.argsort(codes)
        out.append({"codes": codes[order], "masks": (lv["masks"].to(torch.int64) & 0xFFFFFFFF)[order],
                    "centre": lv["centre"][order], "spread": lv["spread"][order]})
    return out


def crossing_cells(net, L, isos, prec="fp32"):
    """(codes, masks) of the finest cells where dense marching cubes emits a triangle, per iso: the
    list isx_extract_dense writes (codes in cell order, mask bit q = the cell has a triangle of iso q)."""
    import torch
    res = net.extract(L, isos, prec=prec, dense=True, active_cap=1 << 22, tri_cap=1 << 24)
    codes = res["codes"].to(torch.int64) & 0xFFFFFFFF
    order = torch.argsort(codes)
    return codes[order], (res["masks"].to(torch.int64) & 0xFFFFFFFF)[order]


def ancestor_table(cross_codes, cross_masks, L, level):
    """Sorted ancestor codes at `level` of the crossing cells with the OR of their masks."""
    import torch
    s = L - level
    i, j, k = split_codes(cross_codes)
    anc = join_codes(i >> s, j >> s, k >> s)
    key, inv = torch.unique(anc, return_inverse=True)
    m = torch.zeros_like(key)
    for q in range(32):
        sel = ((cross_masks >> q) & 1) != 0
        if not sel.any():
            continue
        hit = torch.zeros_like(key, dtype=torch.bool)
        hit[inv[sel]] = True
        m[hit] |= 1 << q
    return key, m


def lookup(sorted_codes, values, query):
    """values at the positions of `query` in `sorted_codes` (every query must be present)."""
    import torch
    pos = torch.searchsorted(sorted_codes, query)
    pos = pos.clamp(max=sorted_codes.numel() - 1)
    assert bool((sorted_codes[pos] == query).all()), "ancestor not visited"
    return values[pos]


def features(codes, level, iso, anc_c, anc_s, gap):
    """The 8 feature rows (float32 [n, 8]) of (cell, iso) pairs."""
    import torch
    i, j, k = split_codes(codes)
    h = 2.0 ** (-level)
    ctr = [(-1.0 + (2 * t.to(torch.float32) + 1.0) * h) for t in (i, j, k)]
    n = codes.numel()
    lev = torch.full((n,), -float(level), device=codes.device)
    return torch.stack(ctr + [lev, iso, anc_c - iso, anc_s, gap.to(torch.float32)], dim=1).contiguous()


def sample_pairs(levels, cross, L, isos, min_level, per_level, seed, max_gap=3):
    """Feature rows and labels of (cell, iso) pairs sampled from the visited cells of levels
    min_level..L; ancestor gap uniform in 1..max_gap."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    iso_t = torch.tensor(np.asarray(isos, dtype=np.float32), device="cuda")
    X, Y = [], []
    for level in range(max(1, min_level), L + 1):
        rec = levels[level]
        n = rec["codes"].numel()
        if n == 0:
            continue
        m = min(per_level, n)
        idx = torch.randint(0, n, (m,), device="cuda", generator=g)
        codes, masks = rec["codes"][idx], rec["masks"][idx]
        # one random iso of the cell's mask
        r = torch.rand(m, len(isos), device="cuda", generator=g) * (((masks[:, None] >> torch.arange(
            len(isos), device="cuda")) & 1).to(torch.float32))
        q = r.argmax(dim=1)
        ok = r.max(dim=1).values > 0
        codes, q = codes[ok], q[ok]
        gap = torch.randint(1, min(max_gap, level) + 1, (codes.numel(),), device="cuda", generator=g)
        anc_c = torch.empty(codes.numel(), device="cuda")
        anc_s = torch.empty_like(anc_c)
        for gg in range(1, min(max_gap, level) + 1):
            sel = gap == gg
            if not sel.any():
                continue
            i, j, k = split_codes(codes[sel])
            a = join_codes(i >> gg, j >> gg, k >> gg)
            up = levels[level - gg]
            anc_c[sel] = lookup(up["codes"], up["centre"], a)
            anc_s[sel] = lookup(up["codes"], up["spread"], a)
        key, lm = ancestor_table(cross[0], cross[1], L, level)
        if key.numel():
            pos = torch.searchsorted(key, codes).clamp(max=key.numel() - 1)
            lab = torch.where(key[pos] == codes, (lm[pos] >> q) & 1, torch.zeros_like(q)).to(torch.float32)
        else:
            lab = torch.zeros(codes.numel(), device="cuda")
        X.append(features(codes, level, iso_t[q], anc_c, anc_s, gap))
        Y.append(lab)
    return torch.cat(X), torch.cat(Y)


def train(feat, label, epochs=4, batch=8192, lr=2e-3, seed=0, log=None):
    """A Proposer trained with the library's kernels on (feat [n, 8], label [n]) CUDA tensors."""
    import torch
    mean = feat.mean(dim=0).cpu().numpy()
    std = feat.std(dim=0).clamp(min=1e-6).cpu().numpy()
    prop = _lib.Proposer(he_params(seed), mean, std)
    g = torch.Generator(device="cuda").manual_seed(seed)
    n = feat.shape[0]
    loss = torch.zeros(1, device="cuda")
    hist = []
    steps = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, nb = torch.zeros(1, device="cuda"), 0
        for a in range(0, n - batch + 1, batch):
            sel = perm[a:a + batch]
            step_lr = lr * 0.5 * (1 + math.cos(math.pi * steps / max(1, epochs * (n // batch))))
            prop.train_step(feat[sel].contiguous(), label[sel].contiguous(), step_lr, loss=loss)
            tot += loss
            nb += 1
            steps += 1
        hist.append(float(tot) / max(nb, 1))
        if log:
            log(f"epoch {ep}: mean BCE {hist[-1]:.4f}")
    return prop, hist


def choose_thresholds(prop, feat, label, miss=2e-4):
    """tau_lo: the largest probability with at most `miss` of the positive pairs at or below it;
    tau_hi: 0.5 (a kept negative costs only extra work, never a miss)."""
    import torch
    z = prop.predict(feat)
    p = torch.sigmoid(z)
    pos = p[label > 0.5]
    if pos.numel() == 0:
        return 0.01, 0.5
    lo = float(torch.quantile(pos.float(), miss)) if pos.numel() > 10 else 0.0
    return max(0.0, min(lo, 0.49)), 0.5


def load(path):
    """(Proposer, metadata) from an .npz written by train_proposer: the parameters, the feature
    standardisation and the decision settings (tau_lo, tau_hi, proposer_level)."""
    z = np.load(path)
    prop = _lib.Proposer(z["params"], z["mean"], z["std"])
    meta = {"tau_lo": float(z["tau_lo"]), "tau_hi": float(z["tau_hi"]), "proposer_level": int(z["proposer_level"])}
    return prop, meta
