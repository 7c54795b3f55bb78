"""Training data, training loop and decision thresholds of the cell-subdivision proposer.

The proposer (``Proposer``, C interface ``isx_proposer_*``) is an addition to the paper's method,
whose Algorithm 1 decides by range analysis alone.  Its labels are produced by the method itself:
- dense extraction (``isx_extract_dense``) gives the finest cells crossed by each iso-surface (the
  cells where marching cubes emits a triangle);
- a (cell, iso) pair is positive iff the cell's subtree holds such a cell.
Its features use the bounds of a plain level-by-level pass (``isx_bound_cells`` on the visited
cells, the same bound the extraction computes).  Training runs the library's forward, backward
and Adam kernels (``isx_proposer_train_step``).  Everything here is data plumbing in PyTorch:
index arithmetic on cell codes, sampling and bookkeeping.
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


def boxes(codes, level):
    import torch
    i, j, k = split_codes(codes)
    ijk = torch.stack([i, j, k], dim=1).to(torch.float32)
    size = 2.0 / (1 << level)
    lo = (-1.0 + size * ijk).contiguous()
    return lo, (lo + size).contiguous()


def children(codes):
    import torch
    i, j, k = split_codes(codes)
    out = []
    for c in range(8):
        out.append(join_codes(2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1)))
    return torch.stack(out, dim=1).reshape(-1)


def cull_bits(centre, spread, isos, mode, k):
    """Iso bitmask kept by a bound (the cull test of Algorithm 1, closed interval)."""
    import torch
    if mode == "sound":
        lo, hi = centre - spread, centre + spread
    else:
        lo, hi = centre - k * spread, centre + k * spread
    bits = torch.zeros_like(centre, dtype=torch.int64)
    for q, c in enumerate(isos):
        bits |= ((lo <= float(c)) & (float(c) <= hi)).to(torch.int64) << q
    bits[~(lo <= hi)] = (1 << len(isos)) - 1
    return bits


def plain_levels(net, L, isos, mode="clt", k=3.0, prec="bf16", chunk=1 << 21):
    """The plain level loop, keeping every level: per level a dict with the visited cells' codes
    (sorted), their parent masks, and (for levels < L) their bound.  Level L is visited but not
    bounded (its cells' features need only their ancestors' bounds)."""
    import torch
    dev = torch.device("cuda")
    full = (1 << len(isos)) - 1
    codes = torch.zeros(1, dtype=torch.int64, device=dev)
    masks = torch.full((1,), full, dtype=torch.int64, device=dev)
    out = []
    for level in range(L + 1):
        order = torch.argsort(codes)
        codes, masks = codes[order], masks[order]
        rec = {"codes": codes, "masks": masks}
        if level == L:
            out.append(rec)
            break
        c = torch.empty(codes.numel(), dtype=torch.float32, device=dev)
        s = torch.empty_like(c)
        for a in range(0, codes.numel(), chunk):
            lo, hi = boxes(codes[a:a + chunk], level)
            net.bound_cells(lo, hi, mode=mode, prec=prec, center=c[a:a + chunk], spread=s[a:a + chunk])
        rec["centre"], rec["spread"] = c, s
        out.append(rec)
        keep = masks & cull_bits(c, s, isos, mode, k)
        alive = keep != 0
        codes = children(codes[alive])
        masks = keep[alive].repeat_interleave(8)
    return out


def crossing_cells(net, L, isos, prec="fp32"):
    """(codes, masks) of the finest cells where dense marching cubes emits a triangle, per iso."""
    import torch
    res = net.extract(L, isos, prec=prec, dense=True, tri_cap=1 << 22)
    cell = res["tri_cell"].to(torch.int64) & 0xFFFFFFFF
    tiso = res["tri_iso"].to(torch.int64)
    key = torch.unique(cell)
    masks = torch.zeros_like(key)
    for q in range(len(isos)):
        kq = torch.unique(cell[tiso == q])
        if kq.numel():
            masks[torch.searchsorted(key, kq)] |= 1 << q
    return key, masks


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
