"""Train the cell-subdivision proposer on fields of the scientific kind and evaluate it on held-out
fields against plain extraction and dense extraction.

    python -m paper_2402_13861_gb300.train_proposer --fields 16 --out proposer.npz

Training fields: seeds 2000+i, 256 anisotropic Gaussians + 0.05 sin(6 pi x) sin(6 pi y) sin(6 pi z),
fitted by a 3->256x5->1 ReLU MLP; 8 iso-values over the 10-90 % quantiles; octree to 512^3.  Per
field the plain level loop (UP, k = 3, BF16) records every visited cell and its bound, dense
extraction gives the crossing cells, and (cell, iso) pairs of levels 3..9 are sampled with their
labels.  The proposer is trained with the library's kernels; tau_lo is set on held-out pairs so
that at most 2e-4 of the positive pairs fall below it.  Held-out fields (seeds 3000+i) report,
against dense extraction: missed crossing cells, bounded cells and ACP time for plain and
proposer-assisted extraction.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def _fit(seed, steps):
    from synth import fields, inr
    layers, _ = inr.fit([3] + [256] * 5 + [1], fields.anisotropic_blobs(seed, 256), steps, init_seed=seed,
                        sample_seed=seed + 1)
    isos = inr.quantile_isos(layers, 8)
    return layers, isos


def missed(active_codes, active_masks, cross):
    """Crossing (cell, iso) pairs of the dense extraction that the active set misses, and their total."""
    import torch
    key, masks = cross
    ac = active_codes.to(torch.int64) & 0xFFFFFFFF
    am = active_masks.to(torch.int64) & 0xFFFFFFFF
    have = torch.zeros_like(key)
    if ac.numel():
        order = torch.argsort(ac)
        ac, am = ac[order], am[order]
        pos = torch.searchsorted(ac, key).clamp(max=ac.numel() - 1)
        have = torch.where(ac[pos] == key, am[pos], have)
    miss = masks & ~have

    def pop(m):
        return int(sum(int(((m >> q) & 1).sum()) for q in range(32)))
    return pop(miss), pop(masks)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=16)
    ap.add_argument("--eval-fields", type=int, default=2)
    ap.add_argument("--fit-steps", type=int, default=2000)
    ap.add_argument("--max-level", type=int, default=9)
    ap.add_argument("--per-level", type=int, default=40000)
    ap.add_argument("--proposer-level", type=int, default=5)
    ap.add_argument("--out", default="proposer.npz")
    args = ap.parse_args(argv)
    import torch
    import paper_2402_13861_gb300 as pkg
    from paper_2402_13861_gb300 import proposer as gp
    torch.cuda.set_device(0)
    L = args.max_level
    log = lambda m: print(m, file=sys.stderr, flush=True)
    X, Y = [], []
    t0 = time.time()
    for i in range(args.fields):
        layers, isos = _fit(2000 + i, args.fit_steps)
        net = pkg.Inr(layers)
        levels = gp.plain_levels(net, L, isos)
        cross = gp.crossing_cells(net, L, isos)
        x, y = gp.sample_pairs(levels, cross, L, isos, 3, args.per_level, seed=i)
        X.append(x)
        Y.append(y)
        log(f"field {i}: {x.shape[0]} pairs, positive fraction {float(y.mean()):.3f}, {time.time() - t0:.0f} s")
        del levels
        net.close()
    X, Y = torch.cat(X), torch.cat(Y)
    n = X.shape[0]
    perm = torch.randperm(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    nv = n // 10
    val, tr = perm[:nv], perm[nv:]
    prop, hist = gp.train(X[tr].contiguous(), Y[tr].contiguous(), epochs=6, batch=8192, lr=2e-3, log=log)
    tau_lo, tau_hi = gp.choose_thresholds(prop, X[val].contiguous(), Y[val].contiguous())
    z = prop.predict(X[val].contiguous())
    p = torch.sigmoid(z)
    yv = Y[val]
    stats = {"train_pairs": int(n - nv), "val_pairs": int(nv), "bce_per_epoch": hist,
             "val_accuracy": float(((p > 0.5) == (yv > 0.5)).float().mean()),
             "val_decided_fraction": float(((p <= tau_lo) | (p >= tau_hi)).float().mean()),
             "tau_lo": tau_lo, "tau_hi": tau_hi}
    log(json.dumps(stats))
    np.savez(args.out, params=prop.get_params(), mean=prop.mean, std=prop.std, tau_lo=tau_lo, tau_hi=tau_hi,
             proposer_level=args.proposer_level, max_level=L, train_stats=json.dumps(stats))
    # ---- held-out fields ----
    for e in range(args.eval_fields):
        layers, isos = _fit(3000 + e, args.fit_steps)
        net = pkg.Inr(layers)
        cross = gp.crossing_cells(net, L, isos)
        kw = dict(mode="clt", k=3.0, prec="bf16")
        net.extract(L, isos, active_cap=1 << 25, tri_cap=1 << 25, **kw)           # warm-up, sizes buffers
        plain = net.extract(L, isos, active_cap=1 << 25, tri_cap=1 << 25, **kw)
        assisted = net.extract(L, isos, active_cap=1 << 25, tri_cap=1 << 25, proposer=prop,
                               proposer_level=args.proposer_level, tau_lo=tau_lo, tau_hi=tau_hi, **kw)
        dense = net.extract(L, isos, prec="fp32", dense=True, tri_cap=1 << 25)
        mp, tot = missed(plain["codes"], plain["masks"], cross)
        ma, _ = missed(assisted["codes"], assisted["masks"], cross)
        rec = {"field_seed": 3000 + e, "crossing_pairs": tot,
               "plain": {"ms_acp": plain["ms_acp"], "ms_total": plain["ms_total"],
                         "cells_bounded": int(sum(plain["cells_bounded"])), "missed_pairs": mp,
                         "missed_rate": mp / max(tot, 1), "n_active": plain["n_active"]},
               "proposer": {"ms_acp": assisted["ms_acp"], "ms_total": assisted["ms_total"],
                            "cells_bounded": int(sum(assisted["cells_bounded"])), "missed_pairs": ma,
                            "missed_rate": ma / max(tot, 1), "n_active": assisted["n_active"]},
               "dense": {"ms_total": dense["ms_total"]}}
        print(json.dumps(rec), flush=True)
        net.close()
    prop.close()


if __name__ == "__main__":
    main()
