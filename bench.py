#!/usr/bin/env python
"""Benchmark: hierarchical iso-surface extraction at 512^3 on the scientific-field workload.

One step = one full extraction through the C interface (isx_extract_isosurface): every octree
level from the root to 512^3 bounded by propagating affine / probabilistic-affine forms through the
3 -> 256 (5 hidden) -> 1 ReLU INR, culling, compaction, corner evaluation of the active cells and
marching cubes for the 8 iso-values.  `value` is AA-bounded cells per second over the timed steps
(cells bounded, summed over levels, divided by extraction time); `ms_per_step` is the extraction
time.  Between steps a 512 MB buffer is written to flush the L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank extracts its own INR replica (independent problems; no
collective on the data path); value = cells bounded on all ranks / max time over ranks.
--impl reference times the float64 CPU oracle on a bounded sample of the same workload (cells of
levels 6-9 drawn at random), on rank 0 only; there `ms_per_step` is the wall time of one sample.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "scientific"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="clt", choices=["sound", "clt", "raua"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--k", type=float, default=3.0)
    ap.add_argument("--eval-prec", default="auto", choices=["auto", "fp32", "bf16"],
                    help="corner evaluation: bf16 = tensor cores with two-term bf16 operands (float32-class)")
    ap.add_argument("--max-level", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--all-forms", action="store_true",
                    help="also the slow forms: RA-Fixed, the SIREN workload (fits a SIREN), the large network at "
                         "1024^3 and the 64-entry batch; the default run keeps the quick ones")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = None
        self.f = None
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        self.f = os.fdopen(fd, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            if self.f is not None:
                self.f.close()
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def traffic_record(kernel, src_file):
    """The ncu DRAM record of `kernel` in profiles/traffic.json (from a capture of a smaller launch of
    the same kernel), if the kernel source is unchanged since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        sha = hashlib.sha256(open(src_file, "rb").read()).hexdigest()[:16]
        return rec if rec.get("src_sha") == sha else None
    except Exception:
        return None


def extraction_forms(pkg, net, L, isos, plain, plain_ms, mode, k, prec, slow=False):
    """End-to-end time of the other extraction forms on the same INR and isos, and the crossing
    (cell, iso) pairs of the dense extraction each form misses: the per-cell tensor-core bound kernel,
    bounding stopped at level 6, the proposer-assisted form (committed proposer), dense extraction
    (FP32 and tensor-core evaluation), sound RA-Fixed bounds, and the k-d tree against the octree
    one level lower (tensor-core corner values throughout).  Each form runs once after a warm-up of
    the same call."""
    import torch
    from paper_2402_13861_gb300 import proposer as gp
    from paper_2402_13861_gb300.train_proposer import missed
    st = torch.cuda.current_stream()
    bufs = {}

    def timed_level(level, reps=2, **kw):
        for rep in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            r = net.extract(level, isos, buffers=bufs, active_cap=1 << 27, tri_cap=1 << 25, **kw)
            b.record(st)
            torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    def timed(reps=2, **kw):
        return timed_level(L, reps=reps, **kw)

    dense32, ms_d32 = timed(prec="fp32", dense=True)
    # the dense extraction's crossing cells (cells with a triangle, per iso), as the library lists them
    key = dense32["codes"].to(torch.int64) & 0xFFFFFFFF
    order = torch.argsort(key)
    cross = (key[order], (dense32["masks"].to(torch.int64) & 0xFFFFFFFF)[order])
    out = {}
    mp, tot = missed(plain["codes"], plain["masks"], cross)
    out["plain"] = {"ms": plain_ms, "cells_bounded": int(sum(plain["cells_bounded"])), "missed_pairs": mp,
                    "missed_rate": mp / max(tot, 1)}
    # sound affine arithmetic (row-batched BF16): without inflation, and with the rounding-error
    # inflation, whose FNR is 0 by construction, so it must miss no crossing pair (timed once: its
    # error symbols make it the slowest form)
    r, ms = timed(mode="sound", prec=prec, eval_prec="bf16")
    m, _ = missed(r["codes"], r["masks"], cross)
    out["sound_bf16"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])),
                         "cells_per_s": sum(r["cells_bounded"]) / (ms / 1e3), "n_active": r["n_active"],
                         "missed_pairs": m, "missed_rate": m / max(tot, 1)}
    r, ms = timed(reps=1, mode="sound", prec=prec, inflate=True, eval_prec="bf16")
    m, _ = missed(r["codes"], r["masks"], cross)
    out["sound_bf16_inflated"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])),
                                  "cells_per_s": sum(r["cells_bounded"]) / (ms / 1e3), "n_active": r["n_active"],
                                  "missed_pairs": m, "missed_rate": m / max(tot, 1), "timed_runs": 1}
    # the confidence multiplier k of the Gaussian read-off (Algorithm 1's t): miss rate against work
    for kk in (2.0, 4.0):
        r, ms = timed(mode=mode, k=kk, prec=prec, eval_prec="bf16")
        m, _ = missed(r["codes"], r["masks"], cross)
        out[f"{mode}_k{int(kk)}"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])),
                                     "n_active": r["n_active"], "missed_pairs": m, "missed_rate": m / max(tot, 1)}
    # bound_stop_level: bound down to level s, keep every descendant of the survivors, evaluate densely
    # inside them (tensor-core corner values); s = max_level is the plain form
    out["stop_level"] = {}
    for stop in range(4, L):
        r, ms = timed(mode=mode, k=k, prec=prec, bound_stop_level=stop, eval_prec="bf16")
        m, _ = missed(r["codes"], r["masks"], cross)
        out["stop_level"][str(stop)] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])),
                                        "n_active": r["n_active"], "n_points": r["n_points"], "missed_pairs": m,
                                        "missed_rate": m / max(tot, 1)}
    out["stop_level"][str(L)] = {"ms": plain_ms, "cells_bounded": int(sum(plain["cells_bounded"])),
                                 "missed_rate": out["plain"]["missed_rate"]}
    out["bound_to_level6_tc_eval"] = dict(out["stop_level"]["6"])
    prop, meta = gp.load(os.path.join(ROOT, "synth", "data", "proposer.npz"))
    r, ms = timed(mode=mode, k=k, prec=prec, eval_prec="bf16", proposer=prop, proposer_level=meta["proposer_level"],
                  tau_lo=meta["tau_lo"], tau_hi=meta["tau_hi"])
    m, _ = missed(r["codes"], r["masks"], cross)
    out["proposer"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])), "missed_pairs": m,
                       "missed_rate": m / max(tot, 1), **meta}
    prop.close()
    _, ms_dtc = timed(prec="fp32", dense=True, eval_prec="bf16")
    out["dense_fp32_eval"] = {"ms": ms_d32, "crossing_pairs": tot}
    out["dense_tc_eval"] = {"ms": ms_dtc}
    # the reduced range-analysis baseline: sound RA-Fixed bounds (one fused float32 kernel)
    if slow:
        r, ms = timed(mode="rafixed", prec="fp32")
        m, _ = missed(r["codes"], r["masks"], cross)
        out["rafixed_fp32"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])), "n_active": r["n_active"],
                               "missed_pairs": m, "missed_rate": m / max(tot, 1)}
    # Algorithm 1's k-d tree (widest-side bisection) against the octree, one level lower (256^3)
    for name, kd in (("octree_256", False), ("kd_tree_256", True)):
        r, ms = timed_level(L - 1, mode=mode, k=k, prec=prec, eval_prec="bf16", kd_tree=kd)
        out[name] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])), "n_active": r["n_active"]}
    return out


def batched_form(pkg, mode, k, workers=8, full=False):
    """The batched form: extractions of mixed shape in flight together.  Networks of hidden width
    64 / 128 / 256 are each fitted for 300 Adam steps to their own field of the scientific kind
    (anisotropic Gaussians + sine) and give 4 entries each (own INR handle), 16 iso-values over the
    10-90 % or 20-80 % quantiles.  Default: 8 networks (3-6 hidden layers, 32-256 Gaussians), octrees
    to 128^3 and 256^3, 32 entries.  `full` (the batched configuration's shape): 16 networks (3-8 hidden
    layers, 16-512 Gaussians), octrees to 128^3, 256^3 and, for widths 64 and 128, 512^3, 64 entries;
    it takes about four minutes, most of it fitting.  Reports the extractions run one after another (a
    batch with one worker) and together (`workers` worker streams), and checks that every entry's mesh
    is the same."""
    import torch
    from synth import fields, inr
    if full:
        specs = [(64, 3, 16), (64, 4, 24), (64, 5, 48), (64, 6, 40), (64, 8, 96), (128, 3, 32), (128, 4, 64),
                 (128, 5, 160), (128, 6, 128), (128, 8, 192), (256, 3, 64), (256, 4, 128), (256, 5, 256),
                 (256, 6, 384), (256, 7, 320), (256, 8, 512)]
    else:
        specs = [(64, 3, 32), (128, 3, 64), (256, 3, 128), (64, 5, 48), (128, 4, 96), (256, 4, 160), (128, 6, 192),
                 (256, 5, 256)]
    nets, params, shapes = [], [], []
    for i, (w, H, nb) in enumerate(specs):
        layers, _ = inr.fit([3] + [w] * H + [1], fields.anisotropic_blobs(4000 + i, nb), 300, init_seed=4000 + i,
                            sample_seed=5000 + i)
        top = 9 if full and w <= 128 else 8
        for j, (L, lo_q, hi_q) in enumerate(((7, 0.1, 0.9), (7, 0.2, 0.8), (8, 0.1, 0.9), (top, 0.2, 0.8))):
            isos = inr.quantile_isos(layers, 16, lo_q=lo_q, hi_q=hi_q, grid=64)
            nets.append(pkg.Inr(layers))
            params.append(dict(max_level=L, isos=isos, mode=mode, k=k, prec="bf16",
                               eval_prec="bf16" if w in (128, 256) else "fp32"))
            shapes.append(f"w{w}xH{H}@{1 << L}^3")
    st = torch.cuda.current_stream()

    def ev_ms(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        out = fn()
        b.record(st)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    # one after another: the same entries on one worker (one workspace); then on `workers` workers
    seq = pkg.Batch(nets, params, workers=1)
    seq.run(active_cap=1 << 21, tri_cap=1 << 23)                              # sizes the buffers
    singles, seq_ms = ev_ms(lambda: seq.run(active_cap=1 << 21, tri_cap=1 << 23))
    singles = [(s["n_active"], s["n_tris"]) for s in singles]
    seq.close()
    batch = pkg.Batch(nets, params, workers=workers)
    batch.run(active_cap=1 << 21, tri_cap=1 << 23)
    res, batch_ms = ev_ms(lambda: batch.run(active_cap=1 << 21, tri_cap=1 << 23))
    same = all((r["n_active"], r["n_tris"]) == s for r, s in zip(res, singles))
    cells = int(sum(sum(r["cells_bounded"]) for r in res))
    batch.close()
    for net in nets:
        net.close()
    return {"entries": len(nets), "shapes": shapes, "isos_each": 16, "workers": workers,
            "sequential_ms": seq_ms, "batch_ms": batch_ms, "speedup": seq_ms / batch_ms, "same_meshes": bool(same),
            "cells_bounded": cells, "batch_cells_per_s": cells / (batch_ms / 1e3)}


def large_form(pkg, full=False):
    """The large configuration: a 3 -> 512 x 8 -> 1 ReLU INR fitted to 1024 anisotropic Gaussians (seed 5;
    committed fixture), one iso-value midway between the 10 % and 90 % quantiles.  BF16 row-batched
    bounds at 512^3 (with `full`, also 1024^3): sound affine arithmetic, whose launch accounting gives the
    row GEMM's bandwidth and the split GEMM's tensor-core rate at width 512, and UP with k = 2, 3, 4, whose
    active pairs are counted against the sound form's (sound bounds miss no crossing cell up to BF16
    rounding; there is no dense tensor-core reference at width 512)."""
    import torch
    from synth import inr
    from paper_2402_13861_gb300.train_proposer import missed
    t0 = time.time()
    layers, isos, wl = inr.load_inr("large")
    fit_s = time.time() - t0
    net = pkg.Inr(layers)
    st = torch.cuda.current_stream()
    bufs = {}
    out = {"dims": wl.dims, "load_or_fit_s": fit_s, "n_iso": int(len(isos))}

    def run(level, reps=1, **kw):
        pkg.profile_reset()
        pkg.profile_enable(True)
        for rep in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            r = net.extract(level, isos, buffers=bufs, prec="bf16", eval_prec="fp32", active_cap=1 << 27,
                            tri_cap=1 << 26, **kw)
            b.record(st)
            torch.cuda.synchronize()
        pkg.profile_enable(False)
        return r, a.elapsed_time(b), pkg.profile_read()

    for L in ((9, 10) if full else (9,)):
        ref, ms_s, stats = run(L, reps=2 if L < 10 else 1, mode="sound")
        key = ref["codes"].to(torch.int64) & 0xFFFFFFFF
        o = torch.argsort(key)
        cross = (key[o], (ref["masks"].to(torch.int64) & 0xFFFFFFFF)[o])
        e = {"ms": ms_s, "cells_bounded": int(sum(ref["cells_bounded"])),
             "cells_per_s": sum(ref["cells_bounded"]) / (ms_s / 1e3), "n_active": ref["n_active"],
             "n_tris": ref["n_tris"]}
        g, sp = stats.get("rows_gemm"), stats.get("rows_split")
        if g and g["ms"] > 0:
            e["rows_gemm_gbs"] = g["bytes"] / (g["ms"] / 1e3) / 1e9
            e["rows_gemm_tflops"] = g["flops"] / (g["ms"] / 1e3) / 1e12
        if sp and sp["ms"] > 0:
            e["rows_split_tflops"] = sp["flops"] / (sp["ms"] / 1e3) / 1e12
        tot_ms = sum(v["ms"] for v in stats.values()) or 1.0
        e["kernel_time_share"] = {k: round(v["ms"] / tot_ms, 4) for k, v in stats.items() if v["ms"] > 0.01 * tot_ms}
        res = {"sound": e}
        for kk in (2.0, 3.0, 4.0):
            r, ms, _ = run(L, mode="clt", k=kk)
            m, tot = missed(r["codes"], r["masks"], cross)
            res[f"clt_k{int(kk)}"] = {"ms": ms, "cells_bounded": int(sum(r["cells_bounded"])),
                                      "cells_bounded_per_level": r["cells_bounded"], "n_active": r["n_active"],
                                      "missed_vs_sound": m, "missed_rate_vs_sound": m / max(tot, 1)}
        out[f"{1 << L}^3"] = res
    net.close()
    return out


def activation_forms(pkg, k, names=("siren", "sdf_elu")):
    """The SIREN (sine, Table VII's sine row) and ELU-SDF workloads at 512^3: hierarchical CLT
    extraction on the tensor cores against dense extraction (FP32 evaluation), the crossing
    (cell, iso) pairs the hierarchy misses, and the fit that made each network."""
    import torch
    from synth import inr
    from paper_2402_13861_gb300.train_proposer import missed
    st = torch.cuda.current_stream()
    out = {}
    for name in names:
        t0 = time.time()
        layers, isos, wl = inr.load_inr(name, device="cuda")
        fit_s = time.time() - t0
        net = pkg.Inr(layers, act=wl.act)
        L = wl.max_level
        bufs = {}

        def timed(**kw):
            for rep in range(2):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                r = net.extract(L, isos, buffers=bufs, active_cap=1 << 27, tri_cap=1 << 25, **kw)
                b.record(st)
                torch.cuda.synchronize()
            return r, a.elapsed_time(b)

        dense, ms_d = timed(prec="fp32", dense=True)
        key = dense["codes"].to(torch.int64) & 0xFFFFFFFF
        order = torch.argsort(key)
        masks = (dense["masks"].to(torch.int64) & 0xFFFFFFFF)[order]
        h, ms_h = timed(mode="clt", k=k, prec="bf16")
        m, tot = missed(h["codes"], h["masks"], (key[order], masks))
        out[name] = {"activation": wl.act, "dims": wl.dims, "n_iso": int(len(isos)), "max_level": L,
                     "fit_s": fit_s, "hier_clt_bf16_ms": ms_h, "cells_bounded": int(sum(h["cells_bounded"])),
                     "n_active": h["n_active"], "n_tris": h["n_tris"], "dense_fp32_ms": ms_d,
                     "dense_tris": dense["n_tris"], "missed_pairs": m, "missed_rate": m / max(tot, 1)}
        net.close()
    return out


def _oracle_rate(mode, budget_s):
    """(cells, seconds) of the float64 oracle bounding random cells of levels 6-9 of the scientific
    network for about budget_s (numpy's matrix products are the only library calls)."""
    from oracle import affine
    from synth import boxes, inr
    layers = inr.load_inr(WORKLOAD)[0]
    ijk, level, lo, hi = boxes.random_cubes(4096, 77, 6, 9)
    done = 0
    t0 = time.perf_counter()
    bs = 16
    while time.perf_counter() - t0 < budget_s and done < 4096:
        affine.bound(layers, lo[done:done + bs], hi[done:done + bs], mode, batch=bs)
        done += bs
    return done, time.perf_counter() - t0


def cpu_baseline(layers, mode, k, budget_s=8.0, single_thread=True):
    """Float64 oracle bounding random cells of levels 6-9 of the same workload: on all host cores (numpy's
    BLAS threads left at their default, the main value) and, in a child process with one BLAS thread,
    single-threaded."""
    done, dt = _oracle_rate(mode, budget_s)
    cores = os.cpu_count() or 1
    single = None
    try:
        if not single_thread:
            raise RuntimeError("not measured in this run")
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
                f"d, t = bench._oracle_rate({mode!r}, {budget_s}); print(json.dumps([d, t]))")
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        d1, t1 = json.loads(out.stdout.strip().splitlines()[-1])
        single = {"value": d1 / t1, "unit": "cells/s", "cores": 1,
                  "sample": f"{d1} random cells of levels 6-9 in {t1:.1f} s, one BLAS thread"}
    except Exception as ex:                       # the single-thread figure never costs the bench line
        single = {"error": repr(ex)}
    return {"value": done / dt, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS", "default (all cores)"),
            "sample": f"{done} random cells of levels 6-9 bounded by the float64 oracle ({mode}) in {dt:.1f} s",
            "single_thread": single}


def precision_sample(net, mode, n=200000):
    """AA-bounded cells/s of the float32 path against the BF16 row path on the same cells (random cubes
    of levels 6-9, the levels that hold 99 % of the bounded cells at 512^3): the float32 path keeps
    every symbol row, so a full 512^3 extraction in float32 would take minutes."""
    import torch
    from synth import boxes
    _, _, lo, hi = boxes.random_cubes(n, 91, 6, 9)
    lo, hi = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    st = torch.cuda.current_stream()
    out = {"cells": n, "sample": f"{n} random cubes of levels 6-9"}
    for prec in ("bf16", "fp32"):
        for rep in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            net.bound_cells(lo, hi, mode=mode, prec=prec)
            b.record(st)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[prec] = {"ms": ms, "cells_per_s": n / (ms / 1e3)}
    out["bf16_over_fp32"] = out["bf16"]["cells_per_s"] / out["fp32"]["cells_per_s"]
    return out


# kernels whose accounted FLOPs run on the tensor cores
TENSOR_KERNELS = {"rows_gemm", "rows_split", "bound_tc", "eval_tc", "prop_gate", "prop_forward", "prop_grad"}
# ... and those of them that issue three bf16 products per algorithmic one (two-term operands)
SPLIT_KERNELS = {"rows_split", "eval_tc"}


def kernel_rooflines(stats, hbm_peak, tc_peak, alu_peak, top=5):
    """Rooflines of the `top` kernels by time, from the library's launch accounting (algorithmic
    bytes and FLOPs of every launch, CUDA-event time on the launching stream): HBM-bound when bytes
    are counted and the FLOPs per byte lie below the ridge of the kernel's compute peak, else
    against the tensor-core peak (tensor-core kernels) or the FP32 issue rate (the others).  A
    kernel without counted bytes or FLOPs gets no bound."""
    total = sum(v["ms"] for v in stats.values()) or 1.0
    out = []
    for name, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"])[:top]:
        e = {"kernel": name, "share": round(v["ms"] / total, 4), "launches": int(v["launches"]), "bound": None}
        secs = v["ms"] / 1e3
        fl, by = float(v["flops"]), float(v["bytes"])
        comp_peak = tc_peak if name in TENSOR_KERNELS else alu_peak
        if secs > 0 and by > 0 and (fl == 0 or (fl / by) * hbm_peak / 1e3 < comp_peak):
            e.update(bound="hbm", unit="GB/s", achieved=by / secs / 1e9, peak=hbm_peak)
        elif secs > 0 and fl > 0:
            e.update(bound="tensor" if name in TENSOR_KERNELS else "alu", unit="TFLOP/s",
                     achieved=fl / secs / 1e12, peak=comp_peak)
            if name in SPLIT_KERNELS:
                e["note"] = "three bf16 products per algorithmic one"
        if e["bound"] is not None:
            e["frac"] = e["achieved"] / e["peak"]
        out.append(e)
    return out


def job_totals(total_ms, cells, world, device):
    """Whole-job totals of a replicas-only run: the slowest rank's time (max over ranks) and the
    cells bounded by all ranks (sum), through the initialised process group when world > 1."""
    import torch
    import torch.distributed as dist
    if world <= 1:
        return float(total_ms), float(cells)
    tmax = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    csum = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(csum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(csum[0])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import inr
    layers, isos, wl = inr.load_inr(WORKLOAD)
    mode = args.mode
    per, wall_ms = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(layers, mode, args.k, budget_s=8.0 if s >= args.warmup else 2.0, single_thread=False)
        if s >= args.warmup:
            per.append(cb["value"])
            wall_ms.append(1e3 * (time.perf_counter() - t0))
    value = statistics.mean(per)
    line = {"impl": "reference", "metric": "AA-bounded cells/s (hierarchical iso-extraction, 512^3, 8 isos)",
            "value": value, "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(wall_ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "scientific-field 512^3, 3->256x5->1 ReLU INR, 8 isos",
                                            "mode": mode, "k": args.k},
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2402_13861_gb300 as pkg
    from synth import inr

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    # weights: committed fixture or per-box cache (rank 0 fits if needed)
    if rank == 0:
        layers, isos, wl = inr.load_inr(WORKLOAD)
    if world > 1:
        dist.barrier()
    if rank != 0:
        layers, isos, wl = inr.load_inr(WORKLOAD)
    L = args.max_level if args.max_level is not None else wl.max_level
    prec = args.prec
    net = pkg.Inr(layers)
    if prec == "auto":
        prec = "bf16" if pkg._lib.load() and _bf16_ok(net, pkg) else "fp32"
    eval_prec = args.eval_prec if args.eval_prec != "auto" else ("bf16" if prec == "bf16" else "fp32")
    kw = dict(mode=args.mode, k=args.k, prec=prec, inflate=(args.mode == "sound"), eval_prec=eval_prec)
    bufs = {}
    res = net.extract(L, isos, buffers=bufs, active_cap=1 << 22, tri_cap=1 << 24, **kw)   # sizes the buffers
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(0, args.warmup - 1)):
        flush.zero_()
        net.extract(L, isos, buffers=bufs, **kw)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    pkg.profile_reset()
    pkg.profile_enable(True)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    total_ms, cells, phases = 0.0, 0, np.zeros(3)
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        res = net.extract(L, isos, buffers=bufs, **kw)
        b.record(st)
        torch.cuda.synchronize()
        total_ms += a.elapsed_time(b)
        cells += sum(res["cells_bounded"])
        phases += [res["ms_acp"], res["ms_inr"], res["ms_mc"]]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    pkg.profile_enable(False)
    stats = pkg.profile_read()
    cells_local = cells
    total_ms, cells = job_totals(total_ms, cells, world, "cuda")
    value = cells / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # end to end through the public API with host buffers: weights in, mesh out
    e2e = None
    if not args.no_e2e:
        e2e_ms, h2d, d2h = 0.0, 0, 0
        pinned = {}
        host_layers = [(np.ascontiguousarray(W), np.ascontiguousarray(b_)) for W, b_ in layers]
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net2 = pkg.Inr(host_layers)
            r = net2.extract(L, isos, buffers=bufs, **kw)
            nt, na = r["n_tris"], r["n_active"]
            for key, tens in (("vert", r["tri_vert"]), ("edge", r["tri_edge"]), ("iso", r["tri_iso"]),
                              ("code", r["codes"]), ("mask", r["masks"])):
                if key not in pinned or pinned[key].numel() < tens.numel():
                    pinned[key] = torch.empty(max(tens.numel(), 1), dtype=tens.dtype, pin_memory=True)
                pinned[key][:tens.numel()].copy_(tens.reshape(-1), non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms += (time.perf_counter() - t0) * 1e3
            net2.close()
            h2d = sum(W.nbytes + b_.nbytes for W, b_ in host_layers)
            d2h = nt * (36 + 24 + 4) + na * 8
            steps_e2e = max(1, min(args.steps, 2))
        cells_one = sum(r["cells_bounded"])
        e2e = {"value": cells_one * world / (e2e_ms / steps_e2e / 1e3), "unit": "cells/s",
               "ms_per_step": e2e_ms / steps_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    peaks = load_peaks()
    # the roofline of the dominant bound kernel: the row-batched tcgen05 GEMM (BF16, default), the
    # per-cell tcgen05 kernel (BF16 with inflation) or the float32 coefficient GEMM
    bound_kernels = ["rows_gemm", "bound_tc", "gemm_fp32"]
    dom = max(bound_kernels, key=lambda k: stats.get(k, {}).get("ms", 0.0))
    ds = stats[dom]
    csrc = os.path.join(ROOT, "paper_2402_13861_gb300", "csrc")
    secs = ds["ms"] / 1e3 if ds["ms"] > 0 else float("inf")
    tc_peak = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm_peak = peaks.get("hbm_gbs", 6674.2)
    if dom == "rows_gemm":
        # arithmetic intensity 2 R w^2 / (4 R w bytes) = w / 2 FLOP/B: below the ridge, HBM-bound
        ai = ds["flops"] / max(ds["bytes"], 1.0)
        if ai * hbm_peak / 1e3 < tc_peak:
            roof = {"bound": "hbm", "unit": "GB/s", "peak_source": "measured hbm_gbs",
                    "arithmetic_intensity": ai, "achieved_tflops": ds["flops"] / secs / 1e12}
            achieved, peak = ds["bytes"] / secs / 1e9, hbm_peak
        else:
            roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": "measured bf16_tflops_sustained"}
            achieved, peak = ds["flops"] / secs / 1e12, tc_peak
        rec = traffic_record(dom, os.path.join(csrc, "rows_gemm.cu"))
        tr = rec["dram_per_alg_byte"] * ds["bytes"] / max(ds["launches"], 1) if rec else None
    elif dom == "bound_tc":
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": "measured bf16_tflops_sustained"}
        achieved, peak = ds["flops"] / secs / 1e12, tc_peak
        rec = traffic_record(dom, os.path.join(csrc, "bound_tc.cu"))
        tr = rec["dram_bytes_per_cell"] * cells_local / max(ds["launches"], 1) if rec else None
    else:
        # float32 FMA issue rate: 152 SMs x 128 lanes x 2 FLOP x max SM clock
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak_source": "152 SM x 128 FP32 lanes x 2 x max SM clock"}
        achieved = ds["flops"] / secs / 1e12
        tr = None
    roof.update({"kernel": dom, "achieved": achieved, "peak": peak, "frac": achieved / peak,
                 "launches": ds["launches"], "avg_launch_ms": ds["ms"] / max(ds["launches"], 1),
                 "traffic": tr})
    launches = int(sum(v["launches"] for v in stats.values()))
    shares = {k: round(v["ms"] / max(sum(x["ms"] for x in stats.values()), 1e-9), 4) for k, v in stats.items()
              if v["ms"] > 0}
    line = {"metric": "AA-bounded cells/s (hierarchical iso-extraction, 512^3, 8 isos)", "value": value,
            "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": f"scientific-field {1 << L}^3: 3->256x5->1 ReLU INR fitted to 256 anisotropic "
                                   f"Gaussians + sine, 8 isos over the 10-90% quantiles", "mode": args.mode,
                       "k": args.k, "precision": prec, "eval_precision": eval_prec, "inflate": kw["inflate"],
                       "max_level": L,
                       "l2": "512 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
            "phase_ms": {"acp": phases[0] / args.steps, "inr": phases[1] / args.steps, "mc": phases[2] / args.steps},
            "cells_bounded_per_step": cells / args.steps / world, "n_active": res["n_active"],
            "n_tris": res["n_tris"], "cells_bounded_per_level": res["cells_bounded"],
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "kernel_time_share": shares}
    try:
        line["rooflines"] = kernel_rooflines(stats, hbm_peak, tc_peak,
                                             152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12)
    except Exception as ex:                      # the per-kernel list never costs the bench line
        line["rooflines"] = {"error": repr(ex)}
    if rank == 0 and world == 1 and not args.no_forms:
        line["forms"] = extraction_forms(pkg, net, L, isos, res, ms_per_step, args.mode, args.k, prec,
                                         slow=args.all_forms)
        # every further form is measured on its own: one that fails records its error, never the line
        extra = [("fp32_vs_bf16", lambda: precision_sample(net, args.mode))]
        if prec == "bf16":
            extra += [("large", lambda: large_form(pkg, full=args.all_forms)),
                      ("batched", lambda: batched_form(pkg, args.mode, args.k, full=args.all_forms)),
                      ("activations", lambda: activation_forms(
                          pkg, args.k, ("siren", "sdf_elu") if args.all_forms else ("sdf_elu",)))]
        for name, fn in extra:
            try:
                line["forms"][name] = fn()
            except Exception as ex:
                line["forms"][name] = {"error": repr(ex)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(layers, args.mode, args.k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    if world > 1:
        dist.destroy_process_group()


def _bf16_ok(net, pkg):
    import torch
    try:
        lo = torch.zeros((1, 3), device="cuda")
        net.bound_cells(lo, lo + 0.5, mode="clt", prec="bf16")
        torch.cuda.synchronize()
        return True
    except pkg.IsxError:
        return False


if __name__ == "__main__":
    main()
