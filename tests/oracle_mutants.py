"""Mutation check of the oracle's pins: plant one plausible mistake at a time (a dropped term, a
wrong sign, index or constant, a transposed operand, a strict comparison) in a fresh copy of
oracle/, run the CPU pins (test_oracle_pins.py, test_oracle_proposer.py) against that copy and
report every mistake that no pin catches.  The repository is never modified.

    python tests/oracle_mutants.py [-j WORKERS] [INDEX ...]

Exit status 0 when every planted mistake is caught.  Not collected by pytest (each mistake costs
one run of the pins, about 20 s); run it after changing the oracle or its pins.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle file, text that occurs exactly once, the mistaken text)
MUTANTS = [
 ("affine.py", "h = h / np.sqrt(3.0)", "h = h / 3.0"),
 ("affine.py", "beta[cross] = -a * l[cross] / 2.0", "beta[cross] = a * l[cross] / 2.0"),
 ("affine.py", "gamma[cross] = -a * l[cross] / 2.0", "gamma[cross] = -a * l[cross]"),
 ("affine.py", "a = u[cross] / (u[cross] - l[cross])", "a = u[cross] / (u[cross] + l[cross])"),
 ("affine.py", "a = erf(-m / (np.sqrt(2.0) * sg))", "a = erf(m / (np.sqrt(2.0) * sg))"),
 ("affine.py", " + a * m * b - b * b", " - b * b"),
 ("affine.py", "b = sg / np.sqrt(2.0 * np.pi) * np.exp(-m * m / (2.0 * sg * sg))", "b = sg / np.sqrt(2.0 * np.pi) * np.exp(-m * m / (sg * sg))"),
 ("affine.py", "sigma = np.sqrt(np.sum(X * X, axis=1))      # Eq. 7", "sigma = np.sum(np.abs(X), axis=1)"),
 ("affine.py", "X = X * alpha[:, None, :]                         # Eq. 4", "X = X  #"),
 ("affine.py", "c = alpha * c + beta                              # Eq. 4", "c = alpha * c  #"),
 ("affine.py", "G[:, np.arange(w), np.arange(w)] = gamma", "G[:, np.arange(w), np.arange(w)] = gamma * gamma"),
 ("affine.py", "np.sqrt(np.sum(coef * coef, axis=1) / 3.0)", "np.sqrt(np.sum(coef * coef, axis=1))"),
 ("affine.py", "r = r @ np.abs(W).T", "r = r @ W.T"),
 ("affine.py", "r = alpha * r + gamma", "r = r + gamma"),
 ("affine.py", "s = np.sum(np.abs(A), axis=1) + r", "s = np.sum(np.abs(A), axis=1)"),
 ("affine.py", "return centre - k * spread, centre + k * spread", "return centre - spread, centre + spread"),
 ("affine.py", "C[:, np.arange(w), np.arange(w)] += gamma * gamma", "C[:, np.arange(w), np.arange(w)] += gamma"),
 ("affine.py", "c = c @ W.T + b                      # Eq. 3", "c = c @ W.T  #"),
 ("affine.py", "alpha[pos] = 1.0", "alpha[pos] = 0.5"),
 ("activations.py", "ef2 = ex2_pos + b2 - 2.0 * b1 + Q", "ef2 = ex2_pos + b2 - b1 + Q"),
 ("activations.py", "xb1 = (mu + s2) * b1 - sigma * phi", "xb1 = (mu + s2) * b1 + sigma * phi"),
 ("activations.py", "exf = mu * ef + sigma * sigma * a * np.cos(mu)", "exf = mu * ef + sigma * a * np.cos(mu)"),
 ("activations.py", "np.exp(-2.0 * sigma * sigma) * np.cos(2.0 * mu)", "np.exp(-sigma * sigma) * np.cos(2.0 * mu)"),
 ("activations.py", "gamma2[s] = ef2 - ef * ef - a * a * sg * sg", "gamma2[s] = ef2 - ef * ef - a * sg * sg"),
 ("activations.py", "alpha = np.where(mu > 0, 1.0, np.exp(np.minimum(mu, 0.0)))", "alpha = np.where(mu > 0, 1.0, 1.0)"),
 ("activations.py", "np.expm1(np.minimum(z, 0.0))", "np.exp(np.minimum(z, 0.0))"),
 ("activations.py", "ex2_pos = (mu * mu + sigma * sigma) * Phi + mu * sigma * phi", "ex2_pos = (mu * mu + sigma * sigma) * Phi"),
 ("activations.py", "ex_neg = mu * Q - sigma * phi", "ex_neg = mu * Q + sigma * phi"),
 ("activations.py", "a = np.exp(-0.5 * sigma * sigma)", "a = np.exp(-sigma * sigma)"),
 ("activations.py", "alpha = np.cos(mu)", "alpha = np.sin(mu)"),
 ("mlp.py", "if l < len(L) - 1:", "if l < len(L):"),
 ("octree.py", "[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1]", "[(c >> 0) & 1, (c >> 0) & 1, (c >> 2) & 1]"),
 ("octree.py", "(lower[:, None] <= isos[None, :])", "(lower[:, None] < isos[None, :])"),
 ("octree.py", "splits = np.array([(depth + 2 - a) // 3 for a in range(3)])", "splits = np.array([(depth + a) // 3 for a in range(3)])"),
 ("octree.py", "axis = depth % 3", "axis = 2 - depth % 3"),
 ("octree.py", "size = 2.0 / float(1 << level)", "size = 1.0 / float(1 << level)"),
 ("octree.py", "t = -1.0 + 2.0 * np.arange(R + 1) / R", "t = -1.0 + 2.0 * np.arange(R + 1) / (R + 1)"),
 ("octree.py", "fpr = fp / (fp + tn) if fp + tn else 0.0", "fpr = fp / (fp + tp) if fp + tp else 0.0"),
 ("octree.py", "masks = np.repeat(new[keep], 8)", "masks = np.repeat(masks[keep], 8)"),
 ("octree.py", "z, y, x = np.meshgrid(t, t, t, indexing=\"ij\")", "x, y, z = np.meshgrid(t, t, t, indexing=\"ij\")"),
 ("mc.py", "off[q] = t >> 1", "off[q] = t & 1"),
 ("mc.py", "return (e1, e2) if side < 0 else (e2, e1)", "return (e1, e2) if side > 0 else (e2, e1)"),
 ("mc.py", "bits = (cv < iso).astype(np.int64)", "bits = (cv <= iso).astype(np.int64)"),
 ("mc.py", "t = (iso - va) / (vb - va)", "t = (iso - vb) / (va - vb)"),
 ("mc.py", "return (np.asarray(k, np.int64) * (R + 1) + np.asarray(j, np.int64)) * (R + 1) + np.asarray(i, np.int64)",
          "return (np.asarray(i, np.int64) * (R + 1) + np.asarray(j, np.int64)) * (R + 1) + np.asarray(k, np.int64)"),
 ("mc.py", "gid = 3 * lattice_index(base[..., 0], base[..., 1], base[..., 2], R) + axis", "gid = 3 * lattice_index(base[..., 0], base[..., 1], base[..., 2], R)"),
 ("mc.py", "pos = -1.0 + 2.0 * base.astype(np.float64) / R", "pos = -1.0 + 2.0 * base.astype(np.float64) / (R + 1)"),
 ("mc.py", "tris.append((loop[0], loop[i], loop[i + 1]))", "tris.append((loop[0], loop[i + 1], loop[i]))"),
 ("mc.py", "all_in &= s", "all_in |= s"),
 ("proposer.py", "delta = (delta @ W) * (pres[l - 1] > 0.0)", "delta = (delta @ W)"),
 ("proposer.py", "grads[l] = (delta.T @ acts[l], delta.sum(axis=0))", "grads[l] = (delta.T @ acts[l], delta.mean(axis=0))"),
 ("proposer.py", "vh = v / (1 - b2 ** t)", "vh = v"),
 ("proposer.py", "np.log1p(np.exp(-np.abs(z)))", "np.log1p(np.exp(-z))"),
 ("proposer.py", "X[:, 0:3] = -1.0 + (2.0 * ijk + 1.0) * h[:, None]", "X[:, 0:3] = -1.0 + (2.0 * ijk) * h[:, None]"),
 ("proposer.py", "X[:, 5] = np.asarray(anc_centre, dtype=np.float64) - iso", "X[:, 5] = iso - np.asarray(anc_centre, dtype=np.float64)"),
 ("proposer.py", "anc = np.asarray(crossing_codes, dtype=np.int64) >> shift", "anc = np.asarray(crossing_codes, dtype=np.int64) >> (shift + 1)"),
 ("proposer.py", "params.append((rng.normal(0.0, np.sqrt(2.0 / fi), size=(fo, fi)), np.zeros(fo)))",
                 "params.append((rng.normal(0.0, np.sqrt(2.0 / fo), size=(fo, fi)), np.zeros(fo)))"),
 ("octree.py", "(isos[None, :] <= upper[:, None])", "(isos[None, :] < upper[:, None])"),
 ("affine.py", "X[:, [0, 1, 2], [0, 1, 2]] = h", "X[:, [0, 1, 2], [2, 1, 0]] = h"),
 ("affine.py", "alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 0.5, 0.0)).astype(np.float64)", "alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 1.0, 0.0)).astype(np.float64)"),
 ("affine.py", "alpha[s] = 0.5 * (1.0 - a)", "alpha[s] = 0.5 * (1.0 + a)"),
 ("affine.py", "        if l == len(L) - 1:\n            break\n        if mode == CLT:", "        if l == len(L):\n            break\n        if mode == CLT:"),
 ("affine.py", "spread[s:s + batch] = np.sqrt(np.sum(coef * coef, axis=1))     # Eq. 7", "spread[s:s + batch] = np.sum(np.abs(coef), axis=1)"),
 ("affine.py", "var_in = ((hi - lo) / 2.0) ** 2 / 3.0", "var_in = ((hi - lo) / 2.0) ** 2"),
 ("affine.py", "c, A = input_form(lo, hi, SOUND)", "c, A = input_form(lo, hi, CLT)"),
 ("affine.py", "return c[:, 0], np.sum(np.abs(A[:, :, 0]), axis=1) + r[:, 0]", "return c[:, 0], np.sum(np.abs(A[:, :, 0]), axis=1)"),
 ("affine.py", "xc = (lo + hi) / 2.0", "xc = lo"),
 ("activations.py", "ex_pos = mu * Phi + sigma * phi", "ex_pos = mu * Phi - sigma * phi"),
 ("activations.py", "ef = ex_pos + b1 - Q", "ef = ex_pos + b1 + Q"),
 ("activations.py", "exf = ex2_pos + xb1 - ex_neg", "exf = ex2_pos + xb1 + ex_neg"),
 ("activations.py", "b1, b2 = e_exp_neg(1.0), e_exp_neg(2.0)", "b1, b2 = e_exp_neg(1.0), e_exp_neg(1.0)"),
 ("activations.py", "np.exp(s * mu + 0.5 * s * s * s2)", "np.exp(s * mu + 0.5 * s * s2)"),
 ("activations.py", "beta[s] = ef - a * m", "beta[s] = ef - a"),
 ("activations.py", "alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 0.5, 0.0))", "alpha = np.where(mu > 0, 1.0, np.where(mu == 0, 1.0, 0.0))"),
 ("activations.py", "erfc((mu + s * s2) / (np.sqrt(2.0) * sigma))", "erfc((mu - s * s2) / (np.sqrt(2.0) * sigma))"),
 ("activations.py", "ef = a * np.sin(mu)", "ef = a * np.cos(mu)"),
 ("mlp.py", "a = np.maximum(a, 0.0) if act == \"relu\" else forward(act, a)", "a = np.abs(a) if act == \"relu\" else forward(act, a)"),
 ("octree.py", "masks = np.repeat(new[keep], 2)", "masks = np.repeat(masks[keep], 2)"),
 ("octree.py", "full = (1 << isos.shape[0]) - 1\n    if start_cells", "full = 1\n    if start_cells"),
 ("octree.py", "        lower, upper = affine.interval(centre, spread, mode, k)\n        new = masks & iso_bits(lower, upper, isos)\n        depths", "        lower, upper = affine.interval(centre, spread, mode, k)\n        new = iso_bits(lower, upper, isos)\n        depths"),
 ("mc.py", "for i in range(1, len(loop) - 1):", "for i in range(1, len(loop) - 2):"),
 ("mc.py", "return np.stack([i, j, k], axis=1)", "return np.stack([k, j, i], axis=1)"),
 ("mc.py", "n[a] = 1.0 if s else -1.0", "n[a] = 1.0"),
 ("mc.py", "np.put_along_axis(step, axis[..., None], (2.0 / R) * t[..., None], axis=2)", "np.put_along_axis(step, axis[..., None], (1.0 / R) * t[..., None], axis=2)"),
 ("mc.py", "e = np.take_along_axis(e, idx, axis=1)", "e = np.sort(e, axis=1)"),
 ("proposer.py", "out[~pos] = ez / (1.0 + ez)", "out[~pos] = 1.0 / (1.0 + ez)"),
 ("proposer.py", "a = (a - mu) / sd", "a = (a - mu) * sd"),
 ("proposer.py", "X[:, 3] = -level", "X[:, 3] = level"),
 ("proposer.py", "table[key] = table.get(key, 0) | m", "table[key] = m"),
 ("proposer.py", "m = state[\"m\"][l][k] = b1 * state[\"m\"][l][k] + (1 - b1) * g", "m = state[\"m\"][l][k] = b1 * state[\"m\"][l][k] + (1 - b1) * g * g"),
 ("proposer.py", "a = np.maximum(zl, 0.0) if l < len(params) - 1 else zl", "a = np.maximum(zl, 0.0)")
]


def run_one(idx):
    f, old, new = MUTANTS[idx]
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        for sub in ("oracle", "tests", "synth"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("__pycache__"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
        p = os.path.join(d, "oracle", f)
        src = open(p).read()
        if src.count(old) != 1:
            return idx, "pattern occurs %d times" % src.count(old), ""
        open(p, "w").write(src.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                            "tests/test_oracle_pins.py", "tests/test_oracle_proposer.py"],
                           cwd=d, capture_output=True, text=True, timeout=1800)
        failed = [ln for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]
        return idx, "caught" if r.returncode != 0 else "NOT CAUGHT", failed[0].split(" - ")[0] if failed else ""
    finally:
        shutil.rmtree(d, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    ap.add_argument("index", type=int, nargs="*")
    args = ap.parse_args()
    sel = args.index or list(range(len(MUTANTS)))
    with ThreadPoolExecutor(args.j) as ex:
        results = sorted(ex.map(run_one, sel))
    for idx, verdict, where in results:
        f, old, _ = MUTANTS[idx]
        print(f"{idx:3d} {f:15s} {verdict:10s} {old.splitlines()[0].strip()[:60]:60s} {where}")
    missed = [r for r in results if r[1] != "caught"]
    print(f"{len(results) - len(missed)} of {len(results)} planted mistakes caught")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
