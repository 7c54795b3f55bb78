"""Seeded ReLU-MLP implicit neural representations fitted to the synthetic fields.

An INR here is a list of ``(W, b)`` float32 pairs, ``W`` row-major ``[out, in]``; layer 0 maps
``R^3 -> R^w``, hidden layers ``R^w -> R^w``, the last layer ``R^w -> R``, with ReLU between
linear layers (the ReLU INRs of App. E).  Weights start from He initialisation (normal with
standard deviation ``sqrt(2 / fan_in)``, zero biases, drawn layer by layer from
``numpy.random.default_rng(init_seed)``) and are fitted with Adam on mean squared error against
the field at uniform random samples of ``[-1, 1]^3``.

Fitting is fixture generation, not part of the extraction method: it produces the weights that
both the CPU oracle and the CUDA library then take as input.  It uses PyTorch autograd (on the GPU
when one is present).  Fitted weights are cached as ``.npz``; the small configuration's weights are
committed under ``synth/data`` so that CPU-only runs never refit.
"""
from __future__ import annotations

import os
import time
from dataclasses import dataclass, field as dc_field
from pathlib import Path

import numpy as np

from . import fields

DATA_DIR = Path(__file__).resolve().parent / "data"


def he_init(dims, seed):
    rng = np.random.default_rng(seed)
    layers = []
    for fan_in, fan_out in zip(dims[:-1], dims[1:]):
        W = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(fan_out, fan_in)).astype(np.float32)
        b = np.zeros(fan_out, dtype=np.float32)
        layers.append((W, b))
    return layers


def siren_init(dims, seed, omega0=30.0):
    """SIREN initialisation with the frequency factor folded in: a hidden layer computes sin(W x + b)
    with W = omega0 W', W' uniform on +-1/fan_in (first layer) or +-sqrt(6/fan_in)/omega0 (others),
    b = omega0 b', b' uniform on +-1/sqrt(fan_in); the output layer is linear (W' unscaled)."""
    rng = np.random.default_rng(seed)
    layers = []
    n = len(dims) - 1
    for l, (fan_in, fan_out) in enumerate(zip(dims[:-1], dims[1:])):
        lim = 1.0 / fan_in if l == 0 else np.sqrt(6.0 / fan_in) / omega0
        W = rng.uniform(-lim, lim, size=(fan_out, fan_in))
        b = rng.uniform(-1.0, 1.0, size=fan_out) / np.sqrt(fan_in)
        scale = omega0 if l < n - 1 else 1.0
        layers.append(((W * scale).astype(np.float32), (b * scale).astype(np.float32)))
    return layers


def _torch_act(act):
    import torch
    return {"relu": torch.relu, "elu": torch.nn.functional.elu, "sine": torch.sin}[act]


def _torch_forward(params, x, act="relu"):
    f = _torch_act(act)
    n = len(params) // 2
    a = x
    for l in range(n):
        a = a @ params[2 * l].T + params[2 * l + 1]
        if l < n - 1:
            a = f(a)
    return a[:, 0]


def fit(dims, target, steps, lr=1e-3, batch=65536, init_seed=0, sample_seed=1, device=None,
        log_every=0, act="relu"):
    """Adam fit of an MLP to ``target`` (a field with ``torch_eval``) on uniform samples: He
    initialisation for ReLU / ELU, SIREN initialisation (omega0 = 30, folded) for sine."""
    import torch
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    layers = siren_init(dims, init_seed) if act == "sine" else he_init(dims, init_seed)
    params = []
    for W, b in layers:
        params.append(torch.tensor(W, device=device, requires_grad=True))
        params.append(torch.tensor(b, device=device, requires_grad=True))
    opt = torch.optim.Adam(params, lr=lr)
    gen = torch.Generator(device=device)
    gen.manual_seed(sample_seed)
    for step in range(steps):
        x = torch.rand(batch, 3, generator=gen, device=device) * 2 - 1
        with torch.no_grad():
            y = target.torch_eval(x)
        loss = torch.mean((_torch_forward(params, x, act) - y) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        if log_every and step % log_every == 0:
            print(f"fit step {step} loss {loss.item():.3e}", flush=True)
    out = []
    for l in range(len(layers)):
        out.append((params[2 * l].detach().cpu().numpy().astype(np.float32),
                    params[2 * l + 1].detach().cpu().numpy().astype(np.float32)))
    return out, float(loss.item())


def lattice_centers(n):
    """Centres of the ``n^3`` cells of a uniform grid on [-1,1]^3, x fastest."""
    t = -1.0 + (2.0 * np.arange(n) + 1.0) / n
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def quantile_isos(layers, n_iso, lo_q=0.10, hi_q=0.90, grid=128, device=None, act="relu"):
    """``n_iso`` iso-values evenly spaced between the ``lo_q`` and ``hi_q`` quantiles of the fitted
    INR over the centres of a ``grid^3`` lattice (iso_q = q_lo + q (q_hi - q_lo) / (n_iso - 1))."""
    import torch
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    params = []
    for W, b in layers:
        params += [torch.tensor(W, device=device), torch.tensor(b, device=device)]
    x = lattice_centers(grid)
    vals = []
    with torch.no_grad():
        for s in range(0, x.shape[0], 1 << 18):
            xs = torch.tensor(x[s:s + (1 << 18)], dtype=torch.float32, device=device)
            vals.append(_torch_forward(params, xs, act).cpu().numpy())
    v = np.concatenate(vals)
    ql, qh = np.quantile(v, [lo_q, hi_q])
    if n_iso == 1:
        return np.array([(ql + qh) / 2], dtype=np.float32)
    return (ql + (qh - ql) * np.arange(n_iso) / (n_iso - 1)).astype(np.float32)


@dataclass
class Workload:
    """One named configuration: network shape, field, fit schedule, octree depth and iso-values."""
    name: str
    dims: list
    field_fn: object
    fit_steps: int
    init_seed: int
    sample_seed: int
    max_level: int
    n_iso: int = 1
    fixed_isos: list = dc_field(default_factory=list)
    k: float = 3.0
    lr: float = 1e-3
    batch: int = 65536
    act: str = "relu"


WORKLOADS = {
    # 3->64->64->1, 8 isotropic blobs (seed 0), 2000 Adam steps, octree to 64^3, iso 0.5, k = 3.
    "small": Workload("small", [3, 64, 64, 1], lambda: fields.isotropic_blobs(0, 8), 2000, 0, 1,
                      max_level=6, fixed_isos=[0.5]),
    # 3->256 (5 hidden)->1, 256 anisotropic blobs + 0.05 sin texture (seed 2), 5000 steps,
    # octree to 512^3, 8 iso-values over the 10-90 % quantiles.
    "scientific": Workload("scientific", [3] + [256] * 5 + [1], lambda: fields.anisotropic_blobs(2, 256),
                           5000, 2, 3, max_level=9, n_iso=8),
    # SIREN 3->256 (3 hidden)->1 (sine, omega0 = 30 folded in) on the scientific field (seed 2),
    # 3000 steps at lr 5e-4 (on the folded weights), octree to 512^3, 8 iso-values over the 10-90 % quantiles.
    "siren": Workload("siren", [3] + [256] * 3 + [1], lambda: fields.anisotropic_blobs(2, 256), 3000, 12, 13,
                      max_level=9, n_iso=8, lr=5e-4, act="sine"),
    # ELU SDF 3->128 (4 hidden)->1 of a torus with three spheres, 3000 steps, octree to 512^3, iso 0.
    "sdf_elu": Workload("sdf_elu", [3] + [128] * 4 + [1], fields.torus_and_spheres, 3000, 14, 15,
                        max_level=9, fixed_isos=[0.0], act="elu"),
    # 3->512 (8 hidden)->1, 1024 anisotropic blobs (seed 5), octree to 1024^3.
    "large": Workload("large", [3] + [512] * 8 + [1], lambda: fields.anisotropic_blobs(5, 1024),
                      5000, 5, 6, max_level=10, n_iso=1),
}


def _cache_dir() -> Path:
    return Path(os.environ.get("ISX_CACHE", "/tmp/isx_cache"))


def load_inr(name: str, device=None, verbose=False):
    """Weights and iso-values of a named workload: committed fixture, else cache, else fit now."""
    wl = WORKLOADS[name]
    for path in (DATA_DIR / f"{name}.npz", _cache_dir() / f"{name}.npz"):
        if path.exists():
            z = np.load(path)
            n = int(z["n_layers"])
            layers = [(z[f"W{l}"], z[f"b{l}"]) for l in range(n)]
            return layers, z["isos"].astype(np.float32), wl
    t0 = time.time()
    layers, loss = fit(wl.dims, wl.field_fn(), wl.fit_steps, wl.lr, wl.batch, wl.init_seed,
                       wl.sample_seed, device=device, act=wl.act)
    if wl.fixed_isos:
        isos = np.array(wl.fixed_isos, dtype=np.float32)
    else:
        isos = quantile_isos(layers, wl.n_iso, device=device, act=wl.act)
    if verbose:
        print(f"fitted {name} in {time.time() - t0:.1f}s, final loss {loss:.3e}", flush=True)
    save_inr(_cache_dir() / f"{name}.npz", layers, isos, loss)
    return layers, isos, wl


def save_inr(path: Path, layers, isos, loss=float("nan")):
    path.parent.mkdir(parents=True, exist_ok=True)
    arrs = {"n_layers": np.array(len(layers)), "isos": np.asarray(isos, np.float32),
            "final_loss": np.array(loss)}
    for l, (W, b) in enumerate(layers):
        arrs[f"W{l}"] = W
        arrs[f"b{l}"] = b
    tmp = path.with_suffix(".tmp.npz")
    np.savez(tmp, **arrs)
    os.replace(tmp, path)


def random_inr(dims, seed, act="relu"):
    """Unfitted MLP for shape and edge-case tests: He initialisation (ReLU, ELU) or the folded
    SIREN initialisation (sine)."""
    return siren_init(dims, seed) if act == "sine" else he_init(dims, seed)
