"""Seeded synthetic scalar fields on the domain [-1, 1]^3.

The paper measures on simulation volumes (Vortex, Ethanediol, Combustion, Isotropic; Sec. V-A.1)
that are not available here.  These analytic fields stand in for them: sums of Gaussian blobs
(isotropic or anisotropic with random rotations) plus an optional low-amplitude sine texture,
which give the multi-scale, oscillating structure that makes range analysis loose on scientific
data (Sec. I).

This module holds no part of the extraction method: it only defines fields, draws their
parameters from ``numpy.random.default_rng(seed)`` in a fixed order, and evaluates them.

Draw order for a field with ``n`` blobs (documented so that any reimplementation reproduces it):
centres ``(n, 3)`` uniform in ``[-0.7, 0.7]``; then widths (``(n,)`` for isotropic blobs,
``(n, 3)`` axis widths for anisotropic ones); then amplitudes ``(n,)`` uniform in ``[0.5, 1]``;
then, for anisotropic blobs only, ``(n, 4)`` standard normals normalised to unit quaternions
(a Haar-random rotation).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices from unit quaternions ``q = (w, x, y, z)``, shape ``(n, 4) -> (n, 3, 3)``."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


@dataclass
class GaussianField:
    """f(x) = sum_b a_b exp(-1/2 (x-c_b)^T P_b (x-c_b)) + s * sin(f pi x) sin(f pi y) sin(f pi z).

    ``P_b`` is the precision matrix ``R diag(sigma^-2) R^T`` of blob ``b``.
    """

    centers: np.ndarray      # (n, 3)
    precisions: np.ndarray   # (n, 3, 3)
    amps: np.ndarray         # (n,)
    sine_amp: float = 0.0
    sine_freq: float = 6.0

    def __call__(self, x: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        out = np.empty(x.shape[0])
        for s in range(0, x.shape[0], chunk):
            xs = x[s:s + chunk]
            d = xs[:, None, :] - self.centers[None, :, :]                 # (m, n, 3)
            q = np.einsum("mni,nij,mnj->mn", d, self.precisions, d)
            v = np.exp(-0.5 * q) @ self.amps
            if self.sine_amp:
                f = self.sine_freq * np.pi
                v = v + self.sine_amp * np.sin(f * xs[:, 0]) * np.sin(f * xs[:, 1]) * np.sin(f * xs[:, 2])
            out[s:s + chunk] = v
        return out

    def torch_eval(self, x):
        """Same field on a torch tensor ``x`` of shape (m, 3) (used only to make fitting targets)."""
        import torch
        c = torch.as_tensor(self.centers, dtype=x.dtype, device=x.device)
        P = torch.as_tensor(self.precisions, dtype=x.dtype, device=x.device)
        a = torch.as_tensor(self.amps, dtype=x.dtype, device=x.device)
        d = x[:, None, :] - c[None]
        q = torch.einsum("mni,nij,mnj->mn", d, P, d)
        v = torch.exp(-0.5 * q) @ a
        if self.sine_amp:
            f = self.sine_freq * np.pi
            v = v + self.sine_amp * torch.sin(f * x[:, 0]) * torch.sin(f * x[:, 1]) * torch.sin(f * x[:, 2])
        return v


def isotropic_blobs(seed: int, n: int = 8, sigma_range=(0.1, 0.3), amp_range=(0.5, 1.0)) -> GaussianField:
    """``n`` isotropic blobs: centres U[-0.7,0.7]^3, width U[sigma_range], amplitude U[amp_range]."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-0.7, 0.7, size=(n, 3))
    sig = rng.uniform(*sigma_range, size=n)
    amps = rng.uniform(*amp_range, size=n)
    P = np.eye(3)[None] / (sig ** 2)[:, None, None]
    return GaussianField(centers, P, amps)


def anisotropic_blobs(seed: int, n: int = 256, sigma_range=(0.02, 0.2), amp_range=(0.5, 1.0),
                      sine_amp: float = 0.05, sine_freq: float = 6.0) -> GaussianField:
    """``n`` anisotropic blobs with Haar-random rotations plus ``sine_amp * sin(6 pi x) sin(6 pi y) sin(6 pi z)``."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-0.7, 0.7, size=(n, 3))
    sig = rng.uniform(*sigma_range, size=(n, 3))
    amps = rng.uniform(*amp_range, size=n)
    q = rng.standard_normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = _quat_to_rot(q)
    P = np.einsum("nij,nj,nkj->nik", R, 1.0 / sig ** 2, R)
    return GaussianField(centers, P, amps, sine_amp=sine_amp, sine_freq=sine_freq)


def sphere_sdf(radius: float = 0.5):
    """Analytic signed distance to a sphere at the origin: ``|x| - radius`` (negative inside)."""
    def f(x):
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        return np.linalg.norm(x, axis=1) - radius
    return f


@dataclass
class SdfField:
    """Signed distance (negative inside) to the union of a torus in the z = 0 plane (major radius
    ``R``, minor ``r``) and spheres ``(centre, radius)``: the min of the parts' distances, which is
    an exact distance outside the union and a lower bound on the depth inside."""
    R: float
    r: float
    spheres: list

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
        q = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) - self.R
        d = np.sqrt(q * q + x[:, 2] ** 2) - self.r
        for c, rad in self.spheres:
            d = np.minimum(d, np.linalg.norm(x - np.asarray(c), axis=1) - rad)
        return d

    def torch_eval(self, x):
        import torch
        q = torch.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) - self.R
        d = torch.sqrt(q * q + x[:, 2] ** 2) - self.r
        for c, rad in self.spheres:
            d = torch.minimum(d, torch.linalg.norm(x - torch.tensor(c, dtype=x.dtype, device=x.device), dim=1) - rad)
        return d


def torus_and_spheres():
    """The synthetic SDF of the mesh-extraction workload: a torus (R = 0.5, r = 0.18) with three
    spheres (radii 0.22, 0.15, 0.12) placed on and off its ring."""
    return SdfField(0.5, 0.18, [((0.5, 0.0, 0.0), 0.22), ((-0.25, 0.43, 0.1), 0.15), ((0.0, 0.0, 0.45), 0.12)])
