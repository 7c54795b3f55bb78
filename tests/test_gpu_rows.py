"""The row-batched tensor-core bound path (bound_rows.cu): bounds of many cells, over several
chunks of the layer-synchronous loop, against the per-cell tensor-core kernel (reached through
isx_bound_cells_noalloc, which always runs it) and the float32 path.  A sample of the cells is
checked against the float64 oracle with per-result bands (tests/_rounding_model.py); every cell is
also held to the blanket band 3 H u_b (|x0| + spread) (u_b = 2^-8) against the other two paths,
a check for gross errors such as a row of another cell or a wrong chunk boundary.  The path really
runs: its GEMM kernel is counted by the launch accounting."""
import numpy as np
import pytest
import torch

from synth import boxes, inr

import _rounding_model as rm
from _helpers import to_np

pytestmark = pytest.mark.gpu
UB = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _cubes(n, seed, lmin, lmax):
    ijk, level, lo, hi = boxes.random_cubes(n, seed, lmin, lmax)
    return torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")


def per_cell_kernel(net, lo, hi, mode):
    """Bounds from the per-cell tensor-core kernel (isx_bound_cells_noalloc runs only that kernel)."""
    import ctypes as C
    from paper_2402_13861_gb300 import _lib
    n = lo.shape[0]
    c = torch.empty(n, device="cuda")
    s = torch.empty(n, device="cuda")
    st = _lib.load().isx_bound_cells_noalloc(net.handle, C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()), n,
                                             _lib.MODES[mode], 0, C.c_void_p(c.data_ptr()), C.c_void_p(s.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.load().isx_last_error()
    torch.cuda.synchronize()
    return c, s


@pytest.mark.parametrize("dims", [[3, 128, 128, 128, 1], "scientific"])
@pytest.mark.parametrize("mode", ["clt", "sound", "raua"])
def test_rows_path_matches_per_cell_kernel(pkg, dims, mode):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 5)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    n = 60000 if isinstance(dims, str) else 20000          # several chunks of the row loop at w = 256
    lo, hi = _cubes(n, 12, 3, 9)
    c, s = net.bound_cells(lo, hi, mode=mode, prec="bf16")
    c, s = to_np(c).astype(np.float64), to_np(s).astype(np.float64)
    c1, s1 = per_cell_kernel(net, lo, hi, mode)
    c1, s1 = to_np(c1).astype(np.float64), to_np(s1).astype(np.float64)
    # a sample spread over the chunks against the oracle, with per-result bands
    idx = np.linspace(0, n - 1, 16 if isinstance(dims, str) else 48).astype(np.int64)
    b = rm.bound_bands(layers, to_np(lo)[idx], to_np(hi)[idx], mode, batch=16)
    for name, (cc, ss) in (("rows", (c, s)), ("per-cell", (c1, s1))):
        dc, ds = np.abs(cc[idx] - b["centre"]), np.abs(ss[idx] - b["spread"])
        print(f"{name} {mode}: max |d x0| / band {np.max(dc / b['band_c']):.3f}, |d spread| / band "
              f"{np.max(ds / b['band_s']):.3f}")
        assert np.all(dc <= b["band_c"]) and np.all(ds <= b["band_s"])
    m = 4000
    c32, s32 = net.bound_cells(lo[:m], hi[:m], mode=mode, prec="fp32")
    c32, s32 = to_np(c32).astype(np.float64), to_np(s32).astype(np.float64)
    tol = 3 * H * UB * (np.abs(c1) + s1) + 1e-6
    print(f"{dims if isinstance(dims, str) else dims[1:-1]} {mode}: rows vs per-cell max |dc|/tol "
          f"{np.max(np.abs(c - c1) / tol):.3f}, |ds|/tol {np.max(np.abs(s - s1) / tol):.3f}; rows vs fp32 "
          f"|ds|/s {np.max(np.abs(s[:m] - s32) / np.maximum(s32, 1e-30)):.2e}")
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(s))
    assert np.all(np.abs(c - c1) <= 2 * tol) and np.all(np.abs(s - s1) <= 2 * tol)
    tol32 = 3 * H * UB * (np.abs(c32) + s32) + 1e-6
    assert np.all(np.abs(c[:m] - c32) <= tol32) and np.all(np.abs(s[:m] - s32) <= tol32)
    net.close()


def test_rows_path_runs_its_kernels(pkg):
    from paper_2402_13861_gb300 import _lib
    net = pkg.Inr(inr.random_inr([3, 256, 256, 256, 1], 6))
    lo, hi = _cubes(3000, 13, 2, 8)
    _lib.profile_enable(True)
    _lib.profile_reset()
    net.bound_cells(lo, hi, mode="clt", prec="bf16")
    torch.cuda.synchronize()
    prof = _lib.profile_read()
    _lib.profile_enable(False)
    assert prof["rows_gemm"]["launches"] >= 1 and prof.get("bound_tc", {"launches": 0})["launches"] == 0
    print("rows_gemm launches", prof["rows_gemm"]["launches"], "GFLOP", prof["rows_gemm"]["flops"] / 1e9)
    net.close()


@pytest.mark.parametrize("mode", ["clt", "sound"])
def test_rows_path_width_64_matches_fp32(pkg, mode):
    """Width 64 (no per-cell tensor-core kernel) against the float32 path, over several tiles."""
    layers = inr.random_inr([3, 64, 64, 64, 64, 1], 8)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    lo, hi = _cubes(30000, 14, 2, 9)
    c, s = net.bound_cells(lo, hi, mode=mode, prec="bf16")
    c32, s32 = net.bound_cells(lo, hi, mode=mode, prec="fp32")
    c, s, c32, s32 = (to_np(x).astype(np.float64) for x in (c, s, c32, s32))
    tol = 3 * H * UB * (np.abs(c32) + s32) + 1e-6
    print(f"w64 {mode}: max |dc|/tol {np.max(np.abs(c - c32) / tol):.3f}, |ds|/tol {np.max(np.abs(s - s32) / tol):.3f}")
    assert np.all(np.abs(c - c32) <= tol) and np.all(np.abs(s - s32) <= tol)
    net.close()


@pytest.mark.parametrize("mode", ["clt", "sound"])
def test_rows_path_width_512_matches_fp32(pkg, mode):
    """Width 512 against the float32 path over many tiles of the quartered row GEMM and the halved
    split GEMM (the blanket band; per-result bands against the oracle are in test_gpu_bf16.py)."""
    layers = inr.random_inr([3, 512, 512, 512, 512, 1], 18)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    lo, hi = _cubes(6000, 15, 2, 9)
    c, s = net.bound_cells(lo, hi, mode=mode, prec="bf16")
    c32, s32 = net.bound_cells(lo, hi, mode=mode, prec="fp32")
    c, s, c32, s32 = (to_np(x).astype(np.float64) for x in (c, s, c32, s32))
    tol = 3 * H * UB * (np.abs(c32) + s32) + 1e-6
    print(f"w512 {mode}: max |dc|/tol {np.max(np.abs(c - c32) / tol):.3f}, |ds|/tol {np.max(np.abs(s - s32) / tol):.3f}")
    assert np.all(np.isfinite(c)) and np.all(np.abs(c - c32) <= tol) and np.all(np.abs(s - s32) <= tol)
    net.close()


def test_rows_path_width_64_extraction(pkg):
    """A BF16 extraction of the 3 -> 64 -> 64 -> 1 fixture runs on the row path and keeps the FP32
    extraction's active set up to cells near an iso-value."""
    layers, isos, wl = inr.load_inr("small")
    net = pkg.Inr(layers)
    a = net.extract(wl.max_level, isos, mode="clt", k=3.0, prec="bf16")
    b = net.extract(wl.max_level, isos, mode="clt", k=3.0, prec="fp32")
    sa = set((to_np(a["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist())
    sb = set((to_np(b["codes"]).astype(np.int64) & 0xFFFFFFFF).tolist())
    print(f"w64 extraction: bf16 {len(sa)} vs fp32 {len(sb)} active, symmetric difference {len(sa ^ sb)}")
    assert len(sb) > 1000 and len(sa ^ sb) <= 0.01 * len(sb)
    net.close()
