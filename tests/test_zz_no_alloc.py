"""The allocation-free bound entry point, isx_bound_cells_noalloc, called through the C interface.

Some callers cannot allocate device memory once they are running: their device memory belongs to a
framework's caching allocator, or they sit in a latency-critical loop that must not take the
device-wide synchronisation of cudaMalloc / cudaFree.  This entry point takes its scratch from an
array compiled into the library instead of the INR's workspace.  Checked here:
  - on a fresh INR that was never bounded before, two calls leave the device's free memory
    unchanged (the kernel and the array are brought in by a first call on another INR);
  - two calls in a row give bit-identical bounds, which agree with isx_bound_cells (the existing
    entry point) within the tolerance the other bf16 tests use, and with the float64 oracle within
    each result's band (tests/_rounding_model.py);
  - unsupported widths are rejected.
This file is collected last, so that a run that stops at the first failure has already run every
other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import boxes, inr

import _rounding_model as rm

pytestmark = pytest.mark.gpu

UB = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _call_noalloc(net, lo, hi, mode, c, s, inflate=False):
    from paper_2402_13861_gb300 import _lib
    st = _lib.load().isx_bound_cells_noalloc(net.handle, C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()),
                                             lo.shape[0], _lib.MODES[mode], int(inflate), C.c_void_p(c.data_ptr()),
                                             C.c_void_p(s.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.load().isx_last_error()


def test_noalloc_allocates_nothing_on_a_fresh_inr(pkg):
    from paper_2402_13861_gb300 import _lib
    _lib.profile_enable(False)
    lo, hi = boxes.random_boxes(700, 5, -8, -2)
    dlo, dhi = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    c = torch.empty(700, device="cuda")
    s = torch.empty(700, device="cuda")
    warm = pkg.Inr(inr.random_inr([3, 128, 128, 128, 1], 7))
    _call_noalloc(warm, dlo, dhi, "clt", c, s)                # loads the kernel, looks up the array
    torch.cuda.synchronize()
    fresh = pkg.Inr(inr.random_inr([3] + [256] * 5 + [1], 8))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _call_noalloc(fresh, dlo, dhi, "sound", c, s)
    _call_noalloc(fresh, dlo, dhi, "clt", c, s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    print(f"free device memory before {free0}, after {free1}")
    assert free1 == free0
    assert torch.isfinite(c).all() and torch.isfinite(s).all()
    fresh.close()
    warm.close()


@pytest.mark.parametrize("dims,mode", [("scientific", "clt"), ("scientific", "sound"),
                                       ([3, 128, 128, 128, 128, 1], "raua")])
def test_noalloc_matches_bound_cells_twice(pkg, dims, mode):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 44)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    n = 1500
    lo, hi = boxes.random_boxes(n, 61, -9, -1)
    dlo, dhi = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    c_ref, s_ref = net.bound_cells(dlo, dhi, mode=mode, prec="bf16")
    c_ref, s_ref = c_ref.cpu().numpy().astype(np.float64), s_ref.cpu().numpy().astype(np.float64)
    tol = 3 * H * UB          # the blanket bf16 tolerance of the other bf16 tests' gross-error checks
    first = None
    for _ in range(2):
        c = torch.full((n,), float("nan"), device="cuda")
        s = torch.full((n,), float("nan"), device="cuda")
        _call_noalloc(net, dlo, dhi, mode, c, s)
        torch.cuda.synchronize()
        c, s = c.cpu().numpy(), s.cpu().numpy()
        assert np.all(np.isfinite(c)) and np.all(np.isfinite(s))
        if first is None:
            first = (c, s)
        else:
            assert np.array_equal(c, first[0]) and np.array_equal(s, first[1])
        c, s = c.astype(np.float64), s.astype(np.float64)
        assert np.all(np.abs(s - s_ref) <= tol * np.abs(s_ref) + 1e-6)
        assert np.all(np.abs(c - c_ref) <= tol * (np.abs(c_ref) + np.abs(s_ref)) + 1e-6)
    idx = np.linspace(0, n - 1, 16).astype(np.int64)
    b = rm.bound_bands(layers, lo[idx], hi[idx], mode, batch=16)
    c, s = first[0][idx].astype(np.float64), first[1][idx].astype(np.float64)
    print(f"{mode}: max |d x0| / band {np.max(np.abs(c - b['centre']) / b['band_c']):.3f}, |d spread| / band "
          f"{np.max(np.abs(s - b['spread']) / b['band_s']):.3f}")
    assert np.all(np.abs(c - b["centre"]) <= b["band_c"]) and np.all(np.abs(s - b["spread"]) <= b["band_s"])
    net.close()


def test_noalloc_rejects_unsupported_width(pkg):
    from paper_2402_13861_gb300 import _lib
    net = pkg.Inr(inr.random_inr([3, 64, 64, 1], 3))
    lo = torch.zeros((8, 3), device="cuda")
    out = torch.empty(8, device="cuda")
    st = _lib.load().isx_bound_cells_noalloc(net.handle, C.c_void_p(lo.data_ptr()), C.c_void_p(lo.data_ptr()), 8,
                                             0, 0, C.c_void_p(out.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert st == 5 and b"128 or 256" in _lib.load().isx_last_error()
    net.close()
