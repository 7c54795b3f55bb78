"""The allocation-free bound entry point (isx_bound_cells_noalloc) gives the same bounds as
isx_bound_cells in bf16, on two calls in a row, through the C interface.

It exists for callers that may not allocate device memory once running (a framework-owned
allocator, a loop that must not take cudaMalloc's device-wide synchronisation); it takes its
scratch from an array compiled into the library.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import boxes, inr

pytestmark = pytest.mark.gpu

UB = 2.0 ** -8


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_2402_13861_gb300 as p
    torch.cuda.set_device(0)
    return p


def _call_noalloc(pkg, net, lo, hi, mode, inflate=False):
    from paper_2402_13861_gb300 import _lib
    n = lo.shape[0]
    c = torch.full((n,), float("nan"), device="cuda")
    s = torch.full((n,), float("nan"), device="cuda")
    st = _lib.load().isx_bound_cells_noalloc(net.handle, C.c_void_p(lo.data_ptr()), C.c_void_p(hi.data_ptr()), n,
                                             _lib.MODES[mode], int(inflate), C.c_void_p(c.data_ptr()),
                                             C.c_void_p(s.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.load().isx_last_error()
    torch.cuda.synchronize()
    return c.cpu().numpy(), s.cpu().numpy()


@pytest.mark.parametrize("dims,mode", [("scientific", "clt"), ("scientific", "sound"),
                                       ([3, 128, 128, 128, 128, 1], "raua")])
def test_noalloc_matches_bound_cells_twice(pkg, dims, mode):
    layers = inr.load_inr(dims)[0] if isinstance(dims, str) else inr.random_inr(dims, 44)
    H = len(layers) - 1
    net = pkg.Inr(layers)
    lo, hi = boxes.random_boxes(1500, 61, -9, -1)
    dlo, dhi = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    infl = mode == "sound"
    c_ref, s_ref = net.bound_cells(dlo, dhi, mode=mode, prec="bf16", inflate=infl)
    c_ref, s_ref = c_ref.cpu().numpy(), s_ref.cpu().numpy()
    tol = 3 * H * UB          # the bf16 tolerance used by the other bf16 tests
    for _ in range(2):
        c, s = _call_noalloc(pkg, net, dlo, dhi, mode, inflate=infl)
        assert np.all(np.isfinite(c)) and np.all(np.isfinite(s))
        assert np.all(np.abs(s - s_ref) <= tol * np.abs(s_ref) + 1e-6)
        assert np.all(np.abs(c - c_ref) <= tol * (np.abs(c_ref) + np.abs(s_ref)) + 1e-6)
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
