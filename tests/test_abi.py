"""The C-ABI library builds, loads and exports every entry point that include/isx.h declares;
host-only entry points behave.  No GPU needed."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_13861_gb300 import build as b
    b.build()
    from paper_2402_13861_gb300 import _lib
    return _lib.load()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "isx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(isx_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert "isx_bound_cells" in names and "isx_extract_isosurface" in names
    for n in names:
        assert hasattr(lib, n), n


def test_mc_table_equals_oracle_golden(lib):
    from paper_2402_13861_gb300 import mc_table
    ntri, tris = mc_table()
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "mc_table.txt"))
            if l.strip() and not l.startswith("#")]
    g_ntri = np.array([int(r[1]) for r in rows], dtype=np.int8)
    g_tris = np.array([list(map(int, r[2:])) for r in rows], dtype=np.int8).reshape(256, 5, 3)
    np.testing.assert_array_equal(ntri, g_ntri)
    np.testing.assert_array_equal(tris, g_tris)


def test_argument_errors_without_gpu(lib):
    from paper_2402_13861_gb300 import _lib
    h = C.c_void_p()
    assert lib.isx_create_inr(None, C.byref(h)) == 1
    assert lib.isx_mc_table(None, None) == 1
    assert b"null" in lib.isx_last_error()
    # malformed descriptors are rejected before any device call
    dims = (C.c_int * 3)(3, 64, 2)
    W = (C.POINTER(C.c_float) * 2)()
    desc = _lib.InrDesc(2, dims, W, W)
    assert lib.isx_create_inr(C.byref(desc), C.byref(h)) == 1
    dims = (C.c_int * 3)(3, 20, 1)
    desc = _lib.InrDesc(2, dims, W, W)
    assert lib.isx_create_inr(C.byref(desc), C.byref(h)) == 5
    dims = (C.c_int * 3)(3, 64, 1)
    desc = _lib.InrDesc(2, dims, W, W, 7)                  # no such activation
    assert lib.isx_create_inr(C.byref(desc), C.byref(h)) == 1
    assert b"activation" in lib.isx_last_error()
    assert lib.isx_version() == 100
    # null handles are argument errors on every entry point that takes one; destroying one is a no-op
    assert lib.isx_bound_cells(None, None, None, 0, 0, 0, 0, None, None, None) == 1
    assert lib.isx_bound_cells_noalloc(None, None, None, 0, 0, 0, None, None, None) == 1
    assert lib.isx_eval_points(None, None, 0, 0, None, None) == 1
    assert lib.isx_extract_isosurface(None, None, None, None) == 1
    assert lib.isx_extract_dense(None, None, None, None) == 1
    assert lib.isx_batch_create(None, None, 0, 0, C.byref(h)) == 1
    assert lib.isx_batch_run(None, None, None) == 1
    assert lib.isx_destroy_inr(None) == 0
    assert lib.isx_batch_destroy(None) == 0
    assert lib.isx_proposer_destroy(None) == 0


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """The ctypes mirrors of isx_extract_params, isx_mesh and isx_inr_desc have the C compiler's sizes
    and offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2402_13861_gb300 import _lib
    src = tmp_path / "layout.c"
    fields_p = [f for f, _ in _lib.ExtractParams._fields_]
    fields_m = [f for f, _ in _lib.Mesh._fields_]
    fields_d = [f for f, _ in _lib.InrDesc._fields_]
    body = "\n".join([f'printf("P {f} %zu\\n", offsetof(isx_extract_params, {f}));' for f in fields_p] +
                     [f'printf("M {f} %zu\\n", offsetof(isx_mesh, {f}));' for f in fields_m] +
                     [f'printf("D {f} %zu\\n", offsetof(isx_inr_desc, {f}));' for f in fields_d] +
                     ['printf("SP %zu\\nSM %zu\\nSD %zu\\n", sizeof(isx_extract_params), sizeof(isx_mesh), '
                      'sizeof(isx_inr_desc));'])
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "isx.h"\nint main(void){' + body + 'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    for f in fields_p:
        assert int(out[f"P {f}"]) == getattr(_lib.ExtractParams, f).offset, f
    for f in fields_m:
        assert int(out[f"M {f}"]) == getattr(_lib.Mesh, f).offset, f
    for f in fields_d:
        assert int(out[f"D {f}"]) == getattr(_lib.InrDesc, f).offset, f
    assert int(out["SP"]) == C.sizeof(_lib.ExtractParams) and int(out["SM"]) == C.sizeof(_lib.Mesh)
    assert int(out["SD"]) == C.sizeof(_lib.InrDesc)


def test_proposer_argument_errors_without_gpu(lib):
    h = C.c_void_p()
    f32p = C.POINTER(C.c_float)
    assert lib.isx_proposer_create(None, None, None, C.byref(h)) == 1
    params = np.zeros(8961, dtype=np.float32)
    mean = np.zeros(8, dtype=np.float32)
    std = np.zeros(8, dtype=np.float32)          # std must be > 0
    assert lib.isx_proposer_create(params.ctypes.data_as(f32p), mean.ctypes.data_as(f32p),
                                   std.ctypes.data_as(f32p), C.byref(h)) == 1
    assert b"standard deviation" in lib.isx_last_error()
    assert lib.isx_proposer_predict(None, None, 0, None, None) == 1


def test_c_program_links_against_the_library(tmp_path):
    """A plain C program includes isx.h, links libisx.so and gets argument errors (no GPU call)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2402_13861_gb300 import _lib
    libdir = os.path.dirname(_lib.LIB_PATH)
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include "isx.h"
int main(void) {
  isx_inr h = 0;
  if (isx_version() != 100) return 1;
  if (isx_create_inr(NULL, &h) != ISX_ERR_ARG) return 2;
  int dims[3] = {3, 20, 1};
  const float* W[2] = {0, 0};
  isx_inr_desc d = {2, dims, W, W, ISX_ACT_RELU};
  if (isx_create_inr(&d, &h) != ISX_ERR_UNSUPPORTED) return 3;   /* width 20 */
  printf("%s\n", isx_last_error());
  return 0;
}
""")
    exe = tmp_path / "use"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lisx",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "width" in r.stdout
