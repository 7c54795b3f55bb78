"""The Python binding's host side, without a GPU: its enum tables and limits are the C header's, and
the extraction parameters it marshals land in the right fields."""
import os
import re

import numpy as np

from paper_2402_13861_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_constants():
    src = open(os.path.join(ROOT, "include", "isx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {m[0]: int(m[1]) for m in re.findall(r"\b(ISX_[A-Z0-9_]+)\s*=\s*(\d+)", src)}
    consts.update({m[0]: int(m[1]) for m in re.findall(r"#define\s+(ISX_[A-Z0-9_]+)\s+(\d+)", src)})
    return consts


def test_enums_and_limits_match_the_header():
    h = _header_constants()
    assert _lib.MODES == {"sound": h["ISX_BOUND_SOUND"], "clt": h["ISX_BOUND_CLT"], "raua": h["ISX_BOUND_RAUA"],
                          "rafixed": h["ISX_BOUND_RAFIXED"]}
    assert _lib.PRECS == {"fp32": h["ISX_PREC_FP32"], "bf16": h["ISX_PREC_BF16"]}
    assert _lib.ACTS == {"relu": h["ISX_ACT_RELU"], "elu": h["ISX_ACT_ELU"], "sine": h["ISX_ACT_SINE"]}
    for code, name in _lib.STATUS.items():
        assert h[name] == code, name
    assert {n for n in h if n.startswith("ISX_ERR_") or n == "ISX_OK"} == set(_lib.STATUS.values())
    assert (_lib.ISX_MAX_ISO, _lib.ISX_MAX_LEVEL, _lib.ISX_MC_MAX_TRI) == (
        h["ISX_MAX_ISO"], h["ISX_MAX_LEVEL"], h["ISX_MC_MAX_TRI"])


def test_extract_params_marshalling():
    isos = np.array([0.25, -1.5, 3.0], dtype=np.float64)
    p = _lib.Inr.params(7, isos, mode="raua", k=2.5, prec="bf16", inflate=True, bound_stop_level=4,
                        proposer_level=3, tau_lo=0.1, tau_hi=0.9, eval_prec="bf16", kd_tree=True)
    assert (p.max_level, p.n_iso, p.mode, p.prec, p.eval_prec) == (7, 3, _lib.RAUA, _lib.BF16, _lib.BF16)
    assert list(p.iso)[:3] == [0.25, -1.5, 3.0] and all(v == 0.0 for v in list(p.iso)[3:])
    assert abs(p.k - 2.5) == 0.0 and p.inflate == 1 and p.bound_stop_level == 4 and p.kd_tree == 1
    assert p.proposer is None and p.proposer_level == 3
    assert abs(p.tau_lo - 0.1) < 1e-7 and abs(p.tau_hi - 0.9) < 1e-7
    # a scalar iso-value and the defaults: sound, float32 everywhere, every level bounded
    d = _lib.Inr.params(5, 0.5)
    assert (d.n_iso, d.iso[0], d.mode, d.prec, d.eval_prec, d.inflate, d.bound_stop_level, d.kd_tree) == (
        1, 0.5, _lib.SOUND, _lib.FP32, _lib.FP32, 0, -1, 0)


def test_iso_values_are_rounded_to_float32_once():
    """The iso-values travel as float32 (the header's float iso[]): the binding rounds each once."""
    c = 0.1
    p = _lib.Inr.params(3, [c])
    assert p.iso[0] == float(np.float32(c))
