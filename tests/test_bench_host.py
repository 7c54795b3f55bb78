"""Host-side logic of bench.py that needs no GPU: the clock-sample parser, the ncu traffic record
lookup (keyed to the kernel source it was captured on) and the oracle arm's JSON line."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(lines, tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.f = open(s.path, "a")
    s.proc = _FakeProc()
    return s


def test_clock_parser_median_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = _sampler_with(rows, tmp_path).stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_parser_flags_thermal(tmp_path):
    rows = ["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"]
    out = _sampler_with(rows, tmp_path).stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    s = bench.ClockSampler(0)
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
    # started where nvidia-smi cannot run: unsampled, and its temporary file is gone
    monkeypatch.setenv("PATH", "/nonexistent")
    s = bench.ClockSampler(0)
    s.start()
    path = s.path
    assert os.path.exists(path)
    assert s.stop()["reasons"] == ["unsampled"]
    assert not os.path.exists(path)


def test_traffic_record_is_keyed_to_the_source(tmp_path):
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert "rows_gemm" in rec and rec["rows_gemm"]["dram_per_alg_byte"] > 0
    # another source (an edited kernel) drops the record
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    assert bench.traffic_record("rows_gemm", str(src)) is None
    assert bench.traffic_record("no_such_kernel", str(src)) is None
    cur = os.path.join(ROOT, "paper_2402_13861_gb300", "csrc", "rows_gemm.cu")
    got = bench.traffic_record("rows_gemm", cur)
    if got is not None:
        assert got["src_sha"] == hashlib.sha256(open(cur, "rb").read()).hexdigest()[:16]


def test_job_totals_single_rank():
    assert bench.job_totals(12.5, 1000, 1, "cpu") == (12.5, 1000.0)


def test_reference_line_shape(monkeypatch, capsys):
    """The oracle arm prints one JSON line with the contract's keys (the oracle itself is replaced
    by a stub sample here so that the test takes no CPU time)."""
    monkeypatch.setattr(bench, "cpu_baseline", lambda layers, mode, k, budget_s=12.0, single_thread=True: {
        "value": 100.0, "unit": "cells/s", "cores": 2, "kind": "oracle", "sample": "stub"})
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "0"])
    args = bench.parse()
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["value"] == pytest.approx(100.0)
    assert line["ms_per_step"] >= 0.0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_kernel_rooflines_of_the_row_path():
    """Launch accounting shaped like a 512^3 extraction on the row path: the reduction pass (bytes
    only) is HBM-bound, the row GEMM (w / 2 FLOP per byte, below the ridge) too, the split GEMM
    (FLOPs only) is measured against the tensor peak, and kernels without counts get no bound."""
    stats = {
        "rows_reduce": dict(launches=936, ms=540.0, flops=0.0, bytes=1.2e12),
        "rows_gemm": dict(launches=936, ms=516.0, flops=2.1e14, bytes=1.64e12),
        "rows_split": dict(launches=936, ms=262.0, flops=5.0e13, bytes=0.0),
        "rows_new": dict(launches=936, ms=259.0, flops=0.0, bytes=0.0),
        "rows_out": dict(launches=234, ms=220.0, flops=1.0e12, bytes=0.0),
        "eval_tc": dict(launches=1, ms=44.0, flops=3.0e13, bytes=0.0),
    }
    out = bench.kernel_rooflines(stats, 6674.2, 1701.1, 80.5)
    assert [e["kernel"] for e in out] == ["rows_reduce", "rows_gemm", "rows_split", "rows_new", "rows_out"]
    assert abs(sum(v["ms"] for v in stats.values()) * out[0]["share"] - 540.0) < 1.0
    red, gemm, split, new, outp = out
    assert red["bound"] == "hbm" and red["achieved"] == pytest.approx(1.2e12 / 0.54 / 1e9)
    assert red["frac"] == pytest.approx(red["achieved"] / 6674.2)
    assert gemm["bound"] == "hbm" and gemm["achieved"] == pytest.approx(1.64e12 / 0.516 / 1e9)
    assert split["bound"] == "tensor" and split["unit"] == "TFLOP/s" and "note" in split
    assert split["achieved"] == pytest.approx(5.0e13 / 0.262 / 1e12)
    assert new["bound"] is None and "frac" not in new
    assert outp["bound"] == "alu" and outp["peak"] == 80.5
    json.dumps(out)
    # a contraction above the ridge is compute-bound
    hot = bench.kernel_rooflines({"rows_gemm": dict(launches=1, ms=1.0, flops=1e12, bytes=1e9)}, 6674.2, 1701.1, 80.5)
    assert hot[0]["bound"] == "tensor"
    assert bench.kernel_rooflines({}, 6674.2, 1701.1, 80.5) == []


def test_clock_sampler_with_a_fake_nvidia_smi(tmp_path, monkeypatch):
    """start / stop around a stand-in nvidia-smi that prints two samples and keeps running."""
    exe = tmp_path / "nvidia-smi"
    exe.write_text("#!/bin/sh\n"
                   "echo '0, 2055, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                   "echo '0, 2070, 2070, 1180.0, 0x0, Not Active, Not Active, Not Active, Active'\n"
                   "exec sleep 30\n")
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    import time
    for _ in range(50):
        if os.path.getsize(s.path) > 0 and open(s.path).read().count("\n") >= 2:
            break
        time.sleep(0.05)
    path = s.path
    out = s.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == pytest.approx(2062.5) and out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(path)
