"""Host-side parts of bench.py, without a GPU: the reference arm's JSON line
(the oracle timed on the host cores), the roofline helpers, and the rule that
the committed ncu traffic figure is used only for the kernel source it was
taken from."""

import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CONTRACT_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config")


def _run_reference(env=None):
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run_reference()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in CONTRACT_KEYS:
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "GCUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = _run_reference(env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_pipe_peaks():
    # int16: 64 cells/clk/SM; FP32: 128/3 cells/clk/SM (152 SMs, 2070 MHz)
    assert bench.alu_peak_gcups(152, 2070.0, "int16") == pytest.approx(152 * 64 * 2.07)
    assert bench.alu_peak_gcups(152, 2070.0, "fp32") == pytest.approx(152 * 128 / 3 * 2.07)


def test_dram_rate():
    # 10 MB per batch; 1e11 cells at 1e4 GCUPS is a 10 ms sweep -> 1 GB/s
    d = bench.dram_rate(1.0e7, 1.0e11, 1.0e4)
    assert d["dram_gbs"] == pytest.approx(1.0)
    if d["hbm_peak_gbs"]:
        assert d["dram_frac_of_hbm"] == pytest.approx(1.0 / d["hbm_peak_gbs"])
    assert bench.dram_rate(None, 1.0e11, 1.0e4) == {"dram_gbs": None}


def test_traffic_figure_follows_the_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2211_07340_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "sdtw_kernels.cuh").write_bytes(b"// kernels\n")
    (csrc / "haru_internal.h").write_bytes(b"// internal\n")
    sha = hashlib.sha1(b"// kernels\n// internal\n").hexdigest()
    (tmp_path / "profiles" / "sdtw_sweep_sars_uneven_8192.md").write_text(
        "# summary\n\nFigures:\n\n"
        "    traffic_bytes_per_step_int16: 123\n"
        "    traffic_bytes_per_step_fp32: 456\n"
        f"    kernel_source_sha1: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("int16") == 123.0
    assert bench.profiled_traffic("fp32") == 456.0
    (csrc / "sdtw_kernels.cuh").write_bytes(b"// kernels, changed\n")
    assert bench.profiled_traffic("int16") is None


def test_committed_traffic_figure_is_well_formed():
    # the committed summary carries both figures and a 40-hex-digit source hash
    vals = {}
    with open(os.path.join(ROOT, "profiles", "sdtw_sweep_sars_uneven_8192.md")) as f:
        for line in f:
            if ":" in line and line.startswith("    "):
                k, v = line.strip().split(":", 1)
                vals[k.strip()] = v.strip()
    assert int(vals["traffic_bytes_per_step_int16"]) > 0
    assert int(vals["traffic_bytes_per_step_fp32"]) > 0
    assert len(vals["kernel_source_sha1"]) == 40
