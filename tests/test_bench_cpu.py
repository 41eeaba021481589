"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract; small inputs keep these runs to a few seconds."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"] + args,
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def _check(line, workload):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["config"]["workload"] == workload
    assert line["value"] > 0 and line["unit"] == "points/s" and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_one_set():
    line = _run(["--n", "2500", "--steps", "1", "--warmup", "0"])
    _check(line, "blobs_n100k_d64")
    # one measured oracle run on the whole workload: no scaling law
    assert "the whole workload" in line["cpu_baseline"]["sample"] and "not scaled" in line["cpu_baseline"]["sample"]
    n = line["config"]["n"]
    assert n == 2500 and line["ms_per_step"] == pytest.approx(n / line["value"] * 1000.0, rel=1e-9)
    assert line["steps"] == 1 and line["warmup"] == 0


def test_reference_arm_batched():
    line = _run(["--workload", "batched_4096_d32", "--nsets", "6", "--steps", "1", "--warmup", "0"])
    _check(line, "batched_4096_d32")
    assert line["config"]["nsets"] == 6
    assert "not scaled" in line["cpu_baseline"]["sample"]


def test_reference_arm_moons_is_measured_whole():
    line = _run(["--workload", "moons_n20k_d128", "--n", "600", "--steps", "2", "--warmup", "1"])
    _check(line, "moons_n20k_d128")
    assert line["config"]["n"] == 600 and "not scaled" in line["cpu_baseline"]["sample"]


def test_omega_gram_roofline_reports_scaled_traffic():
    """The Gram-path roofline (host arithmetic only): the slower kernel is the
    line's, its DRAM traffic is the capture's bytes per unit times the run's
    units at the captured row length, and null at another one."""
    sys.path.insert(0, ROOT)
    import bench
    prof = [{"omega_gram_ms": 7.5, "omega_gram_blocks": 146222, "omega_gram_direct_pairs": 30836874}]
    peaks = {"bf16_tflops": 1940.5}
    r = bench.omega_gram_roofline(prof, peaks, "measured", 40.27, 152, 24.5, 285302, 64, 7.65e11)
    assert r["kernel"].startswith("k_weights_sym") and r["bound"] == "alu"
    assert r["traffic"] == pytest.approx(285302 * (1.504621e9 + 0.045260e9) / 42831)
    assert r["other_kernel"]["traffic"] == pytest.approx(146222 * (0.236092e9 + 1.348661e9) / 22524)
    assert 0.0 < r["frac"] < 1.0 and r["other_kernel"]["bound"] == "tensor"
    r2 = bench.omega_gram_roofline(prof, peaks, "measured", 40.27, 152, 24.5, 285302, 128, 7.65e11)
    assert r2["traffic"] is None and r2["other_kernel"]["traffic"] is None
