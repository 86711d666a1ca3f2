"""The repo arm of bench.py run exactly as the benchmark driver runs it (one GPU, 20 timed steps,
5 warm-up steps): exit code 0 and one JSON line carrying the contract's keys, the roofline of the
dominant kernel, the CPU baseline, the end-to-end figure with its copies, and the store variants."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_driver_command_prints_a_complete_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "1", "--steps", "20", "--warmup", "5"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "step_roofline", "cpu_baseline",
              "e2e", "variants", "gpu_launches", "clocks", "vs_fp64_oracle"):
        assert k in d, k
    assert d["steps"] == 20 and d["warmup"] == 5 and d["n_gpus"] == 1 and d["value"] > 0
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0 < rf["frac"] < 1.5 and rf["peak"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] > 0
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    for st in ("f16", "bf16", "mom"):
        v = d["variants"][st]
        assert v["value"] > 0 and v["phi_mass_drift"] <= 1e-9
    o = d["vs_fp64_oracle"]
    assert o["steps"] >= 1 and o["f32"]["max_dphi"] <= 1e-5 and o["f32"]["max_du"] <= 1e-6
    assert d["gpu_launches"] == 5 * 20
    # the untimed per-kernel split times every pass: the passes add up to about a step
    ks = d["kernels_ms_per_step"]
    assert 0.8 * d["ms_per_step"] <= ks["nci"] + ks["hydro"] + ks["phase"] <= 1.5 * d["ms_per_step"]
    assert abs(ks["hydro"] - rf["avg_ms"]) <= 0.2 * rf["avg_ms"]
    sp = d["split_step"]
    assert all(sp[f"scan_blocks_{b}"]["value"] > 0 and sp[f"scan_blocks_{b}"]["one_stream_value"] > 0
               for b in (38, 76, 152))


@pytest.mark.parametrize("extra", [["--store", "f16"], ["--store", "mom"], ["--lattice", "27"]])
def test_other_stores_and_lattices_print_a_line(extra):
    """The bench's other population stores and the D3Q27 lattice run through the same timed path."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "5", "--warmup", "3", "--no-e2e",
                        "--no-cpu-baseline", "--no-variants", *extra], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["value"] > 0 and d["roofline"]["frac"] > 0
    if extra[1] == "mom":
        assert d["split_step"] is None and d["roofline"]["bytes_per_cell"] == 144
