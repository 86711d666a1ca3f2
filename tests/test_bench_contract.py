"""The reference arm of bench.py (the FP64 oracle on the host cores) prints exactly one JSON line with
the keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line(orc):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-budget", "2"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"] and "sample" in d["config"]


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


import pytest  # noqa: E402


@pytest.mark.parametrize("argv", [["--gpus", "1", "--steps", "20", "--warmup", "5"], ["--steps", "1", "--warmup", "0"],
                                  ["--steps", "3", "--warmup", "3"], [], ["--steps", "2000", "--warmup", "20"]])
def test_repo_arm_plan_has_no_negative_step_count(argv):
    """The repo arm's step counts for any --steps/--warmup (the driver runs --steps 20 --warmup 5):
    every count is non-negative and the store variants keep their own fixed horizons."""
    bm = _bench()
    args = bm.parse_args(argv)
    plan = bm.run_plan(args, world=1, rank=0)
    for k, v in plan.items():
        if isinstance(v, int) and not isinstance(v, bool):
            assert v >= 0, (k, v)
    assert plan["timed"] == args.steps and plan["warmup"] == args.warmup
    assert plan["variant_stores"] == ("f16", "bf16", "mom")
    assert plan["early"] == bm.EARLY and plan["late"] == bm.LATE and bm.EARLY < bm.LATE
    assert plan["variant_timed"] >= 1 and plan["split_steps"] >= 1 and plan["e2e_steps"] >= 1
    assert plan["split_compare_steps"] >= 1
    assert plan["cpu_baseline"] is True
    # other ranks and multi-GPU runs skip the variants and the CPU baseline
    p2 = bm.run_plan(args, world=2, rank=1)
    assert p2["variant_stores"] == () and p2["cpu_baseline"] is False


def test_repo_arm_rejects_bad_step_counts():
    bm = _bench()
    for argv in (["--steps", "0"], ["--warmup", "-1"]):
        with pytest.raises(SystemExit):
            bm.parse_args(argv)
