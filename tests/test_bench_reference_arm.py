"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints the one JSON line of the benchmark contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["unit"] == "time-steps/s"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_extras_are_checked_against_the_oracle_in_the_cpu_baseline_leg():
    """bench.py's extras hand their GPU results to oracle_checks (run only in
    the CPU-baseline leg); here with stand-in results: the exact oracle output
    gives 0, a perturbed one its relative error, several checks under one key
    keep the largest, and an extra that failed keeps its error."""
    import sys
    import numpy as np
    import oracle
    from paper_2512_13319_gb300 import synth
    sys.path.insert(0, ROOT)
    import bench

    model = synth.wiener_velocity(2)
    _, y = synth.simulate(model, 200, 0.01, seed=3)
    x = oracle.smooth_lti(model, y, 0.01)
    out = {"a": {"ms": 1.0}, "b": {"ms": 1.0}, "c": {"error": "RuntimeError: x"}}
    checks = [("a", "rel_err_vs_oracle", "smooth_lti", (model, y, 0.01), x),
              ("b", "max_err", "smooth_lti", (model, y, 0.01), x),
              ("b", "max_err", "smooth_lti", (model, y, 0.01), 1.01 * x),
              ("c", "rel_err_vs_oracle", "smooth_lti", (model, y, 0.01), x)]
    bench.oracle_checks(out, checks)
    assert out["a"]["rel_err_vs_oracle"] == 0.0
    assert abs(out["b"]["max_err"] - 0.01) < 1e-12
    assert "rel_err_vs_oracle" not in out["c"]
