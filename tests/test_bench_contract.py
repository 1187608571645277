"""bench.py's output contract on the CPU: the reference arm (the oracle, timed
on the host) prints one JSON line with the keys and types the benchmark
line requires, workloads without an oracle arm print a one-line
`unavailable`, and fewer than 3 warm-up steps are refused.  No GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                       text=True, cwd=ROOT, timeout=300)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return r.returncode, (json.loads(lines[-1]) if lines else None), r.stderr


def test_reference_line_keys():
    rc, d, err = _run("--impl", "reference", "--workload", "ksat3_n50_m215_b1", "--steps", "2", "--warmup", "3")
    assert rc == 0, err
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "fwd+bwd literal-evals/s"
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == "literal-evals/s" and d["vs_baseline"] is None
    assert d["config"]["workload"] == "ksat3_n50_m215_b1"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_workloads_without_an_oracle_arm():
    for w in ("structured_cost_time", "next_rows_loss_partial"):
        rc, d, err = _run("--impl", "reference", "--workload", w)
        assert rc == 0, err
        assert d["impl"] == "reference" and isinstance(d["unavailable"], str) and d["unavailable"]


def test_fewer_than_three_warmup_steps_are_refused():
    rc, d, err = _run("--warmup", "2")
    assert rc == 2 and d is None and "warmup" in err
