"""The benchmark's host-side arms (no GPU): the reference arm (the FP64 oracle on the host cores,
`bench.py --impl reference`) and the oracle timer behind `cpu_baseline` print positive rates and
the keys the benchmark's JSON line carries, even for runs short enough that the y0
initialisation, which every oracle run repeats, is comparable to the timed steps."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["unit"] == "chain-steps/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    for k in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "dtype", "data", "config"):
        assert k in line, k
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


@pytest.mark.parametrize("q", [1, 2])
def test_cpu_baseline_is_positive(oracle_mod, q):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2501_17334_gb300 import workload as W
    r = bench.cpu_baseline(oracle_mod, W.config_problem(q), 0.5, label=f"{q}-qubit", max_steps=200)
    assert r["value"] > 0 and r["cores"] >= 1 and r["kind"] == "oracle"
