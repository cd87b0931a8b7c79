"""The benchmark's reference arm (the CPU oracle on a bounded sample of the
benchmark workload) keeps the one-line JSON contract: the cxbwt arm's metric,
unit and workload, a cpu_baseline describing the run, and an e2e object with
no host-device copies.  Ranks other than 0 print nothing and exit 0.  No GPU
is needed: this arm runs only the oracle."""
import argparse
import io
import json
import os
import subprocess
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    import bench
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                          "--cpu-sample-reads", "2000"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["data"] == "synthetic"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # The same workload string as the cxbwt arm's benchmark line.
    desc, _, lens = bench.load_workload("genome-like", 0, 0)
    assert line["config"]["workload"] == desc.format(n=lens.size, N=int(lens.sum()) + lens.size)
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"] and cpu["unit"] == line["unit"]
    assert cpu["cores"] >= 1 and "2,000 reads" in cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    import bench
    args = argparse.Namespace(impl="reference", steps=1, warmup=3, cpu_sample_reads=2000,
                              workload="genome-like", reads=0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(args, rank=1, world=2)
    assert rc == 0 and buf.getvalue() == ""
