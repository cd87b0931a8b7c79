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
    # The same workload string as the cxbwt arm's benchmark line (the
    # repeat-rich collection, of which only the sample's reads are drawn).
    assert line["config"]["workload"] == bench.WORKLOADS["repeat-rich"].format(n=50_000_000, N=5_050_000_000)
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"] and cpu["unit"] == line["unit"]
    assert cpu["cores"] >= 1 and "2,000 reads" in cpu["sample"]
    assert isinstance(cpu["cpu_model"], str) and cpu["cpu_model"]
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


def test_phase_rates_against_each_phase_bytes():
    """The per-phase figures of the benchmark line, from the library's
    counters over two builds of 1M reads x 100 bp with 32-bit ids."""
    import bench
    n, bases, steps = 1_000_000, 100_000_000, 2
    N = n + bases
    st = {"sort_pass_ms": 2 * 2.61, "group_ms": 2 * 1.69, "emit_ms": 2 * 0.37, "build_ms": 2 * 4.84,
          "sort_pass_items": 2 * 4 * N, "carried_pass_ms": 2 * 1.9, "carried_pass_items": 2 * 3 * N, "slices": 2}
    ph = bench.phase_rates(st, steps, n, bases, 4, 6792.0)
    assert set(ph) == {"digit_passes", "carried_passes", "generating_passes", "group_finish", "emission",
                       "histograms_and_planning"}
    assert abs(ph["digit_passes"]["bytes_per_step"] - 16 * 4 * N) < 1
    assert abs(ph["digit_passes"]["gbs"] - 16 * 4 * N / 2.61e-3 / 1e9) < 1e-6
    # One generating pass (ids and keys written, the store read) and three carried ones per build.
    assert abs(ph["carried_passes"]["bytes_per_step"] - 16 * 3 * N) < 1
    assert abs(ph["generating_passes"]["bytes_per_step"] - (8 * N + bases / 4)) < 1
    assert abs(ph["generating_passes"]["ms_per_step"] - (2.61 - 1.9)) < 1e-9
    assert abs(ph["group_finish"]["bytes_per_step"] - 12 * N) < 1
    assert abs(ph["emission"]["bytes_per_step"] - (4 * N + N / 4 + 8 * n + bases / 4)) < 1
    assert abs(ph["histograms_and_planning"]["ms_per_step"] - (4.84 - 2.61 - 1.69 - 0.37)) < 1e-9
    for v in ph.values():
        assert abs(v["frac_of_hbm"] - v["gbs"] / 6792.0) < 1e-12
    # A plan without a group finish (every digit by LSD passes) reports no such phase.
    st["group_ms"] = 0.0
    assert "group_finish" not in bench.phase_rates(st, steps, n, bases, 4, 6792.0)


class _FakeNvml:
    """Answers the read-only NVML queries the clock sampler makes."""

    def __init__(self):
        self.shutdown = 0

    def nvmlInit_v2(self):
        return 0

    def nvmlShutdown(self):
        self.shutdown += 1
        return 0

    def nvmlDeviceGetHandleByPciBusId_v2(self, bus, handle):
        self.bus = bus
        return 0

    def nvmlDeviceGetMaxClockInfo(self, handle, kind, out):
        out._obj.value = 2070
        return 0

    def nvmlDeviceGetClockInfo(self, handle, kind, out):
        out._obj.value = 1965
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, handle, out):
        out._obj.value = 0x4 | 0x1  # power cap, idle (not reported)
        return 0


def test_clock_sampler_reads_nvml(monkeypatch):
    import ctypes
    import time

    import bench
    fake = _FakeNvml()
    monkeypatch.setattr(ctypes, "CDLL", lambda name: fake)
    with bench.ClockSampler("00000000:1B:00.0", period_s=0.001) as c:
        time.sleep(0.05)
    s = c.summary()
    assert fake.shutdown == 1 and fake.bus == b"00000000:1B:00.0"
    assert s["samples"] >= 5 and s["sm_mhz"] == 1965 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["source"].startswith("nvml")


def test_clock_sampler_without_nvml_or_smi(monkeypatch):
    """No NVML library and no nvidia-smi (this host): no record, no error."""
    import ctypes

    import bench

    def missing(name):
        raise OSError(name)

    monkeypatch.setattr(ctypes, "CDLL", missing)
    monkeypatch.setenv("PATH", "/nonexistent")
    with bench.ClockSampler(0) as c:
        pass
    assert c.summary() is None and c.path is None  # no temporary file left behind


def test_summarize_clocks():
    import bench
    rows = [(2070.0, 2070.0, set()), (1900.0, 2070.0, {"sw_power_cap"}), (2000.0, 2070.0, set())]
    s = bench.summarize_clocks(rows, "x")
    assert s == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"], "source": "x"}
    assert bench.summarize_clocks([], "x") is None


def test_smaller_copy_of_a_workload_keeps_its_coverage():
    """--genome-mbp with --reads draws a smaller copy of a workload at the
    coverage the reads give (for profiling captures); the description names
    the genome it was drawn from, and the default draw is unchanged."""
    import bench
    from paper_1401_7457_gb300 import synth
    desc, codes, lens = bench.load_workload("repeat-rich", 0, 4000, 8_000)
    assert "8000 Mbp" not in desc and "0.008 Mbp" in desc and "100 Mbp" not in desc
    assert lens.size == 4000 and int(lens.sum()) == codes.size == 400_000
    want_codes, want_lens = synth.repeat_rich(seed=3, n_reads=4000, genome_size=8_000)
    assert (codes == want_codes).all() and (lens == want_lens).all()
    desc0, codes0, _ = bench.load_workload("repeat-rich", 0, 4000)
    assert desc0 == bench.WORKLOADS["repeat-rich"]
    assert (codes0 == synth.repeat_rich(seed=3, n_reads=4000)[0]).all()
    desc_gl, _, lens_gl = bench.load_workload("genome-like", 0, 2000, 20_000)
    assert "0.02 Mbp" in desc_gl and lens_gl.size == 2000
