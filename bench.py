"""Benchmark: BWT build throughput (Gbase/s) of one read collection per GPU.

Workload (N=1 default): the repeat-rich collection, 50M reads x 100 bp
sampled from both strands of a seeded 100 Mbp random genome in which 5% of
the sequence is 10-copy 1 kb repeats at 0.5% divergence, with 1%
substitutions (50x coverage): 5.05G suffixes, more than one 32-bit-row
slice, so the build runs in device-memory-bounded bucket slices (Figure 2
of the paper) with 64-bit suffix ids.  One step = one whole ``cxbwt_build``
(histograms, every radix pass of every slice, group finish, emission) on
device-resident input.  ``value`` = bases of all ranks / max over ranks of
the summed device time of K steps (CUDA events on the build stream; L2
flushed by a 512 MB write between steps, outside the timed events; the
working set, about 100 GB, is far larger than L2 anyway).

Extra keys: ``e2e`` (same metric through the C ABI with pinned host buffers,
input copy and the streamed BWT, $ rows and counts inside the timed region),
``roofline`` of the dominant kernel (the onesweep carried-key digit pass:
key and id read and written, 24 B per item with 64-bit ids, each pass timed
live between the library's own CUDA events), ``phases`` (every phase of a
build against its own algorithmic bytes), ``cpu_baseline`` (the oracle on a
bounded sample on this host's cores, rank 0 only), ``clocks`` (sampled during
the timed region), ``gpu_launches`` and ``config2`` (the same measurement on
the genome-like collection: 1M reads x 100 bp from a 5 Mbp genome at 20x).

``--impl reference`` times the CPU oracle instead (the reference arm of this
method is the definition itself): each step sorts a bounded sample of the same
workload on all host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BWT build Gbases/s at 1 GB300 (% HBM roofline); served p50/p99 vs plain loop"
UNIT = "Gbase/s"
WORKLOAD = ("genome-like: {n:,} reads x 100 bp from both strands of a seeded 5 Mbp uniform genome "
            "(1M reads = 20x coverage), 1% substitutions, seed 2; {N:,} suffixes")
WORKLOAD_READS = {"genome-like": 1_000_000, "repeat-rich": 50_000_000, "tiny": 10_000}
WORKLOADS = {
    "genome-like": WORKLOAD,
    "repeat-rich": ("repeat-rich: {n:,} reads x 100 bp from a seeded 100 Mbp genome, 5% in 10-copy 1 kb repeats "
                    "at 0.5% divergence, both strands, 1% substitutions, seed 3; {N:,} suffixes"),
    "tiny": "tiny: {n:,} reads x 100 bp, i.i.d. uniform bases, seed 1; {N:,} suffixes",
}


# Reads are drawn in chunks of this many (synth.sample_reads): a draw of a
# multiple of it starts with exactly the reads of any larger draw, so the CPU
# samples below are the workload's own first reads without drawing it whole.
SAMPLE_CHUNK = 1 << 17


def load_workload(name, rank=0, n_reads=0, genome_bp=0):
    """(description, codes, lens) of a workload; rank > 0 draws an independent collection of the same shape.
    genome_bp > 0 replaces the genome size of the genome-like and repeat-rich workloads (a smaller copy
    of a workload at its own coverage, for profiling captures)."""
    from paper_1401_7457_gb300 import synth
    desc = WORKLOADS[name]
    if name == "genome-like":
        seed = 2 if rank == 0 else synth.derive_seed(2, rank)
        codes, lens = synth.genome_like(seed=seed, n_reads=n_reads or 1_000_000, genome_size=genome_bp or 5_000_000)
    elif name == "repeat-rich":
        seed = 3 if rank == 0 else synth.derive_seed(3, rank)
        codes, lens = synth.repeat_rich(seed=seed, n_reads=n_reads or 50_000_000,
                                        genome_size=genome_bp or 100_000_000)
    else:
        seed = 1 if rank == 0 else synth.derive_seed(1, rank)
        codes, lens = synth.uniform_reads(n_reads or 10_000, 100, seed)
    if genome_bp and name in ("genome-like", "repeat-rich"):
        desc = desc.replace("5 Mbp" if name == "genome-like" else "100 Mbp", f"{genome_bp / 1e6:g} Mbp")
    return desc, codes, lens


# ncu summaries of the carried-key digit pass, by suffix id width.
PROFILES = {4: os.path.join(ROOT, "profiles", "onesweep_digit_pass_genome_like.md"),
            8: os.path.join(ROOT, "profiles", "onesweep_carried_pass_repeat_rich.md")}
KERNEL_SRC = os.path.join(ROOT, "paper_1401_7457_gb300", "csrc", "onesweep.cuh")
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def id_bytes(n_reads: int, read_len: int, store_bytes: int) -> int:
    """Suffix id width the library picks for reads of one length: (read, k)
    in 32 bits when they fit, plus two bits for the preceding base when the
    store is larger than 64 MB (and those still fit)."""
    len_bits = max(read_len, 1).bit_length()
    sym = 2 if store_bytes > (64 << 20) else 0
    if sym and (n_reads - 1) < (1 << (32 - len_bits - sym)):
        return 4
    return 4 if (n_reads - 1) < (1 << (32 - len_bits)) else 8


def profiled_traffic(idb):
    """DRAM bytes per item of the carried-key digit pass with idb-byte ids
    from the committed ncu summary, or None when that summary is missing or
    the kernel source changed since it was taken."""
    try:
        text = open(PROFILES[idb]).read()
    except OSError:
        return None
    m = re.search(r"dram_bytes_per_item:\s*([0-9.]+)", text)
    s = re.search(r"k_sort_sha256:\s*([0-9a-f]+)", text)
    if not m or not s:
        return None
    cur = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    if not cur.startswith(s.group(1)):
        return None
    return float(m.group(1))


# Clock-event reason bits of NVML (nvml.h), under the names nvidia-smi uses.
NVML_REASONS = {"hw_slowdown": 0x8 | 0x80, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                "sw_power_cap": 0x4}
NVML_CLOCK_SM = 1


def summarize_clocks(rows, source):
    """rows: (sm_mhz, sm_max_mhz, reasons) samples; reasons a set of names."""
    if not rows:
        return None
    return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
            "samples": len(rows), "reasons": sorted(set().union(*(r[2] for r in rows))), "source": source}


class ClockSampler:
    """SM clock and clock-event reasons during a timed region.  NVML is read
    (read-only queries) from a thread every 5 ms; where NVML cannot be loaded,
    nvidia-smi samples every 200 ms (too coarse for a region of a few tens
    of milliseconds, hence NVML first)."""

    def __init__(self, gpu, period_s: float = 0.005):
        self.gpu = gpu  # NVML / nvidia-smi id: a PCI bus id string, or an index
        self.period = period_s
        self.rows = []
        self.source = None
        self.proc = None
        self.path = None
        self.thread = None

    def __enter__(self):
        if not self._start_nvml():
            self._start_smi()
        return self

    def _start_nvml(self):
        import ctypes
        import threading
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            reasons = (getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
                       or lib.nvmlDeviceGetCurrentClocksThrottleReasons)
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            mx = ctypes.c_uint()
            if isinstance(self.gpu, str):
                found = lib.nvmlDeviceGetHandleByPciBusId_v2(self.gpu.encode(), ctypes.byref(h))
            else:
                found = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h))
            if found != 0 or lib.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx)) != 0:
                lib.nvmlShutdown()
                return False
        except (OSError, AttributeError):
            return False
        self.lib = lib
        self.stop = threading.Event()

        def loop():
            clk, r = ctypes.c_uint(), ctypes.c_ulonglong()
            while not self.stop.is_set():
                if (lib.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(clk)) == 0
                        and reasons(h, ctypes.byref(r)) == 0):
                    names = {k for k, bits in NVML_REASONS.items() if r.value & bits}
                    self.rows.append((float(clk.value), float(mx.value), names))
                self.stop.wait(self.period)

        self.source = f"nvml every {self.period * 1e3:g} ms"
        self.thread = threading.Thread(target=loop, daemon=True)
        self.thread.start()
        return True

    def _start_smi(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi every 200 ms"
        except Exception:
            self.proc = None
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
            self.path = None

    def __exit__(self, *exc):
        if self.thread:
            self.stop.set()
            self.thread.join()
            self.lib.nvmlShutdown()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.thread:
            return summarize_clocks(self.rows, self.source)
        if not self.proc or not self.path:
            return None
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                flags = {names[i] for i, f in enumerate(parts[5:9]) if f.lower().startswith("active")}
                rows.append((float(parts[1]), float(parts[2]), flags))
            except ValueError:
                continue
        os.unlink(self.path)
        return summarize_clocks(rows, self.source)


def nvml_id(dev):
    """The GPU's PCI bus id, as NVML and nvidia-smi name it (their indices
    differ from CUDA's when CUDA_VISIBLE_DEVICES is set), or the CUDA index
    when torch does not report the bus."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except AttributeError:
        return dev.index


def aggregate(dist, local_ms, bases_per_rank, world, steps):
    """Whole-job throughput: bases of all ranks / the slowest rank's time.
    Returns (gbase_per_s, max_ms).  With world == 1 no collective is used."""
    total = local_ms
    if world > 1:
        import torch
        t = torch.tensor([local_ms], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return bases_per_rank * world * steps / (total * 1e-3) / 1e9, total


def phase_rates(st, steps, n_reads, bases, idb, peak):
    """Device time of each phase of one build and its bandwidth against the
    phase's own algorithmic bytes (N = bases + n_reads suffixes, idb = bytes
    of a suffix id):

    * digit passes: key (4 B) and id read and written, per item of each pass;
    * group finish: the window key and the id of every suffix read, the id
      written;
    * emission: the id of every suffix read, its 2-bit symbol written, 8 B per
      $ row, the read store (a quarter byte per base) read once;
    * histograms and planning (the rest of the build): the read store and the
      read lengths read once.

    st holds the library's counters over `steps` builds (timing enabled).  A
    phase that did not run (no time) is left out."""
    N = bases + n_reads
    sort_ms = st["sort_pass_ms"] / steps
    group_ms = st["group_ms"] / steps
    emit_ms = st["emit_ms"] / steps
    rest_ms = st["build_ms"] / steps - sort_ms - group_ms - emit_ms
    carried_ms = st["carried_pass_ms"] / steps
    gen_items = (st["sort_pass_items"] - st["carried_pass_items"]) / steps
    slices = st["slices"] / steps
    model = {"digit_passes": (sort_ms, (8 + 2 * idb) * st["sort_pass_items"] / steps),
             # carried-key passes: key and id read and written
             "carried_passes": (carried_ms, (8 + 2 * idb) * st["carried_pass_items"] / steps),
             # passes that make the ids (generated in the first pass of each
             # slice) or gather a key window: key and id written, the store
             # read once per slice
             "generating_passes": (sort_ms - carried_ms, (4 + idb) * gen_items + slices * bases / 4),
             "group_finish": (group_ms, (4 + 2 * idb) * N),
             "emission": (emit_ms, idb * N + N / 4 + 8 * n_reads + bases / 4),
             "histograms_and_planning": (rest_ms, bases / 4 + 4 * n_reads)}
    out = {}
    for name, (ms, nbytes) in model.items():
        if ms <= 0:
            continue
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_step": ms, "bytes_per_step": nbytes, "gbs": gbs, "frac_of_hbm": gbs / peak}
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_oracle_rate(codes, lens, n_sample_reads, threads):
    """Oracle throughput on the first n_sample_reads reads: (Gbase/s, seconds, bases)."""
    import oracle
    n_s = min(n_sample_reads, lens.size)
    sc, sl = codes[:int(lens[:n_s].sum())], lens[:n_s]
    col = oracle.Collection(sc, sl)
    t0 = time.perf_counter()
    oracle.sort(col, threads=threads)
    dt = time.perf_counter() - t0
    bases = int(sl.sum())
    return bases / dt / 1e9, dt, bases


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on a bounded sample of the workload per step."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_sample = args.cpu_sample_reads
    # Only the sample's reads are drawn (a whole number of draw chunks: the
    # workload's own first reads); the description names the whole workload.
    n_full = args.reads or WORKLOAD_READS[args.workload]
    desc = WORKLOADS[args.workload]
    _, codes, lens = load_workload(args.workload, 0, min(n_full, -(-n_sample // SAMPLE_CHUNK) * SAMPLE_CHUNK))
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_rate(codes, lens, n_sample // 4, threads)
    times = []
    bases = 0
    for _ in range(args.steps):
        _, dt, bases = cpu_oracle_rate(codes, lens, n_sample, threads)
        times.append(dt)
    total = sum(times)
    value = bases * args.steps / total / 1e9
    sample = f"first {n_sample:,} reads ({bases:,} bases) of the workload per step, std::sort / parallel-mode sort"
    L = int(lens[0])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": desc.format(n=n_full, N=n_full * (L + 1))},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch_bench(args, rank, world):
    """The batched workload: 256 collections (n log-uniform in [10k, 2M], read
    length from {36, 76, 100, 150}, genome-like reads).  The autotuner first
    picks the tile and the sort plan for each (read length, size class) that
    occurs, on the first collection of that class; then cxbwt_build_batch is
    timed against the plain loop of one cxbwt_build per collection, both with
    the tuned plans, on device-resident inputs and outputs.  Every result of
    both is compared with the oracle's stored digest of its collection.  One
    JSON line (not the benchmark's default workload)."""
    import torch

    from paper_1401_7457_gb300 import binding, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    specs = synth.batch_specs()
    if args.reads:
        specs = specs[:args.reads]
    want = oracle_item_digests("batched")
    colls, bases, suffixes = [], 0, 0
    for sp in specs:
        codes, lens = synth.batch_collection(sp)
        words = binding.pack_codes(codes)
        N = int(lens.sum()) + lens.size
        colls.append((torch.from_numpy(words.view(np.int32)).to(dev), torch.from_numpy(lens.view(np.int32)).to(dev),
                      torch.zeros((N + 15) // 16, dtype=torch.int32, device=dev),
                      torch.zeros(lens.size, dtype=torch.int64, device=dev),
                      torch.zeros(5, dtype=torch.int64, device=dev)))
        bases += int(lens.sum())
        suffixes += N
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(device=0, budget_bytes=int(args.budget_gb * (1 << 30)))
    # Autotune each (read length, size class) on its first collection.
    picks, t0 = {}, time.perf_counter()
    for sp, c in zip(specs, colls):
        cls = (sp["length"], (int(c[1].numel()) * (sp["length"] + 1)).bit_length())
        if cls not in picks:
            picks[cls] = ctx.autotune(c[0], c[1], c[2], c[3], stream=stream)
    tune_s = time.perf_counter() - t0
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def plain():
        for c in colls:
            ctx.build(*c, stream=stream)

    def batched():
        ctx.build_batch(colls, stream=stream)

    def check():
        if want is None:
            return None
        torch.cuda.synchronize()
        ok = all(packed_digest(c[2].cpu().numpy().view(np.uint32), c[3].cpu().numpy(), c[4].cpu().numpy()) == d
                 for c, d in zip(colls, want))
        for c in colls:
            for t in c[2:]:
                t.zero_()
        return ok

    out, equal = {}, {}
    for name, fn in (("plain", plain), ("batched", batched)):
        for _ in range(max(args.warmup, 1)):
            fn()
        equal[name] = check()
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[name] = sum(ts) / len(ts)
        equal[name] = equal[name] and check() if equal[name] is not None else None
    ctx.close()
    chosen = {}
    for (L, cls), t in sorted(picks.items()):
        plan = f"groups l={t['prefix_len']}" if t['algorithm'] == 2 else "lsd"
        k = f"tile {t['tile_items']}, {plan}"
        chosen[k] = chosen.get(k, 0) + 1
    line = {"metric": METRIC, "value": bases / out["batched"] / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["batched"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batched: {len(colls)} collections, {bases:,} bases, {suffixes:,} suffixes",
                       "l2": "flushed between steps", "input": "device-resident"},
            "plain_loop": {"value": bases / out["plain"] / 1e9, "unit": UNIT, "ms_per_step": out["plain"] * 1e3},
            "speedup_vs_plain_loop": out["plain"] / out["batched"],
            "autotune": {"classes": len(picks), "seconds": tune_s, "choices": chosen},
            "results_equal_oracle": equal}
    print(json.dumps(line), flush=True)
    return 0


def oracle_item_digests(name):
    """Packed digests of the oracle's results for the items of the batched or
    served workload (tests/golden/oracle_digests.json, written by a script
    that calls only the oracle), or None when they are not stored."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_digests.json")
    try:
        with open(p) as f:
            return [it["packed_sha256"] for it in json.load(f)[name]["items"]]
    except (OSError, KeyError):
        return None


def packed_digest(words, dpos, cnt):
    """SHA-256 of one result in packed form (the BWT words, then the $ rows
    and the counts as little-endian integers), the form the stored oracle
    digests take."""
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(words, dtype="<u4")).cast("B"))
    h.update(np.ascontiguousarray(dpos, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(cnt, dtype="<u8").tobytes())
    return h.hexdigest()


def run_serve_bench(args, rank, world):
    """The served workload: 256 requests (n log-uniform in [50k, 5M], length
    100 or 150, i.i.d. reads with per-request seeds) arriving as open-loop
    Poisson streams at 0.5, 0.8, 1.0 and 1.5 times the plain loop's measured
    capacity (one seeded arrival trace per load).  Under each trace, in real
    time:

    * the plain loop: one cxbwt_build at a time, first come first served,
      pinned host buffers;
    * the server: cxbwt_submit at each arrival time (continuous batching,
      2 and 3 workers).

    Latency = completion - arrival.  Every result of every run is compared
    with the oracle's stored digest of that request.  One JSON line with
    p50/p99 latency and aggregate Gbase/s of both per load (not the
    benchmark's default line)."""
    import collections
    import threading

    import torch

    from paper_1401_7457_gb300 import binding, build, synth
    build.build()
    k = args.reads or 256
    reqs = synth.serve_requests(k=k)
    want = oracle_item_digests("served")
    inputs = []
    total_bases = 0
    for rq in reqs:
        codes, lens = synth.request_reads(rq)
        words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).pin_memory()
        lt = torch.from_numpy(lens.view(np.int32)).pin_memory()
        N = int(lens.sum()) + lens.size
        inputs.append((words, lt, N, lens.size))
        total_bases += int(lens.sum())
    outs = [(torch.empty((N + 15) // 16, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory(),
             torch.zeros(5, dtype=torch.int64).pin_memory()) for (_, _, N, n) in inputs]

    def check_and_clear():
        """Digests of every result against the oracle's (when stored); then zero the outputs."""
        ok = None
        if want is not None:
            ok = all(packed_digest(o[0].numpy().view(np.uint32), o[1].numpy(), o[2].numpy()) == d
                     for o, d in zip(outs, want[:len(outs)]))
        for o in outs:
            for t in o:
                t.zero_()
        return ok

    budget = int(args.budget_gb * (1 << 30))
    ctx = binding.Context(device=0, budget_bytes=budget)
    ctx.build(inputs[0][0], inputs[0][1], *outs[0])  # warm-up
    # Service times of the plain loop (every request alone, back to back).
    service = []
    for (w, lt, N, n), o in zip(inputs, outs):
        t0 = time.perf_counter()
        ctx.build(w, lt, *o)
        service.append(time.perf_counter() - t0)
    alone_ok = check_and_clear()
    capacity = len(service) / sum(service)  # requests per second

    def plain_run(arrivals):
        """The plain loop under an arrival trace, in real time."""
        q = collections.deque()
        cv = threading.Condition()
        lat = [0.0] * len(inputs)
        t0 = time.perf_counter()

        def submitter():
            for i in range(len(inputs)):
                delay = arrivals[i] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                with cv:
                    q.append(i)
                    cv.notify()

        th = threading.Thread(target=submitter)
        th.start()
        for _ in range(len(inputs)):
            with cv:
                while not q:
                    cv.wait()
                i = q.popleft()
            w, lt, _, _ = inputs[i]
            ctx.build(w, lt, *outs[i])
            lat[i] = (time.perf_counter() - t0 - arrivals[i]) * 1e3
        th.join()
        return lat, time.perf_counter() - t0

    def served_run(srv, arrivals):
        tickets = [None] * len(inputs)
        t0 = time.perf_counter()
        for i, ((w, lt, N, n), o) in enumerate(zip(inputs, outs)):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[i] = srv.submit(w, lt, *o)
        for t in tickets:
            srv.wait(t)
        span = time.perf_counter() - t0
        return [srv.times(t)[1] for t in tickets], span

    p = lambda xs, q: float(np.percentile(np.asarray(xs), q))
    loads = {}
    traces = []
    for j, f in enumerate((0.5, 0.8, 1.0, 1.5)):
        trace_seed = 50 + j
        rng = np.random.default_rng(trace_seed)
        gaps = rng.exponential(1.0 / (f * capacity), size=len(inputs))
        traces.append((f, trace_seed, np.cumsum(gaps) - gaps[0]))  # the first request arrives at time 0
    for f, trace_seed, arrivals in traces:
        lat_p, span_p = plain_run(arrivals)
        ok_p = check_and_clear()
        loads[f"{f:g}x"] = {
            "arrival_rate_per_s": f * capacity, "trace_seed": trace_seed,
            "plain_loop": {"p50_ms": p(lat_p, 50), "p99_ms": p(lat_p, 99), "gbase_per_s": total_bases / span_p / 1e9,
                           "span_s": span_p, "results_equal_oracle": ok_p}}
    ctx.close()
    for workers in (2, 3):
        srv = binding.Server(device=0, budget_bytes=budget or (120 << 30), workers=workers)
        warm = srv.submit(inputs[0][0], inputs[0][1], *outs[0])
        srv.wait(warm)
        check_and_clear()
        for f, _, arrivals in traces:
            before = srv.counters()["packs"]
            lat_s, span_s = served_run(srv, arrivals)
            ok_s = check_and_clear()
            loads[f"{f:g}x"][f"served_{workers}_workers"] = {
                "p50_ms": p(lat_s, 50), "p99_ms": p(lat_s, 99), "gbase_per_s": total_bases / span_s / 1e9,
                "span_s": span_s, "builds": srv.counters()["packs"] - before, "results_equal_oracle": ok_s}
        srv.close()
    sat = loads["1.5x"]["served_2_workers"]
    line = {"metric": METRIC, "value": sat["gbase_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": sat["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"served: {len(inputs)} requests, {total_bases:,} bases, Poisson arrivals at 0.5, "
                                   f"0.8, 1.0 and 1.5x the plain loop's measured {capacity:.1f} requests/s",
                       "workers": [2, 3], "value": "served Gbase/s at 1.5x (saturated), 2 workers (the default)"},
            "loads": loads, "plain_alone_equal_oracle": alone_ok, "oracle_digests": want is not None}
    print(json.dumps(line), flush=True)
    return 0


def run_length_bench(args, rank, world):
    """Read-length sensitivity at equal total bases (after Table exp-len of the
    paper: 100/200/400 bp): genome-like reads from the 5 Mbp genome at 20x,
    1M x 100, 500k x 200 and 250k x 400 bp.  One JSON line with Gbase/s per
    length (not the benchmark's default line)."""
    import torch

    from paper_1401_7457_gb300 import binding, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    g = synth.random_genome(5_000_000, 2)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for L, n in ((100, 1_000_000), (200, 500_000), (400, 250_000)):
        codes, lens = synth.sample_reads(g, n, L, synth.derive_seed(2, L), 0.01)
        w = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).to(dev)
        ln = torch.from_numpy(lens.view(np.int32)).to(dev)
        ctx = binding.Context(device=0, timing=True)
        outs = ctx.build(w, ln)
        for _ in range(max(args.warmup, 1)):
            ctx.build(w, ln, *outs)
        ctx.reset_stats()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.build(w, ln, *outs)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        st = ctx.stats()
        ms = sum(ts) / len(ts)
        res[f"{L}bp"] = {"reads": n, "ms": ms, "gbase_per_s": n * L / (ms * 1e-3) / 1e9,
                         "group_finish_ms": st["group_ms"] / len(ts), "sort_pass_ms": st["sort_pass_ms"] / len(ts)}
        ctx.close()
    base = res["100bp"]["ms"]
    for k in res:
        res[k]["time_vs_100bp"] = res[k]["ms"] / base
    line = {"metric": METRIC, "value": res["100bp"]["gbase_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": base, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "read-length series: 100 Mbase of genome-like reads at 100, 200 and 400 bp"},
            "lengths": res}
    print(json.dumps(line), flush=True)
    return 0


def _timed(fn, steps, flush):
    """Mean CUDA-event time of fn() over steps calls, L2 flushed before each."""
    import torch
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sum(ts) / len(ts)


def run_parts_bench(args, rank, world):
    """Bucket-range parts of the genome-like collection (Section 3.3's
    partition, built one after another on this GPU): per-part device time for
    2, 4 and 8 parts against the whole build, and the checkpointed rounds
    (Section 3.1) end to end into files.  One JSON line (not the benchmark's
    default line)."""
    import tempfile

    import torch

    from paper_1401_7457_gb300 import binding, build, parts
    build.build()
    dev = torch.device("cuda", 0)
    _, codes, lens = load_workload("genome-like", 0, args.reads)
    bases = int(lens.sum())
    w = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).to(dev)
    ln = torch.from_numpy(lens.view(np.int32)).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = binding.Context(device=0, plan_flags=args.plan_flags)
    outs = ctx.build(w, ln)
    whole_ms = _timed(lambda: ctx.build(w, ln, *outs), args.steps, flush)
    counts = ctx.bucket_counts(w, ln)
    res = {"whole_ms": whole_ms}
    for P in (2, 4, 8):
        plan = parts.plan_parts(counts, P)
        per = []
        for p in plan:
            o = ctx.build_part(w, ln, p.lo, p.hi, p.row0, p.rows, bucket_counts=counts)
            for _ in range(max(args.warmup, 1)):
                ctx.build_part(w, ln, p.lo, p.hi, p.row0, p.rows, *o, bucket_counts=counts)
            per.append(_timed(lambda: ctx.build_part(w, ln, p.lo, p.hi, p.row0, p.rows, *o, bucket_counts=counts),
                              args.steps, flush))
        res[f"{P}_parts"] = {"part_ms": per, "sum_ms": sum(per), "max_ms": max(per),
                             "rows": [p.rows for p in plan]}
    with tempfile.TemporaryDirectory() as tmp:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = parts.build_rounds(ctx, w, ln, 4, tmp)
        rounds_s = time.perf_counter() - t0
        assert st["done"]
        ref = outs[0].cpu().numpy().view(np.uint32)
        same = bool(np.array_equal(np.fromfile(f"{tmp}/bwt.u32", dtype=np.uint32), ref))
    res["rounds_4_to_files"] = {"s": rounds_s, "gbase_per_s": bases / rounds_s / 1e9, "equal_to_whole_build": same}
    ctx.close()
    line = {"metric": METRIC, "value": bases / (whole_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": whole_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "bucket-range parts of the genome-like collection (1M x 100 bp)",
                       "l2": "flushed between steps"},
            "parts": res}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded_bench(args, rank, world):
    """Bucket-range parts of one collection across the ranks (Section 3.3):
    every rank holds the whole read store, counts the 8-base buckets itself,
    and builds the part of B_R made of its range of buckets (about N / world
    suffixes); one step = every rank's part, device-resident input and output,
    timed with CUDA events (max over ranks).  ``value`` = the collection's
    bases / that time: strong scaling, the work is one collection whatever
    the number of ranks.  ``e2e`` = parts.build_sharded end to end (the count,
    the part, its copy to the host and the gather of every part to rank 0 as
    tensors), wall time max over ranks.  One JSON line on rank 0."""
    import torch
    import torch.distributed as dist

    from paper_1401_7457_gb300 import binding, build, parts

    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    name = args.shard_workload
    desc, codes, lens = load_workload(name, 0, args.reads)  # the same collection on every rank
    words = binding.pack_codes(codes)
    del codes
    n, bases = lens.size, int(lens.sum())
    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    d_lens = torch.from_numpy(lens.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = binding.Context(device=local, budget_bytes=int(args.budget_gb * (1 << 30)), plan_flags=args.plan_flags)
    counts = ctx.bucket_counts(d_words, d_lens, stream=stream)
    plan = parts.plan_parts(counts, world)
    mine = plan[rank]
    out = ctx.build_part(d_words, d_lens, mine.lo, mine.hi, mine.row0, mine.rows, stream=stream, bucket_counts=counts)
    for _ in range(max(args.warmup, 3) - 1):
        ctx.build_part(d_words, d_lens, mine.lo, mine.hi, mine.row0, mine.rows, *out, stream=stream,
                       bucket_counts=counts)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.build_part(d_words, d_lens, mine.lo, mine.hi, mine.row0, mine.rows, *out, stream=stream,
                       bucket_counts=counts)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    value, total_ms = aggregate(dist, sum(ms), bases / world, world, args.steps)
    # End to end: the whole sharded build through parts.build_sharded.
    t_e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = parts.build_sharded(ctx, d_words, d_lens, stream=stream) if world > 1 else \
            parts.build_part_host(ctx, d_words, d_lens, mine, stream=stream)
        t_e2e.append(time.perf_counter() - t0)
        del res
    e2e_value, e2e_ms = aggregate(dist, sum(t_e2e) * 1e3, bases / world, world, len(t_e2e))
    ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "u64" if id_bytes(n, int(lens.max()), (bases + 15) // 16 * 4) == 8 else "u32",
                "data": "synthetic",
                "config": {"workload": "bucket-range parts of one collection, one per rank: " + desc.format(n=n, N=bases + n),
                           "parts": [{"lo": p.lo, "hi": p.hi, "rows": p.rows} for p in plan],
                           "l2": "flushed between steps (512 MB write outside the events)"},
                "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms / len(t_e2e),
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": (bases + n) // 4 + 8 * n,
                        "path": "parts.build_sharded: bucket counts, the part, its copy to the host, gather to rank 0"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cxbwt", choices=["cxbwt", "reference"])
    ap.add_argument("--cpu-sample-reads", type=int, default=None,
                    help="reads of the CPU samples (default: 15 draw chunks, 1,966,080 reads, for the benchmark's "
                         "cpu_baseline; 4 chunks, 524,288 reads, per step of the reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config2", action="store_true", help="skip the genome-like measurement (config2 key)")
    ap.add_argument("--reads", type=int, default=0,
                    help="reads per GPU (0: the workload's own size; smaller only for profiling captures)")
    ap.add_argument("--genome-mbp", type=float, default=0.0,
                    help="genome size of the genome-like / repeat-rich workload in Mbp (0: its own; with --reads, "
                         "a smaller copy at the workload's coverage for profiling captures)")
    ap.add_argument("--shard-workload", default="repeat-rich", choices=sorted(WORKLOADS),
                    help="the collection --workload sharded splits across the ranks")
    ap.add_argument("--workload", default="repeat-rich",
                    choices=sorted(WORKLOADS) + ["batch", "serve", "length", "parts", "sharded"],
                    help="repeat-rich is the benchmark; the others are the other workloads, timed for reference")
    ap.add_argument("--tile-items", type=int, default=0,
                    help="items per radix tile of the benchmark's contexts (0: the library's choice)")
    ap.add_argument("--plan-flags", type=int, default=0,
                    help="CXBWT_PLAN_* bits of the benchmark's contexts (1: 64-bit ids; for profiling captures)")
    ap.add_argument("--prefix-len", type=int, default=0,
                    help="l of the group plan of the benchmark's contexts (12 or 16; 0: the library's choice)")
    ap.add_argument("--budget-gb", type=float, default=0.0,
                    help="device budget of the library context (0: 90%% of free memory)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.cpu_sample_reads is None:
        args.cpu_sample_reads = (4 if args.impl == "reference" else 15) * SAMPLE_CHUNK
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch_bench(args, rank, world)
    if args.workload == "serve":
        return run_serve_bench(args, rank, world)
    if args.workload == "length":
        return run_length_bench(args, rank, world)
    if args.workload == "parts":
        return run_parts_bench(args, rank, world)
    if args.workload == "sharded":
        return run_sharded_bench(args, rank, world)

    import torch
    import torch.distributed as dist

    from paper_1401_7457_gb300 import build

    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up builds

    # Each rank builds its own independent collection (weak scaling, no data-path collective).
    desc, codes, lens = load_workload(args.workload, rank, args.reads, int(args.genome_mbp * 1e6))
    res = measure(args, dist, world, local, dev, desc, codes, lens, args.steps, e2e_steps=max(3, min(args.steps, 10)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        rate, dt, sb = cpu_oracle_rate(codes, lens, args.cpu_sample_reads, threads)
        n_s = min(args.cpu_sample_reads, lens.size)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"first {n_s:,} reads ({sb:,} bases) of the workload, {dt:.1f} s wall"}
        # The same oracle on one core, on a smaller sample (a few seconds).
        n1 = max(1, args.cpu_sample_reads // 15)
        rate1, dt1, sb1 = cpu_oracle_rate(codes, lens, n1, 1)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                "sample": f"first {min(n1, lens.size):,} reads ({sb1:,} bases), {dt1:.1f} s wall"}
    del codes, lens

    config2 = None
    if args.workload != "genome-like" and not args.no_config2:
        # The genome-like collection (1M x 100 bp at 20x, one slice, 32-bit ids), measured the same way.
        d2, c2, l2 = load_workload("genome-like", rank, 0)
        r2 = measure(args, dist, world, local, dev, d2, c2, l2, min(args.steps, 20), e2e_steps=max(3, min(args.steps, 10)))
        config2 = {k: r2[k] for k in ("value", "unit", "ms_per_step", "config", "roofline", "phases", "e2e",
                                      "gpu_launches_per_step", "clocks", "detail")}

    if rank == 0:
        line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64" if res["detail"]["id_bytes"] == 8 else "u32",
                "data": "synthetic", "config": res["config"], "roofline": res["roofline"], "phases": res["phases"],
                "cpu_baseline": cpu, "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
                "gpu_launches_per_step": res["gpu_launches_per_step"], "clocks": res["clocks"],
                "detail": res["detail"]}
        if config2 is not None:
            line["config2"] = config2
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure(args, dist, world, local, dev, desc, codes, lens, steps, e2e_steps):
    """One workload: K device-resident builds timed with CUDA events (and
    their phases, from the library's own events), then e2e_steps builds
    through the C ABI with pinned host buffers.  Returns the parts of a
    benchmark line."""
    import torch

    from paper_1401_7457_gb300 import binding

    words = binding.pack_codes(codes)
    n = lens.size
    bases = int(lens.sum())
    N = bases + n
    n_words = (N + 15) // 16
    read_len = int(lens[0])
    budget = int(args.budget_gb * (1 << 30))

    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    d_lens = torch.from_numpy(lens.view(np.int32)).to(dev)
    d_bwt = torch.empty(n_words, dtype=torch.int32, device=dev)
    d_dpos = torch.empty(n, dtype=torch.int64, device=dev)
    d_cnt = torch.zeros(5, dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = binding.Context(device=local, timing=True, budget_bytes=budget, plan_flags=args.plan_flags,
                          tile_items=args.tile_items, prefix_len=args.prefix_len)

    def step():
        ctx.build(d_words, d_lens, d_bwt, d_dpos, d_cnt, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(nvml_id(dev)) as clocks:
        for i in range(steps):
            flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (outside the events)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = ctx.stats()
    ctx.close()
    del ctx
    value, total_ms = aggregate(dist, sum(ms), bases, world, steps)

    # Dominant kernel: the onesweep digit pass that loads the key window the
    # previous pass carried.  Its algorithmic bytes per item are the key
    # (4 B) and the id (4 or 8 B), read and written; each launch is timed
    # between its own events on the build stream.
    idb = 8 if args.plan_flags & 1 else id_bytes(n, int(lens.max()), int((bases + 15) // 16) * 4)
    bytes_per_item = 2 * (4 + idb)
    launches = max(st["carried_pass_launches"], 1)
    pass_ms = st["carried_pass_ms"] / launches
    items_per_launch = st["carried_pass_items"] / launches
    achieved = bytes_per_item * items_per_launch / (pass_ms * 1e-3) / 1e9 if pass_ms > 0 else 0.0
    peak, peak_kind = peak_hbm()
    traffic_per_item = profiled_traffic(idb)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if traffic_per_item is None else traffic_per_item * items_per_launch,
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "k_onesweep, carried-key digit pass",
                "launches_per_step": st["carried_pass_launches"] / steps,
                "bytes_per_item": bytes_per_item, "items_per_launch": items_per_launch,
                "algorithmic_bytes_per_launch": bytes_per_item * items_per_launch,
                "avg_launch_ms": pass_ms, "frac_of_nominal_8tbs": achieved / 8000.0}

    # End to end through the C ABI with pinned host buffers (copies inside the timed region).
    h_words = torch.from_numpy(words.view(np.int32)).pin_memory()
    h_lens = torch.from_numpy(lens.view(np.int32)).pin_memory()
    del words, d_words, d_lens
    h_bwt = torch.empty(n_words, dtype=torch.int32).pin_memory()
    h_dpos = torch.empty(n, dtype=torch.int64).pin_memory()
    h_cnt = torch.zeros(5, dtype=torch.int64).pin_memory()
    ctx2 = binding.Context(device=local, budget_bytes=budget, plan_flags=args.plan_flags, tile_items=args.tile_items,
                           prefix_len=args.prefix_len)
    for _ in range(2):
        ctx2.build(h_words, h_lens, h_bwt, h_dpos, h_cnt, stream=stream)
    ctx2.reset_stats()
    torch.cuda.synchronize()
    t_e2e = []
    for _ in range(e2e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.build(h_words, h_lens, h_bwt, h_dpos, h_cnt, stream=stream)  # synchronous: returns with outputs on host
        t_e2e.append(time.perf_counter() - t0)
    st2 = ctx2.stats()
    ctx2.close()
    e2e_value, e2e_ms = aggregate(dist, sum(t_e2e) * 1e3, bases, world, e2e_steps)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": st2["h2d_bytes"] // e2e_steps, "d2h_bytes_per_step": st2["d2h_bytes"] // e2e_steps,
           "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps,
           "path": "cxbwt_build with pinned host input, lengths and outputs (BWT streamed per slice)"}
    del h_words, h_lens, h_bwt, h_dpos, h_cnt, d_bwt, d_dpos, d_cnt, flush
    torch.cuda.empty_cache()

    return {"value": value, "unit": UNIT, "ms_per_step": total_ms / steps,
            "config": {"workload": desc.format(n=n, N=N), "n_reads": n, "read_len": read_len, "bases_per_gpu": bases,
                       "suffixes_per_gpu": N, "l2": "flushed between steps (512 MB write outside the events)",
                       "input": "device-resident (HBM) before the timed region; outputs left in HBM"},
            "roofline": roofline, "phases": phase_rates(st, steps, n, bases, idb, peak), "e2e": e2e,
            "gpu_launches": int(st["kernel_launches"]), "gpu_launches_per_step": st["kernel_launches"] / steps,
            "clocks": clocks.summary(),
            "detail": {"step_ms": ms, "slices_per_step": st["slices"] / steps,
                       "digit_passes_per_step": st["sort_pass_launches"] / steps,
                       "sort_pass_ms_per_step": st["sort_pass_ms"] / steps,
                       "carried_pass_ms_per_step": st["carried_pass_ms"] / steps,
                       "group_finish_ms_per_step": st["group_ms"] / steps,
                       "emit_ms_per_step": st["emit_ms"] / steps,
                       "build_ms_per_step_lib": st["build_ms"] / steps,
                       "id_bytes": idb,
                       "cta_groups_per_step": st["cta_groups"] / steps,
                       "big_groups_per_step": st["big_groups"] / steps}}


if __name__ == "__main__":
    sys.exit(main())
