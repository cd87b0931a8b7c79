"""Seeded generators: deterministic, right shapes (no GPU)."""
import hashlib

import numpy as np

from paper_1401_7457_gb300 import synth


def test_tiny_uniform_is_stable():
    codes, lens = synth.tiny_uniform()
    assert codes.size == 1_000_000 and lens.size == 10_000 and int(lens.min()) == int(lens.max()) == 100
    # PCG64 streams are the same on every platform; this pins the workload itself.
    assert hashlib.sha256(codes.tobytes()).hexdigest()[:16] == "15f00ff3336764f3"


def test_genome_reads_shape_and_errors():
    g = synth.random_genome(10_000, 1)
    codes, lens = synth.sample_reads(g, 2000, 50, 2, sub_rate=0.0, both_strands=False)
    gs = "".join("ACGT"[c] for c in g)
    reads = codes.reshape(-1, 50)
    for r in reads[:50]:
        assert "".join("ACGT"[c] for c in r) in gs
    codes2, _ = synth.sample_reads(g, 2000, 50, 2, sub_rate=0.0, both_strands=True)
    rc = "".join("ACGT"[3 - c] for c in g[::-1])
    for r in codes2.reshape(-1, 50)[:50]:
        s = "".join("ACGT"[c] for c in r)
        assert s in gs or s in rc


def test_batch_and_serve_specs():
    specs = synth.batch_specs()
    assert len(specs) == 256
    assert all(s["length"] in synth.BATCH_LENGTHS for s in specs)
    assert all(10_000 <= s["n_reads"] <= 2_000_000 for s in specs)
    assert all(1_000_000 <= s["genome_size"] <= 20_000_000 for s in specs)
    reqs = synth.serve_requests()
    assert len(reqs) == 256 and all(r["length"] in synth.SERVE_LENGTHS for r in reqs)
    t = [r["arrival_s"] for r in reqs]
    assert all(a < b for a, b in zip(t, t[1:]))


def test_repeat_rich_genome_has_repeats():
    g = synth.repeat_rich_genome(200_000, 3, repeat_fraction=0.05, repeat_len=1000, copies_per_template=10)
    assert g.size == 200_000 and int(g.max()) <= 3
    # 10 copies of a 1 kb template: some 32-mer occurs many times.
    k = 32
    w = np.lib.stride_tricks.sliding_window_view(g, k)
    keys = [bytes(x) for x in w]
    _, cnt = np.unique(np.array(keys), return_counts=True)
    assert cnt.max() >= 5
