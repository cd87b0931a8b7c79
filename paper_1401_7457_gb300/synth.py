"""Seeded synthetic read collections with the shape of the paper's workloads.

This module only draws random reads.  It holds none of the BWT arithmetic and
imports nothing from the CUDA path or from the oracle, so both sides (and the
benchmark) can take their inputs from it.

The paper measures on real 100 bp Illumina reads over {A,C,G,T} (Section 4,
"Experiments"), which are not available here; these generators stand in for
them with the same read length and alphabet.  Every draw comes from numpy's
PCG64 bit generator (O'Neill 2014), which gives identical streams on every
platform; each workload documents its seed.

A collection is returned as ``(codes, lens)``: ``codes`` is one ``uint8`` array
of base codes (A=0, C=1, G=2, T=3) with all reads concatenated, ``lens`` the
``uint32`` read lengths.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN64 = 0x9E3779B97F4A7C15  # floor(2^64 / phi): derives per-item seeds from one seed


def derive_seed(seed: int, index: int) -> int:
    """Seed of item ``index`` (a collection, a request) of a workload seeded with ``seed``."""
    return (seed ^ ((index * GOLDEN64) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_reads(n: int, length: int, seed: int):
    """n reads of one length, every base i.i.d. uniform over ACGT."""
    rng = _rng(seed)
    codes = rng.integers(0, 4, size=n * length, dtype=np.uint8)
    return codes, np.full(n, length, dtype=np.uint32)


def mixed_length_reads(n: int, min_len: int, max_len: int, seed: int):
    """n reads, lengths uniform in [min_len, max_len], bases i.i.d. uniform."""
    rng = _rng(seed)
    lens = rng.integers(min_len, max_len + 1, size=n, dtype=np.int64).astype(np.uint32)
    codes = rng.integers(0, 4, size=int(lens.sum()), dtype=np.uint8)
    return codes, lens


def random_genome(size: int, seed: int) -> np.ndarray:
    """A genome of ``size`` i.i.d. uniform bases."""
    return _rng(seed).integers(0, 4, size=size, dtype=np.uint8)


def repeat_rich_genome(size: int, seed: int, repeat_fraction: float = 0.05, repeat_len: int = 1000,
                       copies_per_template: int = 10, divergence: float = 0.005) -> np.ndarray:
    """Uniform genome in which ``repeat_fraction`` of the sequence is made of
    copies of ``repeat_len``-base templates (``copies_per_template`` copies of
    each), every copy carrying ``divergence`` substitutions, placed at
    non-overlapping random sites."""
    rng = _rng(seed)
    g = rng.integers(0, 4, size=size, dtype=np.uint8)
    n_copies = int(round(size * repeat_fraction / repeat_len))
    n_templates = max(1, n_copies // copies_per_template)
    templates = rng.integers(0, 4, size=(n_templates, repeat_len), dtype=np.uint8)
    # Non-overlapping sites: choose copy slots among size // repeat_len aligned
    # slots, then jitter each within its slot so sites are not aligned.
    n_slots = size // repeat_len
    slots = rng.choice(n_slots - 1, size=n_copies, replace=False)
    jitter = rng.integers(0, repeat_len, size=n_copies)
    starts = np.minimum(slots * repeat_len + jitter, size - repeat_len)
    order = np.argsort(starts)
    starts = starts[order]
    # After jitter neighbours may touch; push each start past its predecessor.
    for c in range(1, n_copies):
        if starts[c] < starts[c - 1] + repeat_len:
            starts[c] = starts[c - 1] + repeat_len
    keep = starts + repeat_len <= size
    starts = starts[keep]
    which = rng.integers(0, n_templates, size=starts.size)
    for s, t in zip(starts.tolist(), which.tolist()):
        copy = templates[t].copy()
        mut = rng.random(repeat_len) < divergence
        copy[mut] = (copy[mut] + rng.integers(1, 4, size=int(mut.sum()), dtype=np.uint8)) % 4
        g[s:s + repeat_len] = copy
    return g


def sample_reads(genome: np.ndarray, n: int, length: int, seed: int, sub_rate: float = 0.01,
                 both_strands: bool = True, chunk: int = 1 << 17):
    """n reads of ``length`` bases: start uniform in [0, G - length], strand
    forward or reverse complement with probability 1/2 each, and every base
    replaced with probability ``sub_rate`` by one of the other three bases,
    uniformly."""
    rng = _rng(seed)
    G = genome.size
    if G < length:
        raise ValueError("genome shorter than the reads")
    codes = np.empty(n * length, dtype=np.uint8)
    col = np.arange(length, dtype=np.int64)
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        starts = rng.integers(0, G - length + 1, size=m, dtype=np.int64)
        block = genome[starts[:, None] + col[None, :]]
        if both_strands:
            rev = rng.random(m) < 0.5
            block[rev] = 3 - block[rev, ::-1]  # reverse complement: A<->T, C<->G
        if sub_rate > 0:
            mut = rng.random((m, length)) < sub_rate
            k = int(mut.sum())
            block[mut] = (block[mut] + rng.integers(1, 4, size=k, dtype=np.uint8)) % 4
        codes[c0 * length:(c0 + m) * length] = block.reshape(-1)
    return codes, np.full(n, length, dtype=np.uint32)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's 100 bp reads; each function
# below states its recipe.
# ---------------------------------------------------------------------------

def tiny_uniform(seed: int = 1):
    """10,000 reads x 100 bp, i.i.d. uniform (1 Mbase, 1,010,000 suffixes)."""
    return uniform_reads(10_000, 100, seed)


def genome_like(seed: int = 2, n_reads: int = 1_000_000, genome_size: int = 5_000_000, length: int = 100):
    """1M reads x 100 bp from both strands of a 5 Mbp random genome (20x), 1% substitutions."""
    g = random_genome(genome_size, seed)
    return sample_reads(g, n_reads, length, derive_seed(seed, 1), 0.01)


def repeat_rich(seed: int = 3, n_reads: int = 50_000_000, genome_size: int = 100_000_000, length: int = 100):
    """50M reads x 100 bp from a 100 Mbp genome with 5% of 1 kb repeats at 0.5% divergence."""
    g = repeat_rich_genome(genome_size, seed)
    return sample_reads(g, n_reads, length, derive_seed(seed, 1), 0.01)


BATCH_LENGTHS = (36, 76, 100, 150)


def batch_specs(seed: int = 4, k: int = 256, n_min: int = 10_000, n_max: int = 2_000_000):
    """Per-collection (n_reads, length, genome_size, coverage, seed) of the batched workload:
    n log-uniform in [n_min, n_max], length uniform over {36, 76, 100, 150},
    coverage uniform in [20, 50], genome = clamp(round(n*L/cov), 1 Mbp, 20 Mbp)."""
    rng = _rng(seed)
    specs = []
    for c in range(k):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(BATCH_LENGTHS[int(rng.integers(0, len(BATCH_LENGTHS)))])
        cov = float(rng.uniform(20.0, 50.0))
        G = int(min(max(round(n * L / cov), 1_000_000), 20_000_000))
        specs.append({"n_reads": n, "length": L, "genome_size": G, "coverage": n * L / G,
                      "seed": derive_seed(seed, c + 1)})
    return specs


def batch_collection(spec):
    """One collection of the batched workload, from its spec."""
    g = random_genome(spec["genome_size"], spec["seed"])
    return sample_reads(g, spec["n_reads"], spec["length"], derive_seed(spec["seed"], 1), 0.01)


SERVE_LENGTHS = (100, 150)


def serve_requests(seed: int = 5, k: int = 256, n_min: int = 50_000, n_max: int = 5_000_000,
                   rate_per_s: float = 1.0):
    """Open-loop Poisson request stream: (arrival_s, n_reads, length, seed) per request.
    n log-uniform in [n_min, n_max]; length uniform over {100, 150}; reads
    i.i.d. uniform (drawn later by ``request_reads``)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for r in range(k):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(SERVE_LENGTHS[int(rng.integers(0, len(SERVE_LENGTHS)))])
        out.append({"arrival_s": t, "n_reads": n, "length": L, "seed": derive_seed(seed, r + 1)})
    return out


def request_reads(req):
    """The reads of one served request."""
    return uniform_reads(req["n_reads"], req["length"], req["seed"])


def ascii_reads(strings):
    """Reads given as strings over ACGT -> (codes, lens); for hand-written cases."""
    table = np.full(256, 255, dtype=np.uint8)
    for i, c in enumerate(b"ACGT"):
        table[c] = i
    joined = "".join(strings).encode()
    codes = table[np.frombuffer(joined, dtype=np.uint8)] if joined else np.zeros(0, dtype=np.uint8)
    if codes.size and int(codes.max()) > 3:
        raise ValueError("reads must be over ACGT")
    return codes.astype(np.uint8), np.array([len(s) for s in strings], dtype=np.uint32)
