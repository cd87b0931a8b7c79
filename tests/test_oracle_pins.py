"""Pins of the CPU oracle against the paper and the mathematics (no GPU)."""
import itertools
import os

import numpy as np
import pytest

import oracle
import pins
from paper_1401_7457_gb300 import synth


def bwt_str(reads):
    return oracle.bwt(oracle.Collection.from_strings(reads))["bwt"].decode()


def test_figure1_worked_example():
    """Section 2, Figure 1: {ACGT$, TAGT$, GGAA$} -> TTAAG$TAG$CAGG$, and the
    sorted suffix columns printed under the line."""
    reads, sorted_suffixes, want = pins.read_figure1()
    col = oracle.Collection.from_strings(reads)
    res = oracle.bwt(col)
    assert res["bwt"].decode() == want
    got_suffixes = [reads[int(i)][int(k):] + "$" for i, k in zip(res["sa_read"], res["sa_pos"])]
    assert got_suffixes == sorted_suffixes


@pytest.mark.parametrize("reads,want", pins.read_hand_examples())
def test_hand_examples(reads, want):
    assert bwt_str(reads) == want


def test_rotation_brute_force_exhaustive_small():
    """Every collection of one read of length <= 5, two reads of length <= 3 and
    three reads of length <= 2 against rotation sorting."""
    def strings(max_len):
        for L in range(1, max_len + 1):
            for t in itertools.product("ACGT", repeat=L):
                yield "".join(t)
    cases = [[s] for s in strings(5)]
    s3 = list(strings(3))
    cases += [[a, b] for a in s3 for b in s3]
    s2 = list(strings(2))
    cases += [[a, b, c] for a in s2 for b in s2 for c in s2]
    bad = [c for c in cases if bwt_str(c) != pins.rotation_bwt(c)]
    assert not bad, bad[:5]


def test_rotation_brute_force_random():
    """Random small collections, including one- and two-letter alphabets
    (long runs of equal suffixes) and mixed read lengths."""
    rng = np.random.default_rng(2024)
    for _ in range(2000):
        k = int(rng.integers(1, 7))
        alpha = "ACGT"[: int(rng.integers(1, 5))]
        reads = ["".join(rng.choice(list(alpha), size=int(rng.integers(1, 11)))) for _ in range(k)]
        assert bwt_str(reads) == pins.rotation_bwt(reads), reads


def test_single_read_is_textbook_bwt():
    """n = 1: the BWT of S$ by sorted rotations of the single string."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = "".join(rng.choice(list("ACGT"), size=int(rng.integers(1, 40))))
        t = s + "$"
        rots = sorted(t[i:] + t[:i] for i in range(len(t)))  # '$' < 'A' in ASCII
        assert bwt_str([s]) == "".join(r[-1] for r in rots)


def test_identical_reads_closed_form():
    """n copies of S: every symbol of BWT(S$) repeated n times."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        s = "".join(rng.choice(list("ACGT"), size=int(rng.integers(1, 30))))
        n = int(rng.integers(2, 6))
        one = bwt_str([s])
        assert bwt_str([s] * n) == "".join(c * n for c in one)


@pytest.mark.parametrize("case", ["uniform", "genome", "mixed", "all_a"])
def test_invariants_moderate(case):
    if case == "uniform":
        codes, lens = synth.uniform_reads(2000, 100, 3)
    elif case == "genome":
        g = synth.random_genome(20_000, 4)
        codes, lens = synth.sample_reads(g, 4000, 100, 5, 0.01)  # 20x coverage: long shared prefixes
    elif case == "mixed":
        codes, lens = synth.mixed_length_reads(3000, 1, 150, 8)
    else:
        codes = np.zeros(500 * 40, dtype=np.uint8)
        lens = np.full(500, 40, dtype=np.uint32)
    col = oracle.Collection(codes, lens)
    res = oracle.bwt(col)
    pins.check_invariants(codes, lens, res["bwt"], res["dollar_pos"], res["counts"])
    assert oracle.check_sa(col, res["sa_read"], res["sa_pos"]) == -1


def test_rank_and_certificate_agree_with_sort():
    codes, lens = synth.mixed_length_reads(200, 1, 30, 9)
    col = oracle.Collection(codes, lens)
    res = oracle.bwt(col)
    rng = np.random.default_rng(0)
    for r in rng.integers(0, col.n_suffixes, size=50):
        assert oracle.rank(col, int(res["sa_read"][r]), int(res["sa_pos"][r])) == r
    sa_r, sa_p = res["sa_read"].copy(), res["sa_pos"].copy()
    assert oracle.check_sa(col, sa_r, sa_p) == -1
    # swapped neighbours
    sr, sp = sa_r.copy(), sa_p.copy()
    sr[[10, 11]] = sr[[11, 10]]
    sp[[10, 11]] = sp[[11, 10]]
    assert oracle.check_sa(col, sr, sp) == 10
    # a duplicated entry
    sr, sp = sa_r.copy(), sa_p.copy()
    sr[20], sp[20] = sr[5], sp[5]
    assert oracle.check_sa(col, sr, sp) >= 0
    # wrong length
    assert oracle.check_sa(col, sa_r[:-1], sa_p[:-1]) == -2


def test_tiny_uniform_workload_invariants():
    """The 10,000 x 100 bp workload end to end through the oracle (about a second)."""
    codes, lens = synth.tiny_uniform()
    col = oracle.Collection(codes, lens)
    res = oracle.bwt(col)
    assert col.n_suffixes == 1_010_000
    pins.check_invariants(codes, lens, res["bwt"], res["dollar_pos"], res["counts"])


def test_oracle_reproduces_its_stored_digest():
    """The oracle's result for the 10,000 x 100 bp workload has the digest
    that tests/golden/make_oracle_digests.py stored (the GPU tests compare
    with the stored digests)."""
    want = pins.read_oracle_digests()["tiny"]
    codes, lens = synth.tiny_uniform()
    assert pins.input_digest(codes, lens) == want["input_sha256"]
    res = oracle.bwt(oracle.Collection(codes, lens), threads=os.cpu_count() or 1)
    assert len(res["bwt"]) == want["n_symbols"]
    assert pins.result_digest(res["bwt"], res["dollar_pos"], res["counts"]) == want["sha256"]
    # Each part of a result enters the digest.
    flipped = bytearray(res["bwt"])
    flipped[5] = ord("A") if flipped[5] != ord("A") else ord("C")
    assert pins.result_digest(bytes(flipped), res["dollar_pos"], res["counts"]) != want["sha256"]
    assert pins.result_digest(res["bwt"], res["dollar_pos"] + np.uint64(1), res["counts"]) != want["sha256"]
    assert pins.result_digest(res["bwt"], res["dollar_pos"], res["counts"][::-1]) != want["sha256"]


def test_prefix_ranges_match_brute_force():
    """The oracle's sort one range of prefix buckets at a time (Section 3.1:
    suffixes whose first l symbols differ are ordered by those symbols, so the
    buckets sort independently and concatenate in bucket order) against the
    brute-force rotation order, for bucket prefixes of 1 to 4 symbols and
    ranges down to one bucket each; reads shorter than the prefix end inside
    it."""
    rng = np.random.default_rng(31)
    for _ in range(400):
        k = int(rng.integers(1, 7))
        alpha = "ACGT"[: int(rng.integers(1, 5))]
        reads = ["".join(rng.choice(list(alpha), size=int(rng.integers(1, 9)))) for _ in range(k)]
        p = int(rng.integers(1, 5))
        assert pins.prefix_ranges_match(reads, p, int(rng.integers(1, 12))), (reads, p)


def test_prefix_ranges_equal_the_whole_sort():
    """At a moderate size (genome-like reads, long shared prefixes), the
    ranges concatenate to exactly the whole sort, and the bucket counts sum
    to N."""
    g = synth.random_genome(20_000, 41)
    codes, lens = synth.sample_reads(g, 3000, 100, 42, 0.01)
    col = oracle.Collection(codes, lens)
    ref = oracle.bwt(col, threads=2)
    counts = oracle.prefix_counts(col, 3, threads=2)
    assert int(counts.sum()) == col.n_suffixes and counts[0] == col.n  # bucket "$$$": the terminator-only suffixes
    parts = list(oracle.sorted_ranges(col, 3, 20_000, threads=2))
    assert len(parts) > 5
    assert b"".join(b for _, b, _, _ in parts) == ref["bwt"]
    assert np.array_equal(np.concatenate([r for _, _, r, _ in parts]), ref["sa_read"])
    assert np.array_equal(np.concatenate([q for _, _, _, q in parts]), ref["sa_pos"])
