"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact everywhere: the BWT is an exact integer transform, so the packed
symbols, the $ rows of every read, the symbol counts and (where asked) the
suffix order must equal the oracle's.
"""
import numpy as np
import pytest

import oracle
import pins
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


from gpu_helpers import assert_same, ctx, gpu_bwt, oracle_of  # noqa: F401


def test_figure1(ctx):
    reads, _, want = pins.read_figure1()
    codes, lens = synth.ascii_reads(reads)
    got = gpu_bwt(ctx, codes, lens, want_sa=True)
    assert got["bwt"].decode() == want
    assert_same(got, oracle_of(codes, lens), sa=True)


@pytest.mark.parametrize("reads,want", pins.read_hand_examples())
def test_hand_examples(ctx, reads, want):
    codes, lens = synth.ascii_reads(reads)
    assert gpu_bwt(ctx, codes, lens)["bwt"].decode() == want


def test_random_small_collections(ctx):
    """Small mixed-length collections over 1- to 4-letter alphabets."""
    rng = np.random.default_rng(99)
    for t in range(150):
        k = int(rng.integers(1, 40))
        alpha = int(rng.integers(1, 5))
        lens = rng.integers(1, 40, size=k).astype(np.uint32)
        codes = rng.integers(0, alpha, size=int(lens.sum())).astype(np.uint8)
        got = gpu_bwt(ctx, codes, lens, want_sa=True)
        assert_same(got, oracle_of(codes, lens), sa=True)


def test_tiny_uniform_workload_full(ctx):
    """10,000 x 100 bp uniform reads (1,010,000 suffixes, 247 tiles, ragged last tile):
    every symbol, every $ row, the counts and the full suffix order."""
    codes, lens = synth.tiny_uniform()
    ref = oracle_of(codes, lens)
    got = gpu_bwt(ctx, codes, lens, want_sa=True)
    assert_same(got, ref, sa=True)


def test_tiny_uniform_host_buffers(ctx):
    """Same build with host input and output buffers (copies inside the library)."""
    codes, lens = synth.tiny_uniform()
    ref = oracle_of(codes, lens)
    assert_same(gpu_bwt(ctx, codes, lens, where="host"), ref)


def test_genome_like_small(ctx):
    """20x-coverage reads from a 50 kbp genome: long shared prefixes, both strands."""
    g = synth.random_genome(50_000, 21)
    codes, lens = synth.sample_reads(g, 10_000, 100, 22, 0.01)
    assert_same(gpu_bwt(ctx, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


@pytest.mark.parametrize("lo,hi,n", [(1, 150, 3000), (1, 8, 5000), (200, 300, 500), (90, 100, 4000)])
def test_mixed_lengths(ctx, lo, hi, n):
    """Reads of different lengths: the (length, read) start order comes from one
    or two length passes (two when a read is longer than 255)."""
    codes, lens = synth.mixed_length_reads(n, lo, hi, lo * 1000 + hi)
    assert_same(gpu_bwt(ctx, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


@pytest.mark.parametrize("case", ["one_base", "one_read", "all_a", "all_t", "identical", "two_letters",
                                  "tile_exact", "long_read", "max_len_read"])
def test_edge_cases(ctx, case):
    rng = np.random.default_rng(5)
    if case == "one_base":
        codes, lens = np.array([2], dtype=np.uint8), np.array([1], dtype=np.uint32)
    elif case == "one_read":
        codes, lens = synth.uniform_reads(1, 100, 1)
    elif case == "all_a":  # every suffix ties with its A-padded extensions
        codes, lens = np.zeros(3000 * 50, dtype=np.uint8), np.full(3000, 50, dtype=np.uint32)
    elif case == "all_t":
        codes, lens = np.full(3000 * 50, 3, dtype=np.uint8), np.full(3000, 50, dtype=np.uint32)
    elif case == "identical":
        one = rng.integers(0, 4, size=77).astype(np.uint8)
        codes, lens = np.tile(one, 2000), np.full(2000, 77, dtype=np.uint32)
    elif case == "two_letters":
        lens = rng.integers(20, 60, size=3000).astype(np.uint32)
        codes = rng.integers(0, 2, size=int(lens.sum())).astype(np.uint8)
    elif case == "tile_exact":  # N = 2 * 4096 exactly: no ragged tile
        codes, lens = synth.uniform_reads(128, 63, 3)
        assert int(lens.sum()) + lens.size == 8192
    elif case == "long_read":  # one 20,000-base read plus short ones
        lens = np.array([20_000] + [30] * 100, dtype=np.uint32)
        codes = rng.integers(0, 4, size=int(lens.sum())).astype(np.uint8)
    else:  # the longest read the ABI accepts (65,535 bases) plus short ones
        lens = np.array([30] * 50 + [65_535] + [30] * 50, dtype=np.uint32)
        codes = rng.integers(0, 4, size=int(lens.sum())).astype(np.uint8)
    assert_same(gpu_bwt(ctx, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


def test_repeated_builds_are_identical(ctx):
    """Determinism and workspace reuse: a bigger build, then a smaller one, then the first again."""
    a = synth.uniform_reads(5000, 100, 77)
    b = synth.mixed_length_reads(700, 5, 90, 78)
    r1 = gpu_bwt(ctx, *a)
    r2 = gpu_bwt(ctx, *b)
    r3 = gpu_bwt(ctx, *a)
    assert r1["bwt"] == r3["bwt"] and np.array_equal(r1["dollar_pos"], r3["dollar_pos"])
    assert_same(r2, oracle_of(*b))


def test_invalid_arguments(ctx):
    from paper_1401_7457_gb300 import binding
    words = np.zeros(4, dtype=np.uint32)
    with pytest.raises(binding.CxbwtError) as e:
        ctx.build(words, np.array([10, 0, 5], dtype=np.uint32))
    assert e.value.status == -1
    with pytest.raises(binding.CxbwtError) as e:
        ctx.build(words, np.array([70000], dtype=np.uint32))
    assert e.value.status == -1
    with pytest.raises(binding.CxbwtError) as e:
        ctx.build(words, np.zeros(0, dtype=np.uint32))
    assert e.value.status == -1
    # the context still works afterwards
    codes, lens = synth.uniform_reads(10, 10, 1)
    assert_same(gpu_bwt(ctx, codes, lens), oracle_of(codes, lens))


def test_budget_too_small_is_enomem():
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = synth.uniform_reads(10_000, 100, 1)
    with binding.Context(device=0, budget_bytes=1 << 20) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -2


@pytest.mark.parametrize("tile_items", [2048, 4096, 8192])
def test_tile_shapes_identical(tile_items):
    """The result does not depend on the tile shape of the digit passes."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = synth.mixed_length_reads(20_000, 30, 120, 31)
    ref = oracle_of(codes, lens)
    with binding.Context(device=0, tile_items=tile_items) as c:
        assert_same(gpu_bwt(c, codes, lens), ref)


@pytest.mark.parametrize("flags", [0, 1, 16, 17])
@pytest.mark.parametrize("tile_items", [2048, 4096])
def test_prefetching_carried_pass(flags, tile_items):
    """The carried-key digit passes with the tile one resident grid ahead
    read into L2 (the default) and without (plan flag 16): 32- and 64-bit ids
    (plan flag 1), tiles of 2048 (64-bit ids only) and 4096 items, a ragged
    last tile (1,246,845 suffixes), the group plan and the LSD plan (which
    carries every window: 18 of its 25 passes); all equal the oracle."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = synth.sample_reads(synth.random_genome(60_000, 91), 12_345, 100, 92, 0.01)
    ref = oracle_of(codes, lens)
    for algorithm in (1, 2):
        with binding.Context(device=0, algorithm=algorithm, plan_flags=flags, tile_items=tile_items) as c:
            assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)


PLAN_CASES = ["uniform", "genome", "mixed", "all_a", "identical_cta", "identical_big", "two_letters", "short"]


def plan_case(case):
    rng = np.random.default_rng(17)
    if case == "uniform":
        return synth.uniform_reads(20_000, 100, 41)
    if case == "genome":  # 40x coverage of a 50 kbp genome: groups of ~20 share long prefixes
        return synth.sample_reads(synth.random_genome(50_000, 42), 20_000, 100, 43, 0.01)
    if case == "mixed":
        return synth.mixed_length_reads(10_000, 1, 150, 44)
    if case == "all_a":  # one huge group whose remainder is finished by the LSD fallback
        return np.zeros(3000 * 50, dtype=np.uint8), np.full(3000, 50, dtype=np.uint32)
    if case == "identical_cta":  # groups of 2000 equal suffixes: the CTA sort
        one = rng.integers(0, 4, size=77).astype(np.uint8)
        return np.tile(one, 2000), np.full(2000, 77, dtype=np.uint32)
    if case == "identical_big":  # groups of 3000 equal suffixes: the fallback
        one = rng.integers(0, 4, size=60).astype(np.uint8)
        return np.tile(one, 3000), np.full(3000, 60, dtype=np.uint32)
    if case == "two_letters":
        lens = rng.integers(20, 60, size=3000).astype(np.uint32)
        return rng.integers(0, 2, size=int(lens.sum())).astype(np.uint8), lens
    lens = rng.integers(1, 20, size=5000).astype(np.uint32)  # every suffix within the first window
    return rng.integers(0, 4, size=int(lens.sum())).astype(np.uint8), lens


@pytest.mark.parametrize("case", PLAN_CASES)
@pytest.mark.parametrize("algorithm", [1, 2])
def test_plans_identical(case, algorithm):
    """Both sort plans (LSD over every digit; window-0 LSD + on-chip group
    finish) give the oracle's result, suffix order included."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = plan_case(case)
    ref = oracle_of(codes, lens)
    with binding.Context(device=0, algorithm=algorithm) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)


COVERAGE_CASES = ["genome_50x", "repeats_50x", "a_rich_50x", "reads_36_50x", "reads_150_50x", "reads_300_50x"]


def coverage_case(case):
    """Collections whose groups of equal first 16 bases are as large and as
    structured as the benchmark's: reads at 50x coverage (about 21 suffixes
    of one locus per strand, ordered by length, with 1% substitutions), 1 kb
    repeats, an A-rich genome (long A runs: many rows whose A-padded keys are
    equal), and read lengths from 36 to 300 bases (2 to 24 key words)."""
    if case == "genome_50x":
        return synth.sample_reads(synth.random_genome(40_000, 61), 20_000, 100, 62, 0.01)
    if case == "repeats_50x":
        return synth.repeat_rich(seed=63, n_reads=40_000, genome_size=80_000)
    if case == "a_rich_50x":
        g = np.random.default_rng(64).choice(4, size=40_000, p=[0.7, 0.1, 0.1, 0.1]).astype(np.uint8)
        return synth.sample_reads(g, 20_000, 100, 65, 0.01)
    length = int(case.split("_")[1])
    return synth.sample_reads(synth.random_genome(length * 400, 66), 20_000, length, 67, 0.01)


@pytest.mark.parametrize("case", COVERAGE_CASES)
def test_group_finish_at_high_coverage(case):
    """The group plan on groups of benchmark size and shape (warp windows of
    several 20-row groups, ties of equal A-padded keys, 2 to 24 key words):
    the oracle's result, suffix order included."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = coverage_case(case)
    with binding.Context(device=0, algorithm=2) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


@pytest.mark.parametrize("case", PLAN_CASES)
def test_group_plan_depth_12(case):
    """The group plan with l = 12 (prefix_len): three LSD passes sort the
    first 12 bases and the groups sharing them are finished from base 12 on
    (the warp and CTA finishes, and for all-A and identical reads the
    big-group LSD passes over windows starting at base 12); the oracle's
    result, suffix order included."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = plan_case(case)
    with binding.Context(device=0, algorithm=2, prefix_len=12) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


def test_group_plan_depth_12_read_lengths():
    """Keys of 24 words (300-base reads, groups of 1,500 equal suffixes past
    the CTA limit), reads of 524 bases (the longest l = 12 finishes on chip),
    and 528-base reads, which l = 12 leaves to the LSD plan when the plan is
    automatic and refuses when the group plan is asked for."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    one = np.random.default_rng(95).integers(0, 4, size=300).astype(np.uint8)
    cases = [(np.tile(one, 1500), np.full(1500, 300, dtype=np.uint32))]
    g = synth.random_genome(524 * 800 // 30, 96)
    cases.append(synth.sample_reads(g, 800, 524, 97, 0.01))
    for codes, lens in cases:
        with binding.Context(device=0, algorithm=2, prefix_len=12) as c:
            assert_same(gpu_bwt(c, codes, lens), oracle_of(codes, lens))
    codes, lens = synth.uniform_reads(300, 528, 98)
    with binding.Context(device=0, prefix_len=12) as c:
        assert_same(gpu_bwt(c, codes, lens), oracle_of(codes, lens))
    with binding.Context(device=0, algorithm=2, prefix_len=12) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -5


def test_group_plan_depth_12_batch():
    """A batch whose small collections are packed and sorted as one with
    l = 12; every collection's BWT is the oracle's."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cols = []
    for j in range(6):
        g = synth.random_genome(20_000 + 5_000 * j, 110 + j)
        cols.append(synth.sample_reads(g, 2_000 + 700 * j, (36, 76, 100)[j % 3], 120 + j, 0.01))
    with binding.Context(device=0, prefix_len=12) as c:
        outs = []
        for codes, lens in cols:
            n_sym = int(lens.sum()) + lens.size
            outs.append((binding.pack_codes(codes), np.ascontiguousarray(lens, dtype=np.uint32),
                         np.zeros((n_sym + 15) // 16, dtype=np.uint32), np.zeros(lens.size, dtype=np.uint64),
                         np.zeros(5, dtype=np.uint64)))
        c.build_batch(outs)
    for (codes, lens), (_, _, bwt, dpos, cnt) in zip(cols, outs):
        ref = oracle_of(codes, lens)
        assert binding.unpack_ascii(bwt, dpos, len(ref["bwt"])) == ref["bwt"]
        assert np.array_equal(dpos, ref["dollar_pos"]) and np.array_equal(cnt, ref["counts"])


def test_group_plan_rejects_long_reads():
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = synth.uniform_reads(10, 600, 3)
    with binding.Context(device=0, algorithm=2) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -5
    with binding.Context(device=0) as c:  # the automatic plan takes the LSD passes instead
        assert_same(gpu_bwt(c, codes, lens), oracle_of(codes, lens))


def test_autotune_then_build():
    """The autotuner picks a plan on one collection; builds of that size class
    use it and still equal the oracle."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = synth.sample_reads(synth.random_genome(40_000, 81), 12_000, 100, 82, 0.01)
    N = int(lens.sum()) + lens.size
    words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).cuda()
    dl = torch.from_numpy(lens.view(np.int32)).cuda()
    scratch = torch.zeros((N + 15) // 16, dtype=torch.int32, device="cuda")
    with binding.Context(device=0) as c:
        t = c.autotune(words, dl, scratch)
        assert t["tile_items"] in (4096, 8192) and t["algorithm"] in (1, 2) and t["best_ms"] > 0
        assert t["prefix_len"] == (0 if t["algorithm"] == 1 else t["prefix_len"]) and t["prefix_len"] in (0, 12, 16)
        assert_same(gpu_bwt(c, codes, lens), oracle_of(codes, lens))
        # same size class, other data
        codes2, lens2 = synth.uniform_reads(12_000, 100, 83)
        assert_same(gpu_bwt(c, codes2, lens2), oracle_of(codes2, lens2))


@pytest.mark.parametrize("length,n", [(200, 6000), (400, 3000), (528, 1000)])
def test_long_reads_group_plan(length, n):
    """Reads of 200, 400 and 528 bases (the paper's read-length experiment
    uses 100/200/400 bp): genome-like reads at 30x, group plan vs oracle."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = synth.random_genome(n * length // 30, length)
    codes, lens = synth.sample_reads(g, n, length, length + 1, 0.01)
    with binding.Context(device=0, algorithm=2) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)


@pytest.mark.parametrize("flags,algorithm", [(8, 1), (8, 2), (8 | 1, 1), (8 | 1, 2), (8 | 2, 2), (8 | 2 | 1, 2)])
def test_carried_base_plans(flags, algorithm):
    """Ids that carry the base before the suffix (the default for stores out of
    L2), forced on small inputs: 32- and 64-bit ids, read-major slices, both
    sort plans (the LSD plan's first pass gathers the last window, not the
    first); slices (a small budget) run with the group plan only."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = synth.random_genome(40_000, 71)
    codes, lens = synth.sample_reads(g, 6000, 100, 72, 0.01)
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    budget = (6 << 20) + int((28 if flags & 1 else 20) * N / 3) if flags & 2 else 0
    with binding.Context(device=0, algorithm=algorithm, plan_flags=flags, budget_bytes=budget) as c:
        got = gpu_bwt(c, codes, lens, want_sa=True)
    assert_same(got, ref, sa=True)


def test_carried_base_batch():
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cols = []
    for j in range(5):
        codes, lens = synth.uniform_reads(300 + 100 * j, 36 if j % 2 else 76, 80 + j)
        cols.append((codes, lens))
    with binding.Context(device=0, plan_flags=8) as c:
        outs = []
        for codes, lens in cols:
            n_sym = int(lens.sum()) + lens.size
            outs.append((binding.pack_codes(codes), np.ascontiguousarray(lens, dtype=np.uint32),
                         np.zeros((n_sym + 15) // 16, dtype=np.uint32), np.zeros(lens.size, dtype=np.uint64),
                         np.zeros(5, dtype=np.uint64)))
        c.build_batch(outs)
    for (codes, lens), (_, _, bwt, dpos, cnt) in zip(cols, outs):
        ref = oracle_of(codes, lens)
        assert binding.unpack_ascii(bwt, dpos, len(ref["bwt"])) == ref["bwt"]
        assert np.array_equal(dpos, ref["dollar_pos"]) and np.array_equal(cnt, ref["counts"])


def test_wide_key_groups_larger_than_a_cta():
    """1,500 identical 300-base reads on the group plan: keys of 24 words, so
    one CTA finishes at most 1,024 rows, and about 280 groups of 1,500 equal
    suffixes go to the big-group list (sized from that CTA limit) and are
    finished by LSD passes over their rows; the result is the oracle's."""
    from paper_1401_7457_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    one = np.random.default_rng(18).integers(0, 4, size=300).astype(np.uint8)
    codes, lens = np.tile(one, 1500), np.full(1500, 300, dtype=np.uint32)
    ref = oracle_of(codes, lens)
    with binding.Context(device=0, algorithm=2) as c:
        got = gpu_bwt(c, codes, lens, want_sa=True)
        assert c.stats()["big_groups"] > 221  # more than rows / 2048 + 1 big groups
    assert_same(got, ref, sa=True)
