"""Device-memory-bounded builds (Figure 2 steps 1-3): the suffixes are split
into slices of consecutive 4-base buckets (8-base buckets when a 4-base one
does not fit a slice) that fit the context's budget, each
slice is sorted and emitted at its global row offset, and the result equals
the oracle's whatever the number of slices, the id width or the enumeration
order."""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_bwt, oracle_of  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def budget_for(n_suffixes, slices, id_bytes=4, host_sa=False):
    """A budget that leaves room for about n_suffixes / slices rows per slice
    (one slice: twice what it needs)."""
    per_row = 2 * id_bytes + 8 + 8 / 33 + 1 + (8 if host_sa else 0) + 0.5  # + look-back words
    if slices == 1:
        return int(6 << 20) + int(2 * per_row * n_suffixes)
    return int(6 << 20) + int(per_row * n_suffixes / slices)


@pytest.fixture(scope="module")
def genome_reads():
    g = synth.random_genome(100_000, 61)
    codes, lens = synth.sample_reads(g, 20_000, 100, 62, 0.01)
    return codes, lens, oracle_of(codes, lens)


@pytest.mark.parametrize("slices", [1, 2, 5])
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
@pytest.mark.parametrize("where", ["device", "host"])
def test_slices_identical(genome_reads, slices, flags, where):
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens, ref = genome_reads
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, slices, 8 if flags & 1 else 4, where == "host"),
                         plan_flags=flags) as c:
        got = gpu_bwt(c, codes, lens, where=where, want_sa=True)
        st = c.stats()
    assert_same(got, ref, sa=True)
    if slices == 1:
        assert st["slices"] == 1
    else:
        assert st["slices"] >= 2, st


def split_budget(n_suffixes, id_bytes=4, host=False):
    """A budget under which the build needs two slices but holds ids and keys
    for all N rows plus one spare slice: the single listing pass of every
    slice (digit = slice, suffix length) is then taken.  Rows cost
    2 * (id + key) bytes per row of the largest slice when each slice lists
    its own suffixes, and (id + key) bytes per row of N plus of the largest
    slice with the single pass; the budget sits halfway between."""
    fixed = (2 << 20) + 0.5 * n_suffixes  # tables, look-back words
    if host:
        fixed += (8 << 20) + 0.6 * n_suffixes  # read store and output staging
    one_per_row = 2 * id_bytes + 8 + 8 / 33 + (8 if host else 0)  # host: the suffix order's staging
    split_per_n = 1.53 * (id_bytes + 4) + 0.53 * (8 / 33 + 8 / 1025) + (0.53 * 8 if host else 0)
    return int(fixed + n_suffixes * (one_per_row + split_per_n) / 2)


@pytest.mark.parametrize("flags", [0, 1, 8, 9])
@pytest.mark.parametrize("where", ["device", "host"])
def test_split_listing_pass(genome_reads, flags, where):
    """Two slices listed by one generating pass over every suffix (each
    slice's rows written to its own part of one array, ordered by suffix
    length, then sorted between that part and a spare array): the oracle's
    result, suffix order included, with 32- and 64-bit ids, with and without
    the preceding base in the ids."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens, ref = genome_reads
    N = int(lens.sum()) + lens.size
    idb = 8 if flags & 1 else 4
    with binding.Context(device=0, budget_bytes=split_budget(N, idb, where == "host"), plan_flags=flags) as c:
        got = gpu_bwt(c, codes, lens, where=where, want_sa=True)
        st = c.stats()
    assert_same(got, ref, sa=True)
    assert st["slices"] == 2, st
    # One listing pass, then the four window passes of each slice (a pass per
    # slice listing its suffixes would make ten).
    assert st["sort_pass_launches"] == 9, st
    assert st["carried_pass_launches"] == 8, st


def test_uniform_random_slices():
    """i.i.d. reads (mostly distinct 16-base prefixes) in several slices."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(15_000, 100, 63)
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 3)) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)
        assert c.stats()["slices"] >= 2


def test_slices_from_8_base_buckets():
    """Reads of 20 bases that all start with AAAA, under a budget of about 14
    slices: bucket AAAA holds the n terminator-only suffixes and the n whole
    reads (2/21 of all suffixes), more than a slice, so the planner counts
    8-base buckets instead, where the largest holds the n terminators alone
    (1/21)."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(600_000, 20, 64)
    codes = codes.reshape(-1, 20).copy()
    codes[:, :4] = 0
    codes = codes.ravel()
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 14)) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)
        assert c.stats()["slices"] >= 11


def test_refined_8_base_bucket():
    """Reads of 20 bases that all start with AAAAAAAA, under a budget of
    about 14 slices: the 8-base bucket AAAAAAAA holds the n terminator-only
    suffixes and the n whole reads (2/21 of all suffixes), more than a slice
    can hold, so it is refined by the next 8 bases (Section 3.1) into 16-base
    buckets, the largest of which holds the n terminators (1/21)."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(600_000, 20, 65)
    codes = codes.reshape(-1, 20).copy()
    codes[:, :8] = 0
    codes = codes.ravel()
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    for where in ("device", "host"):
        # Host buffers also hold the read store and the output staging on the device.
        budget = budget_for(N, 14, host_sa=where == "host") + (20 << 20 if where == "host" else 0)
        with binding.Context(device=0, budget_bytes=budget) as c:
            assert_same(gpu_bwt(c, codes, lens, where=where, want_sa=True), ref, sa=True)
            assert c.stats()["slices"] >= 11


def test_one_bucket_larger_than_a_slice_is_enomem():
    """All-A reads put every suffix in one 16-base bucket, even after the
    refinement of the 8-base bucket: no slice can hold it."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = np.zeros(20_000 * 50, dtype=np.uint8), np.full(20_000, 50, dtype=np.uint32)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 4)) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -2


@pytest.mark.parametrize("lo,hi", [(50, 100), (1, 30), (200, 300)])
@pytest.mark.parametrize("flags", [0, 1])
def test_mixed_length_slices(lo, hi, flags):
    """Reads of mixed lengths in several slices: each slice lists its
    suffixes in read-major order over reads of any length (a binary search
    for each warp's first read), ordered by the low then, past 255 bases, the
    high byte of the suffix length; with 32- and 64-bit ids."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    n = {30: 200_000, 100: 20_000, 300: 6_000}[hi]  # a few million suffixes: several slices under the budget
    codes, lens = synth.mixed_length_reads(n, lo, hi, 64)
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 4, 8 if flags else 4), plan_flags=flags) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)
        assert c.stats()["slices"] >= 3


@pytest.mark.parametrize("flags", [0, 1 | 8])
def test_group_depth_12_in_slices(genome_reads, flags):
    """The group plan with l = 12 (three LSD passes, groups finished from
    base 12 on) in a build of about three device-memory-bounded slices, with
    32-bit ids and with 64-bit ids carrying the preceding base."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens, ref = genome_reads
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, prefix_len=12, plan_flags=flags,
                         budget_bytes=budget_for(N, 3, 8 if flags & 1 else 4)) as c:
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), ref, sa=True)
        assert c.stats()["slices"] >= 2


@pytest.mark.parametrize("length,n", [(20, 100_000), (60, 40_000), (100, 20_000)])
@pytest.mark.parametrize("flags", [0, 1 | 8, 32])
def test_listing_kernel_split(length, n, flags):
    """Two slices listed by one pass of the listing kernel (each thread owns
    one suffix length of every read of its tile: 195, 67 or 40 reads per
    tile) or, with plan flag 32, of the general digit pass; 32-bit ids, and
    64-bit ids carrying the preceding base: the oracle's result."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    g = synth.random_genome(n * length // 20, 130 + length)
    codes, lens = synth.sample_reads(g, n, length, 131 + length, 0.01)
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=split_budget(N, 8 if flags & 1 else 4), plan_flags=flags) as c:
        got = gpu_bwt(c, codes, lens, want_sa=True)
        st = c.stats()
    assert_same(got, ref, sa=True)
    assert st["slices"] == 2 and st["sort_pass_launches"] == 9, st


@pytest.mark.parametrize("length,n", [(20, 100_000), (100, 20_000), (150, 12_000), (255, 6_000)])
@pytest.mark.parametrize("flags", [2, 2 | 1 | 8, 2 | 32])
def test_listing_kernel_per_slice(length, n, flags):
    """About four slices, each listed by its own read-major pass over every
    suffix that keeps the slice's key range (plan flag 2 takes the read-major
    listing although the store fits L2): the listing kernel with one key
    range (128 threads up to 127 bases, 256 above) or the digit pass (flag
    32); the oracle's result."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    g = synth.random_genome(n * length // 20, 140 + length)
    codes, lens = synth.sample_reads(g, n, length, 141 + length, 0.01)
    ref = oracle_of(codes, lens)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 4, 8 if flags & 1 else 4), plan_flags=flags) as c:
        got = gpu_bwt(c, codes, lens, want_sa=True)
        st = c.stats()
    assert_same(got, ref, sa=True)
    assert st["slices"] >= 3, st
