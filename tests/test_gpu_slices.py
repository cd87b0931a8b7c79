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


def test_one_bucket_larger_than_a_slice_is_enomem():
    """All-A reads put every suffix in one 8-base bucket: no slice can hold it."""
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = np.zeros(20_000 * 50, dtype=np.uint8), np.full(20_000, 50, dtype=np.uint32)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 4)) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -2


def test_mixed_lengths_need_one_slice():
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.mixed_length_reads(20_000, 50, 100, 64)
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=budget_for(N, 4)) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(binding.pack_codes(codes), lens)
        assert e.value.status == -5
    with binding.Context(device=0, plan_flags=1) as c:  # 64-bit ids, one slice
        assert_same(gpu_bwt(c, codes, lens, want_sa=True), oracle_of(codes, lens), sa=True)
