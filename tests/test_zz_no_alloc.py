"""cxbwt_build_noalloc, the build for callers that cannot allocate device
memory (their own pool allocator owns it, or cudaFree's device-wide
synchronisation would stall their other streams).  It must give exactly what
cxbwt_build gives, call after call, with its scratch in the library's static
array.  This file is collected last so a failure here comes after every other
test has run; it passes alone and after the rest."""
import numpy as np
import pytest

from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _both(ctx, codes, lens):
    from paper_1401_7457_gb300 import binding
    dev = torch.device("cuda:0")
    words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).to(dev)
    n = lens.size
    n_words = (int(lens.sum()) + n + 15) // 16
    ref = ctx.build(words, torch.from_numpy(lens.view(np.int32)).to(dev))
    bwt = torch.full((n_words,), -1, dtype=torch.int32, device=dev)  # garbage the call must overwrite
    dpos = torch.full((n,), -1, dtype=torch.int64, device=dev)
    cnt = torch.full((5,), -1, dtype=torch.int64, device=dev)
    binding.build_noalloc(words, lens, bwt, dpos, cnt)
    torch.cuda.synchronize()
    return ref, (bwt, dpos, cnt)


def test_noalloc_equals_build_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    cases = [
        synth.sample_reads(synth.random_genome(60_000, 71), 18_000, 100, 72, 0.01),  # 1.82M suffixes, 30x
        synth.uniform_reads(9_000, 150, 73),                                          # longer reads, fewer rows
        synth.sample_reads(synth.random_genome(60_000, 71), 18_000, 100, 72, 0.01),  # the first again
    ]
    with binding.Context(device=0) as ctx:
        for codes, lens in cases:
            (rb, rd, rc), (b, d, c) = _both(ctx, codes, lens)
            assert torch.equal(rb, b), "BWT words differ from cxbwt_build"
            assert torch.equal(rd, d), "dollar rows differ from cxbwt_build"
            assert torch.equal(rc, c), "counts differ from cxbwt_build"


@pytest.mark.parametrize("L,n", [(255, 8192), (272, 7681)])
def test_noalloc_at_its_limits(L, n):
    """Exactly CXBWT_NOALLOC_MAX_SUFFIXES suffixes (8192 reads x 255 bases),
    and the longest read length it takes (272 bases): the oracle's result,
    and the same words as cxbwt_build."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(n, L, 74 + L)
    N = n * (L + 1)
    assert N <= binding.NOALLOC_MAX_SUFFIXES and L <= binding.NOALLOC_MAX_READ_LEN
    if L == 255:
        assert N == binding.NOALLOC_MAX_SUFFIXES
    ref = oracle.bwt(oracle.Collection(codes, lens), threads=8)
    with binding.Context(device=0) as ctx:
        (rb, rd, rc), (b, d, c) = _both(ctx, codes, lens)
    assert torch.equal(rb, b) and torch.equal(rd, d) and torch.equal(rc, c)
    dpos = d.cpu().numpy().view(np.uint64)
    assert binding.unpack_ascii(b.cpu().numpy().view(np.uint32), dpos, N) == ref["bwt"]
    assert np.array_equal(dpos, ref["dollar_pos"])
    assert np.array_equal(c.cpu().numpy().view(np.uint64), ref["counts"])


def test_noalloc_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    dev = torch.device("cuda:0")
    n = binding.NOALLOC_MAX_SUFFIXES // 101 + 1  # one read too many
    lens = np.full(n, 100, dtype=np.uint32)
    words = torch.zeros((n * 100 + 15) // 16, dtype=torch.int32, device=dev)
    out = torch.zeros((n * 101 + 15) // 16, dtype=torch.int32, device=dev)
    dpos = torch.zeros(n, dtype=torch.int64, device=dev)
    cnt = torch.zeros(5, dtype=torch.int64, device=dev)
    with pytest.raises(binding.CxbwtError) as e:
        binding.build_noalloc(words, lens, out, dpos, cnt)
    assert e.value.status == -5
    mixed = np.array([100, 99], dtype=np.uint32)
    with pytest.raises(binding.CxbwtError) as e:
        binding.build_noalloc(words, mixed, out, dpos, cnt)
    assert e.value.status == -5


def test_noalloc_big_groups_on_consecutive_calls():
    """Groups of more than 2,048 suffixes that share their first 16 bases go
    to the allocation-free build's own fallback (per-group digit counts and
    LSD passes over the group's rows, in the static array): 3,000 identical
    60-base reads and 2,500 all-A reads of 50 bases, each built twice, one
    after the other, so that each call starts from the other's leftovers.
    Every result is the oracle's and the same as cxbwt_build's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1401_7457_gb300 import binding
    one = np.random.default_rng(75).integers(0, 4, size=60).astype(np.uint8)
    cases = [(np.tile(one, 3000), np.full(3000, 60, dtype=np.uint32)),
             (np.zeros(2500 * 50, dtype=np.uint8), np.full(2500, 50, dtype=np.uint32))]
    refs = [oracle.bwt(oracle.Collection(c, l), threads=8) for c, l in cases]
    with binding.Context(device=0) as ctx:
        for rep in range(2):
            for (codes, lens), ref in zip(cases, refs):
                (rb, rd, rc), (b, d, c) = _both(ctx, codes, lens)
                assert torch.equal(rb, b) and torch.equal(rd, d) and torch.equal(rc, c), rep
                N = int(lens.sum()) + lens.size
                dpos = d.cpu().numpy().view(np.uint64)
                assert binding.unpack_ascii(b.cpu().numpy().view(np.uint32), dpos, N) == ref["bwt"], rep
                assert np.array_equal(dpos, ref["dollar_pos"])
                assert np.array_equal(c.cpu().numpy().view(np.uint64), ref["counts"])
