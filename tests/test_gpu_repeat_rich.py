"""The repeat-rich workload: reads from a genome where 5% of the sequence is
copies of 1 kb segments (10 copies each, 0.5% divergence), built in several
device-memory-bounded slices with the BWT streamed to pinned host memory.

* one tenth of the workload (5M reads, 505M suffixes): every symbol, $ row and
  count against the oracle's full sort;
* the full workload (50M reads x 100 bp, 5.05G suffixes, 64-bit suffix ids,
  at least three slices): the whole result (every symbol, $ row and count)
  against the digest of the oracle's result, stored by
  tests/golden/make_oracle_digests.py (the oracle sorted it one range of
  prefix buckets at a time); then exact symbol counts, the first n symbols,
  every $ row, and sampled rows whose suffix the oracle ranks one by one.
"""
import os

import numpy as np
import pytest

import oracle
import pins
from gpu_helpers import assert_same  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def build_sliced(codes, lens, budget, want_sa_device=False):
    """Device-resident reads, host (pinned) BWT / $ rows / counts; optional device SA."""
    from paper_1401_7457_gb300 import binding
    words = binding.pack_codes(codes)
    dev = torch.device("cuda:0")
    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    d_lens = torch.from_numpy(lens.view(np.int32)).to(dev)
    N = int(lens.sum()) + lens.size
    h_bwt = torch.empty((N + 15) // 16, dtype=torch.int32).pin_memory()
    h_dpos = torch.empty(lens.size, dtype=torch.int64).pin_memory()
    h_cnt = torch.zeros(5, dtype=torch.int64).pin_memory()
    d_sa = torch.empty(N, dtype=torch.int64, device=dev) if want_sa_device else None
    with binding.Context(device=0, budget_bytes=budget) as c:
        c.build(d_words, d_lens, h_bwt, h_dpos, h_cnt, out_sa=d_sa)
        st = c.stats()
    del d_words, d_lens
    return h_bwt.numpy().view(np.uint32), h_dpos.numpy().view(np.uint64), h_cnt.numpy().view(np.uint64), d_sa, st


def symbols_at(words, rows):
    rows = np.asarray(rows, dtype=np.int64)
    return (words[rows >> 4] >> (30 - 2 * (rows & 15)).astype(np.uint32)) & 3


def test_repeat_rich_tenth_full_parity():
    _need_gpu()
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.repeat_rich(n_reads=5_000_000, genome_size=10_000_000)
    N = int(lens.sum()) + lens.size
    budget = (400 << 20) + int(0.5 * N) + int(17.25 * N / 3)  # look-back words + a third of the suffixes per slice
    bwt, dpos, cnt, _, st = build_sliced(codes, lens, budget)
    assert st["slices"] >= 3, st
    ref = oracle.bwt(oracle.Collection(codes, lens), threads=THREADS)
    got = {"bwt": binding.unpack_ascii(bwt, dpos, N), "dollar_pos": dpos, "counts": cnt}
    assert_same(got, ref)


@pytest.fixture(scope="module")
def full_build():
    """The whole repeat-rich workload, built once in device-memory-bounded
    slices (a third of the suffixes each) with the suffix order on the device."""
    _need_gpu()
    codes, lens = synth.repeat_rich()
    N = int(lens.sum()) + lens.size
    assert N == 5_050_000_000
    budget = (2 << 30) + int(0.5 * N) + int(25.25 * N / 3)
    bwt, dpos, cnt, d_sa, st = build_sliced(codes, lens, budget, want_sa_device=True)
    yield codes, lens, bwt, dpos, cnt, d_sa, st
    del d_sa
    torch.cuda.empty_cache()


def test_repeat_rich_full_size_digest(full_build):
    """Every symbol, $ row and count of the 5.05G-suffix build equals the
    oracle's result (its stored digest)."""
    codes, lens, bwt, dpos, cnt, _, st = full_build
    want = pins.read_oracle_digests()["repeat-rich"]
    if pins.input_digest(codes, lens) != want["input_sha256"]:
        pytest.skip("this numpy draws another repeat-rich collection than the one the digest was made from")
    assert st["slices"] >= 3, st
    assert bwt.size == (want["n_symbols"] + 15) // 16
    assert pins.packed_result_digest(bwt, dpos, cnt) == want["packed_sha256"]


def test_repeat_rich_default_budget_digest(full_build):
    """The build as the benchmark runs it: the default budget, two slices
    (N > 2^32 rows) listed by one pass, device-resident input and outputs.
    The whole result equals the oracle's."""
    from paper_1401_7457_gb300 import binding
    codes, lens = full_build[0], full_build[1]
    want = pins.read_oracle_digests()["repeat-rich"]
    if pins.input_digest(codes, lens) != want["input_sha256"]:
        pytest.skip("this numpy draws another repeat-rich collection than the one the digest was made from")
    dev = torch.device("cuda:0")
    N = int(lens.sum()) + lens.size
    d_words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).to(dev)
    d_lens = torch.from_numpy(lens.view(np.int32)).to(dev)
    bwt = torch.empty((N + 15) // 16, dtype=torch.int32, device=dev)
    dpos = torch.empty(lens.size, dtype=torch.int64, device=dev)
    cnt = torch.zeros(5, dtype=torch.int64, device=dev)
    with binding.Context(device=0) as c:
        c.build(d_words, d_lens, bwt, dpos, cnt)
        st = c.stats()
    assert st["slices"] == 2 and st["sort_pass_launches"] == 9, st  # one listing pass, 4 window passes per slice
    got = pins.packed_result_digest(bwt.cpu().numpy().view(np.uint32), dpos.cpu().numpy().view(np.uint64),
                                    cnt.cpu().numpy().view(np.uint64))
    del d_words, d_lens, bwt, dpos, cnt
    torch.cuda.empty_cache()
    assert got == want["packed_sha256"]


def test_repeat_rich_full_size_sampled(full_build):
    codes, lens, bwt, dpos, cnt, d_sa, st = full_build
    n = lens.size
    N = int(lens.sum()) + n
    assert st["slices"] >= 3, st
    # Exact counts: the input composition plus n terminators.
    comp = np.bincount(codes, minlength=4)
    assert cnt.tolist() == [n] + comp.tolist()
    # The first n rows are the terminator-only suffixes in read order: each
    # holds its read's last base.
    ends = np.arange(1, n + 1, dtype=np.int64) * 100 - 1
    assert np.array_equal(symbols_at(bwt, np.arange(n)), codes[ends])
    # Every read's $ row is distinct, past the first n rows, and holds code 0.
    assert np.unique(dpos).size == n and int(dpos.min()) >= n and int(dpos.max()) < N
    assert not symbols_at(bwt, dpos.astype(np.int64)).any()
    # Sampled rows: the oracle ranks the suffix the GPU put there, and the
    # symbol there precedes it.
    col = oracle.Collection(codes, lens)
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.integers(0, N, size=5), [n, N - 1]])
    sa = d_sa[torch.from_numpy(rows).to(d_sa.device)].cpu().numpy().view(np.uint64)
    for r, e in zip(rows.tolist(), sa.tolist()):
        i, k = e >> 16, e & 0xFFFF
        assert oracle.rank(col, i, k, threads=THREADS) == r
        want = 0 if k == 0 else int(codes[i * 100 + k - 1])
        assert int(symbols_at(bwt, [r])[0]) == want
