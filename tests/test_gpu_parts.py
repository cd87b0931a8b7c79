"""Bucket-range parts on the GPU: every part built by cxbwt_build_part and
merged equals the oracle's B_R (and the whole build), for several part counts
and device budgets small enough that a part is itself built in slices; the
checkpointed rounds give the same files after an interruption; and the
bucket counts equal the ones the test counts from the reads."""
import numpy as np
import pytest

from gpu_helpers import ctx, oracle_of  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _collection(n, L, seed):
    g = synth.random_genome(max(n * L // 20, 2 * L), seed)
    return synth.sample_reads(g, n, L, seed + 1, 0.01)


def _bucket_counts_host(codes, lens):
    L = int(lens[0])
    n = lens.size
    r = codes.reshape(n, L).astype(np.int64)
    pad = np.concatenate([r, np.zeros((n, 8), dtype=np.int64)], axis=1)
    b = np.zeros((n, L + 1), dtype=np.int64)
    for j in range(8):
        b = (b << 2) | pad[:, j:j + L + 1]
    return np.bincount(b.ravel(), minlength=65536).astype(np.uint64)


def _words(ref_bwt: bytes) -> np.ndarray:
    code = np.zeros(256, dtype=np.uint32)
    code[ord("C")], code[ord("G")], code[ord("T")] = 1, 2, 3
    sym = code[np.frombuffer(ref_bwt, dtype=np.uint8)]
    pad = (-sym.size) % 16
    sym = np.concatenate([sym, np.zeros(pad, dtype=np.uint32)]).reshape(-1, 16)
    return np.bitwise_or.reduce(sym << (30 - 2 * np.arange(16, dtype=np.uint32)), axis=1).astype(np.uint32)


@pytest.mark.parametrize("where", ["device", "host"])
def test_bucket_counts(ctx, where):  # noqa: F811
    from paper_1401_7457_gb300 import binding
    codes, lens = _collection(3000, 100, 41)
    words = binding.pack_codes(codes)
    if where == "device":
        words = torch.from_numpy(words.view(np.int32)).cuda()
        lens_in = torch.from_numpy(lens.view(np.int32)).cuda()
    else:
        lens_in = lens
    got = ctx.bucket_counts(words, lens_in)
    assert np.array_equal(got, _bucket_counts_host(codes, lens))


@pytest.mark.parametrize("n_parts", [1, 2, 3, 7])
@pytest.mark.parametrize("where", ["device", "host"])
def test_parts_merge_to_oracle(ctx, n_parts, where):  # noqa: F811
    from paper_1401_7457_gb300 import binding, parts
    codes, lens = _collection(20000, 100, 43)
    ref = oracle_of(codes, lens)
    words = binding.pack_codes(codes)
    if where == "device":
        words = torch.from_numpy(words.view(np.int32)).cuda()
        lens_in = torch.from_numpy(lens.view(np.int32)).cuda()
    else:
        lens_in = lens
    counts = ctx.bucket_counts(words, lens_in)
    res = parts.empty_result(len(ref["bwt"]), lens.size)
    plan = parts.plan_parts(counts, n_parts)
    for p in plan:
        # Half the parts take the counts from the caller, half count again.
        given = counts if p.lo % 2 == 0 else None
        parts.merge_into(res, p, *parts.build_part_host(ctx, words, lens_in, p, bucket_counts=given))
    torch.cuda.synchronize()
    assert np.array_equal(res[0], _words(ref["bwt"]))
    assert np.array_equal(res[1], ref["dollar_pos"])
    assert np.array_equal(res[2], ref["counts"])


def test_parts_in_slices_under_a_small_budget():
    """A device budget that holds a third of a part: each part is built in
    several slices, and the merge still equals the oracle."""
    from paper_1401_7457_gb300 import binding, parts
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    codes, lens = _collection(60000, 100, 47)
    ref = oracle_of(codes, lens)
    words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).cuda()
    lens_d = torch.from_numpy(lens.view(np.int32)).cuda()
    N = int(lens.sum()) + lens.size
    with binding.Context(device=0, budget_bytes=(6 << 20) + int((2 * 4 + 8 + 8 / 33 + 1.5) * N / 6)) as c:
        plan = parts.plan_parts(c.bucket_counts(words, lens_d), 2)
        res = parts.empty_result(N, lens.size)
        for p in plan:
            c.reset_stats()
            parts.merge_into(res, p, *parts.build_part_host(c, words, lens_d, p))
            assert c.stats()["slices"] >= 2
    assert np.array_equal(res[0], _words(ref["bwt"]))
    assert np.array_equal(res[1], ref["dollar_pos"])


def test_rounds_resume_on_gpu(ctx, tmp_path):  # noqa: F811
    from paper_1401_7457_gb300 import binding, parts
    codes, lens = _collection(8000, 100, 53)
    ref = oracle_of(codes, lens)
    words = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).cuda()
    lens_d = torch.from_numpy(lens.view(np.int32)).cuda()
    out = str(tmp_path / "r")
    st = parts.build_rounds(ctx, words, lens_d, 5, out, stop_after=3)
    assert st["next"] == 3
    st = parts.build_rounds(ctx, words, lens_d, 5, out)
    assert st["done"]
    assert np.array_equal(np.fromfile(f"{out}/bwt.u32", dtype=np.uint32), _words(ref["bwt"]))
    assert np.array_equal(np.fromfile(f"{out}/dollar.u64", dtype=np.uint64), ref["dollar_pos"])
    assert st["counts"] == [int(x) for x in ref["counts"]]


def test_part_rejects_bad_ranges(ctx):  # noqa: F811
    from paper_1401_7457_gb300 import binding
    codes, lens = _collection(100, 50, 59)
    words = binding.pack_codes(codes)
    for lo, hi in ((5, 5), (7, 3), (0, 65537)):
        with pytest.raises(binding.CxbwtError) as e:
            ctx.build_part(words, lens, lo, hi, 0, 10)
        assert e.value.status == -1


@pytest.mark.parametrize("n_parts", [1, 3])
def test_parts_of_mixed_read_lengths(ctx, n_parts):  # noqa: F811
    """Reads of 20 to 300 bases: the bucket counts sum to N, and the parts
    (each listed with the mixed-length generated pass and, past 255 bases,
    the high byte of the suffix length) merge to the oracle's result."""
    from paper_1401_7457_gb300 import binding, parts
    codes, lens = synth.mixed_length_reads(6000, 20, 300, 3)
    ref = oracle_of(codes, lens)
    words = binding.pack_codes(codes)
    counts = ctx.bucket_counts(words, lens)
    assert int(counts.sum()) == len(ref["bwt"])
    res = parts.empty_result(len(ref["bwt"]), lens.size)
    for p in parts.plan_parts(counts, n_parts):
        parts.merge_into(res, p, *parts.build_part_host(ctx, words, lens, p, bucket_counts=counts))
    assert np.array_equal(res[0], _words(ref["bwt"]))
    assert np.array_equal(res[1], ref["dollar_pos"])


def test_part_rejects_counts_of_another_collection(ctx):  # noqa: F811
    from paper_1401_7457_gb300 import binding
    codes, lens = _collection(2000, 100, 61)
    words = binding.pack_codes(codes)
    counts = ctx.bucket_counts(words, lens)
    counts[5] += 1
    with pytest.raises(binding.CxbwtError) as e:
        ctx.build_part(words, lens, 0, 65536, 0, int(counts.sum()) - 1, bucket_counts=counts)
    assert e.value.status == -1
