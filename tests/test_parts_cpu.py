"""Bucket-range parts on the host (no GPU): the split of the bucket counts,
the merge of parts, the fact they rest on (Section 3.3: suffixes of a lower
bucket sort before those of a higher one, checked against the oracle), the
gather of parts across two gloo ranks, and the checkpointed rounds of
Section 3.1 with an interruption and a resume.  Every part's expected output
is cut from the oracle's B_R by the test itself."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1401_7457_gb300 import binding, parts, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_1401_7457_gb300 import build
    build.build()


CODE = {ord("$"): 0, ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def bucket_of_suffixes(codes, lens):
    """Bucket (first 8 bases, A-padded, 2 bits each, first base most
    significant) of every suffix (i, k), k = 0 .. L_i, in (read, k) order."""
    out = []
    off = 0
    for L in (int(x) for x in lens):
        r = codes[off:off + L]
        off += L
        for k in range(L + 1):
            w = list(r[k:k + 8]) + [0] * max(0, 8 - (L - k))
            b = 0
            for x in w[:8]:
                b = (b << 2) | int(x)
            out.append(b)
    return np.array(out, dtype=np.int64)


def bucket_counts(codes, lens):
    return np.bincount(bucket_of_suffixes(codes, lens), minlength=binding.BUCKETS).astype(np.uint64)


def pack_rows(bwt_ascii: bytes, row0: int, rows: int) -> np.ndarray:
    """Words of a part as cxbwt_build_part writes them: global words
    row0 // 16 .., only rows [row0, row0 + rows) set."""
    nw = binding.part_words(row0, rows)
    out = np.zeros(nw, dtype=np.uint32)
    for g in range(row0, row0 + rows):
        w = g // 16 - row0 // 16
        out[w] |= np.uint32(CODE[bwt_ascii[g]] << (30 - 2 * (g % 16)))
    return out


def oracle_part(ref, n_reads, p):
    b = ref["bwt"]
    words = pack_rows(b, p.row0, p.rows)
    d = np.full(n_reads, parts.NO_ROW, dtype=np.uint64)
    mine = (ref["dollar_pos"] >= p.row0) & (ref["dollar_pos"] < p.row0 + p.rows)
    d[mine] = ref["dollar_pos"][mine]
    return words, d, oracle.counts(b[p.row0:p.row0 + p.rows])


def whole_words(bwt_ascii: bytes) -> np.ndarray:
    return pack_rows(bwt_ascii, 0, len(bwt_ascii))


def small_collection(seed=11, n=300, L=30):
    g = synth.random_genome(2000, seed)
    return synth.sample_reads(g, n, L, seed + 1, 0.01)


def test_split_parts_bounds_and_balance():
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 50, binding.BUCKETS).astype(np.uint64)
    counts[rng.integers(0, binding.BUCKETS, 30000)] = 0
    total = int(counts.sum())
    for n_parts in (1, 2, 3, 7, 64):
        bb, rb = binding.split_parts(counts, n_parts)
        assert bb[0] == 0 and bb[-1] == binding.BUCKETS and rb[0] == 0 and rb[-1] == total
        assert np.all(np.diff(bb.astype(np.int64)) >= 0) and np.all(np.diff(rb.astype(np.int64)) >= 0)
        cum = np.concatenate([[0], np.cumsum(counts)])
        assert np.array_equal(cum[bb], rb)  # row bounds are the counts below each bucket bound
        # Every boundary is within one bucket's count of its ideal place.
        for j in range(1, n_parts):
            assert abs(int(rb[j]) - total * j / n_parts) <= int(counts.max())


def test_split_parts_more_parts_than_buckets():
    counts = np.zeros(binding.BUCKETS, dtype=np.uint64)
    counts[[3, 900]] = [5, 7]
    bb, rb = binding.split_parts(counts, 5)
    sizes = np.diff(rb.astype(np.int64))
    assert sizes.sum() == 12 and np.count_nonzero(sizes) == 2
    with pytest.raises(binding.CxbwtError):
        binding.split_parts(counts, 0)


def test_merge_part_or_and_bounds():
    bwt = np.zeros(4, dtype=np.uint32)
    binding.merge_part(bwt, np.array([0x0000FFFF, 0xF0000000], dtype=np.uint32), 8, 10)
    assert bwt.tolist() == [0x0000FFFF, 0xF0000000, 0, 0]
    binding.merge_part(bwt, np.array([0x0FF00000], dtype=np.uint32), 18, 4)
    assert bwt[1] == 0xFFF00000
    with pytest.raises(binding.CxbwtError):
        binding.merge_part(bwt, np.zeros(2, dtype=np.uint32), 60, 10)  # past the last word


def test_buckets_order_the_suffixes():
    """Section 3.3's premise on the oracle's order: the bucket of the
    suffix at row r never decreases with r, and bucket counts give each
    range's rows."""
    codes, lens = small_collection()
    col = oracle.Collection(codes, lens)
    _, sa_read, sa_pos = oracle.sort(col)
    b = bucket_of_suffixes(codes, lens)
    start = np.concatenate([[0], np.cumsum(lens.astype(np.int64) + 1)])
    sorted_b = b[start[sa_read] + sa_pos]
    assert np.all(np.diff(sorted_b) >= 0)
    counts = bucket_counts(codes, lens)
    assert int(counts.sum()) == len(sa_read)


def test_merged_oracle_parts_equal_the_whole():
    codes, lens = small_collection()
    ref = oracle.bwt(oracle.Collection(codes, lens))
    counts = bucket_counts(codes, lens)
    for n_parts in (1, 2, 5, 9):
        res = parts.empty_result(len(ref["bwt"]), lens.size)
        for p in parts.plan_parts(counts, n_parts):
            parts.merge_into(res, p, *oracle_part(ref, lens.size, p))
        assert np.array_equal(res[0], whole_words(ref["bwt"]))
        assert np.array_equal(res[1], ref["dollar_pos"])
        assert np.array_equal(res[2], ref["counts"])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle as orc
    from paper_1401_7457_gb300 import parts as P
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    codes, lens = small_collection()
    ref = orc.bwt(orc.Collection(codes, lens))
    plan = P.plan_parts(bucket_counts(codes, lens), world)
    mine = plan[rank]
    out = P.gather_parts(oracle_part(ref, lens.size, mine), mine, len(ref["bwt"]), lens.size)
    if rank == 0:
        ok = (np.array_equal(out[0], whole_words(ref["bwt"])) and np.array_equal(out[1], ref["dollar_pos"])
              and np.array_equal(out[2], ref["counts"]))
        q.put(("merged", ok, [p.rows for p in plan]))
    else:
        q.put(("rank", out is None, None))
    dist.destroy_process_group()


def test_two_ranks_gather_parts():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = {k: (v, extra) for k, v, extra in got}
    assert d["merged"][0], "rank 0's merged B_R differs from the oracle"
    assert d["rank"][0], "rank 1 must get None"
    assert all(r > 0 for r in d["merged"][1])


def test_rounds_resume_after_interruption(tmp_path):
    codes, lens = small_collection(seed=21)
    ref = oracle.bwt(oracle.Collection(codes, lens))
    counts = bucket_counts(codes, lens)
    calls = []

    def builder(p):
        calls.append(p.lo)
        return oracle_part(ref, lens.size, p)

    out = str(tmp_path / "rounds")
    st = parts.build_rounds(None, None, lens, 4, out, stop_after=2, builder=builder, bucket_counts=counts)
    assert st["next"] == 2 and not st["done"]
    st = parts.build_rounds(None, None, lens, 4, out, builder=builder, bucket_counts=counts)
    assert st["done"] and len(calls) == 4 and len(set(calls)) == 4  # no part built twice
    bwt = np.fromfile(os.path.join(out, "bwt.u32"), dtype=np.uint32)
    dpos = np.fromfile(os.path.join(out, "dollar.u64"), dtype=np.uint64)
    assert np.array_equal(bwt, whole_words(ref["bwt"]))
    assert np.array_equal(dpos, ref["dollar_pos"])
    assert st["counts"] == [int(x) for x in ref["counts"]]
    # A finished build is not redone; another round count is another plan.
    parts.build_rounds(None, None, lens, 4, out, builder=builder, bucket_counts=counts)
    assert len(calls) == 4
    with pytest.raises(ValueError):
        parts.build_rounds(None, None, lens, 3, out, builder=builder, bucket_counts=counts)


def test_rounds_for_host_budget():
    assert parts.rounds_for_host_budget(1000, 1 << 20) == 1
    assert parts.rounds_for_host_budget(4_000_000, 250_000) == 4


class OracleContext:
    """Stands in for a device context on CPU ranks: the bucket counts and
    each part's outputs come from the oracle (cut by oracle_part)."""

    def __init__(self, codes, lens):
        self.codes, self.lens = codes, lens
        self.ref = oracle.bwt(oracle.Collection(codes, lens))
        self.given = []

    def bucket_counts(self, reads_2bit, lens, stream=None):
        return bucket_counts(self.codes, self.lens)

    def build_part(self, reads_2bit, lens, lo, hi, row0, rows, stream=None, bucket_counts=None):
        self.given.append(bucket_counts is not None)
        return oracle_part(self.ref, self.lens.size, parts.Part(lo, hi, row0, rows))


def _rank_sharded(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    import test_parts_cpu as T
    from paper_1401_7457_gb300 import parts as P
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    codes, lens = T.small_collection(seed=31, n=400)
    ctx = T.OracleContext(codes, lens)
    out = P.build_sharded(ctx, T.binding.pack_codes(codes), lens)
    if rank == 0:
        ok = (np.array_equal(out[0], T.whole_words(ctx.ref["bwt"])) and np.array_equal(out[1], ctx.ref["dollar_pos"])
              and np.array_equal(out[2], ctx.ref["counts"]))
        q.put(("merged", ok, ctx.given))
    else:
        q.put(("rank", out is None, ctx.given))
    dist.destroy_process_group()


def test_two_ranks_build_sharded():
    """parts.build_sharded on two gloo ranks: each rank counts the buckets,
    builds its own part with those counts, and rank 0 gets the whole B_R."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = {k: (v, given) for k, v, given in got}
    assert d["merged"][0], "rank 0's merged B_R differs from the oracle"
    assert d["rank"][0], "rank 1 must get None"
    assert d["merged"][1] == [True] and d["rank"][1] == [True], "each rank builds one part with the counts"
