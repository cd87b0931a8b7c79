"""cxbwt_build_batch: every collection's result equals the oracle's (and
cxbwt_build's on that collection alone), whether the collection was packed
with others of its read length or built alone."""
import math

import numpy as np
import pytest

from gpu_helpers import assert_same, oracle_of  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_batch(k, seed, n_min=300, n_max=12_000):
    """k genome-like collections, lengths from the batched workload's set."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(k):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(synth.BATCH_LENGTHS[int(rng.integers(0, 4))])
        g = synth.random_genome(max(2 * L, n * L // 30), seed * 1000 + c)
        out.append(synth.sample_reads(g, n, L, seed * 1000 + c + 500, 0.01))
    return out


def run_batch(ctx, colls, where):
    from paper_1401_7457_gb300 import binding
    dev = torch.device("cuda:0")
    args, outs = [], []
    for codes, lens in colls:
        words = binding.pack_codes(codes)
        N = int(lens.sum()) + lens.size
        if where == "device":
            w = torch.from_numpy(words.view(np.int32)).to(dev)
            ln = torch.from_numpy(lens.view(np.int32)).to(dev)
            bwt = torch.zeros((N + 15) // 16, dtype=torch.int32, device=dev)
            dpos = torch.zeros(lens.size, dtype=torch.int64, device=dev)
            cnt = torch.zeros(5, dtype=torch.int64, device=dev)
        else:
            w, ln = words, lens
            bwt = np.zeros((N + 15) // 16, dtype=np.uint32)
            dpos = np.zeros(lens.size, dtype=np.uint64)
            cnt = np.zeros(5, dtype=np.uint64)
        args.append((w, ln, bwt, dpos, cnt))
        outs.append((N, bwt, dpos, cnt))
    ctx.build_batch(args)
    torch.cuda.synchronize()
    res = []
    for N, bwt, dpos, cnt in outs:
        if where == "device":
            bwt, dpos, cnt = bwt.cpu().numpy(), dpos.cpu().numpy(), cnt.cpu().numpy()
        bwt, dpos, cnt = bwt.view(np.uint32), dpos.view(np.uint64), cnt.view(np.uint64)
        res.append({"bwt": binding.unpack_ascii(bwt, dpos, N), "dollar_pos": dpos, "counts": cnt})
    return res


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("flags", [0, 1])
def test_batch_matches_oracle(where, flags):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    colls = small_batch(24, 5 + flags)
    with binding.Context(device=0, plan_flags=flags) as ctx:
        got = run_batch(ctx, colls, where)
        st = ctx.stats()
    assert st["builds"] == len(colls)
    assert st["slices"] < len(colls)  # collections of one length were packed
    for (codes, lens), g in zip(colls, got):
        assert_same(g, oracle_of(codes, lens))


def test_batch_mixed_and_alone():
    """A mixed-length collection and reads too long for the group plan are built
    alone; the packed ones around them are unaffected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    colls = small_batch(6, 9)
    colls.insert(2, synth.mixed_length_reads(3000, 20, 120, 91))
    colls.insert(4, synth.uniform_reads(300, 400, 92))
    with binding.Context(device=0) as ctx:
        got = run_batch(ctx, colls, "device")
    for (codes, lens), g in zip(colls, got):
        assert_same(g, oracle_of(codes, lens))


def test_batch_equals_single_builds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    colls = small_batch(12, 11, n_min=2_000, n_max=40_000)
    with binding.Context(device=0) as ctx:
        got = run_batch(ctx, colls, "device")
        for (codes, lens), g in zip(colls, got):
            w = torch.from_numpy(binding.pack_codes(codes).view(np.int32)).cuda()
            b, d, c = ctx.build(w, torch.from_numpy(lens.view(np.int32)).cuda())
            N = int(lens.sum()) + lens.size
            one = binding.unpack_ascii(b.cpu().numpy().view(np.uint32), d.cpu().numpy().view(np.uint64), N)
            assert one == g["bwt"]
            assert np.array_equal(d.cpu().numpy().view(np.uint64), g["dollar_pos"])
