"""Serving: requests submitted together are packed and built concurrently by
several workers; every result equals the oracle's and the result of building
that request alone."""
import math

import numpy as np
import pytest

from gpu_helpers import assert_same, oracle_of  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def requests(k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(k):
        n = int(round(math.exp(rng.uniform(math.log(500), math.log(20_000)))))
        L = int(synth.SERVE_LENGTHS[int(rng.integers(0, 2))])
        out.append(synth.uniform_reads(n, L, synth.derive_seed(seed, r)))
    return out


def test_served_results_match_alone():
    """Two large requests (built alone) keep the server's workers busy while
    41 small ones queue behind them; the small ones of one read length are
    then packed and built together.  Every small result equals the oracle's
    and its own solo build; the large ones equal their solo builds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    blockers = [synth.uniform_reads(3_000_000, 100, 31 + b) for b in range(2)]  # 303M suffixes each
    reqs = requests(40, 21)
    reqs.insert(7, synth.mixed_length_reads(2000, 30, 150, 99))  # built alone inside a worker
    prepared = []
    for codes, lens in blockers + reqs:
        N = int(lens.sum()) + lens.size
        prepared.append((binding.pack_codes(codes), lens, N, np.zeros((N + 15) // 16, dtype=np.uint32),
                         np.zeros(lens.size, dtype=np.uint64), np.zeros(5, dtype=np.uint64)))
    with binding.Server(device=0, workers=2) as srv:
        tickets = [srv.submit(w, ln, b, d, c) for (w, ln, _, b, d, c) in prepared]
        for t in tickets:
            srv.wait(t)
        lat = [srv.times(t)[1] for t in tickets]
        counters = srv.counters()
    assert counters["completed"] == len(prepared)
    assert counters["packs"] < len(prepared)  # small requests were built together
    assert all(x > 0 for x in lat)
    with binding.Context(device=0) as ctx:
        for j, ((codes, lens), (w, _, N, bwt, dpos, cnt)) in enumerate(zip(blockers + reqs, prepared)):
            if j >= len(blockers):
                got = {"bwt": binding.unpack_ascii(bwt, dpos, N), "dollar_pos": dpos, "counts": cnt}
                assert_same(got, oracle_of(codes, lens))
            b, d, c = ctx.build(w, lens)
            assert np.array_equal(b, bwt) and np.array_equal(d, dpos) and np.array_equal(c, cnt)


def test_poll_and_bad_requests():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(1000, 100, 5)
    with binding.Server(device=0, workers=1) as srv:
        bwt = np.zeros((101_000 + 15) // 16, dtype=np.uint32)
        dpos = np.zeros(1000, dtype=np.uint64)
        cnt = np.zeros(5, dtype=np.uint64)
        t = srv.submit(binding.pack_codes(codes), lens, bwt, dpos, cnt)
        srv.wait(t)
        assert srv.poll(t)
        with pytest.raises(binding.CxbwtError):
            srv.submit(binding.pack_codes(codes), np.zeros(3, dtype=np.uint32), bwt)
    # The server's own $ rows and counts, against the oracle's.
    assert_same({"bwt": binding.unpack_ascii(bwt, dpos, 101_000), "dollar_pos": dpos, "counts": cnt},
                oracle_of(codes, lens))
