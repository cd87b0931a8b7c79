"""The GPU results of the 10,000 x 100 bp and the genome-like 1M x 100 bp
workloads, and of every collection of the batched workload (through
cxbwt_build_batch) and every request of the served workload (through the
server, all requests queued at once), have the digests of the oracle's
results, stored in tests/golden/oracle_digests.json by
tests/golden/make_oracle_digests.py.  A collection is compared only when the
generator here draws the same one (its input digest matches): numpy does not
promise equal draws across its releases."""
import numpy as np
import pytest

import pins
from gpu_helpers import ctx, gpu_bwt  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,make", [("tiny", synth.tiny_uniform), ("genome-like", synth.genome_like)])
def test_result_digest_equals_the_oracle(ctx, name, make):  # noqa: F811
    want = pins.read_oracle_digests()[name]
    codes, lens = make()
    if pins.input_digest(codes, lens) != want["input_sha256"]:
        pytest.skip(f"this numpy draws another {name} collection than the one the digest was made from")
    got = gpu_bwt(ctx, codes, lens)
    assert len(got["bwt"]) == want["n_symbols"]
    assert pins.result_digest(got["bwt"], got["dollar_pos"], got["counts"]) == want["sha256"]


def _packed_inputs(name, items):
    """Packed reads and lengths of each item of the batched or served
    workload, after checking that this numpy draws the collections the
    digests were made from."""
    from paper_1401_7457_gb300 import binding
    specs = synth.batch_specs() if name == "batched" else synth.serve_requests()
    assert len(specs) == len(items)
    out = []
    for sp, it in zip(specs, items):
        codes, lens = synth.batch_collection(sp) if name == "batched" else synth.request_reads(sp)
        if pins.input_digest(codes, lens) != it["input_sha256"]:
            pytest.skip(f"this numpy draws another {name} collection than the one the digest was made from")
        out.append((binding.pack_codes(codes), lens))
    return out


def test_batched_workload_digests():
    """All 256 collections of the batched workload (8.04 Gbase, read lengths
    36 to 150) in one cxbwt_build_batch call on device buffers: each result
    is the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    items = pins.read_oracle_digests()["batched"]["items"]
    dev = torch.device("cuda:0")
    colls = []
    for words, lens in _packed_inputs("batched", items):
        N = int(lens.sum()) + lens.size
        colls.append((torch.from_numpy(words.view(np.int32)).to(dev), torch.from_numpy(lens.view(np.int32)).to(dev),
                      torch.zeros((N + 15) // 16, dtype=torch.int32, device=dev),
                      torch.zeros(lens.size, dtype=torch.int64, device=dev), torch.zeros(5, dtype=torch.int64, device=dev)))
    with binding.Context(device=0) as c:
        c.build_batch(colls)
    torch.cuda.synchronize()
    bad = [j for j, (cl, it) in enumerate(zip(colls, items))
           if pins.packed_result_digest(cl[2].cpu().numpy().view(np.uint32), cl[3].cpu().numpy().view(np.uint64),
                                        cl[4].cpu().numpy().view(np.uint64)) != it["packed_sha256"]]
    assert not bad, f"collections {bad[:10]} differ from the oracle"
def test_served_workload_digests():
    """All 256 requests of the served workload (34.3 Gbase) queued on a
    server at once (2 workers, each request built alone as its worker frees
    up: every one is above the size packs are made of): each result, written
    to pinned host buffers, is the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    items = pins.read_oracle_digests()["served"]["items"]
    reqs, outs = [], []
    for words, lens in _packed_inputs("served", items):
        N = int(lens.sum()) + lens.size
        reqs.append((torch.from_numpy(words.view(np.int32)).pin_memory(), torch.from_numpy(lens.view(np.int32)).pin_memory()))
        outs.append((torch.zeros((N + 15) // 16, dtype=torch.int32).pin_memory(),
                     torch.zeros(lens.size, dtype=torch.int64).pin_memory(), torch.zeros(5, dtype=torch.int64).pin_memory()))
    with binding.Server(device=0) as srv:
        tickets = [srv.submit(w, lt, *o) for (w, lt), o in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t)
        assert srv.counters()["completed"] == len(tickets)
    bad = [j for j, (o, it) in enumerate(zip(outs, items))
           if pins.packed_result_digest(o[0].numpy().view(np.uint32), o[1].numpy().view(np.uint64),
                                        o[2].numpy().view(np.uint64)) != it["packed_sha256"]]
    assert not bad, f"requests {bad[:10]} differ from the oracle"
