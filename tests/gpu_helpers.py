"""Shared helpers of the GPU tests: a module-scoped context, a build through the
C ABI returning ASCII + $ rows + counts (+ suffix order), and comparison with
the oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding, build
    build.build()
    c = binding.Context(device=0)
    yield c
    c.close()


def gpu_bwt(ctx, codes, lens, where="device", want_sa=False):
    from paper_1401_7457_gb300 import binding
    words = binding.pack_codes(codes)
    lens = np.ascontiguousarray(lens, dtype=np.uint32)
    n_sym = int(lens.sum()) + lens.size
    if where == "device":
        dev = torch.device("cuda:0")
        out = ctx.build(torch.from_numpy(words.view(np.int32)).to(dev), torch.from_numpy(lens.view(np.int32)).to(dev),
                        want_sa=want_sa)
        torch.cuda.synchronize()
        out = [o.cpu().numpy() for o in out]
    else:
        out = list(ctx.build(words, lens, want_sa=want_sa))
    bwt_words, dpos, cnt = out[0].view(np.uint32), out[1].view(np.uint64), out[2].view(np.uint64)
    res = {"bwt": binding.unpack_ascii(bwt_words, dpos, n_sym), "words": bwt_words, "dollar_pos": dpos,
           "counts": cnt}
    if want_sa:
        res["sa_read"], res["sa_pos"] = binding.decode_sa(out[3])
    return res


def assert_same(got, ref, sa=False):
    assert len(got["bwt"]) == len(ref["bwt"])
    if got["bwt"] != ref["bwt"]:
        a = np.frombuffer(got["bwt"], dtype=np.uint8)
        b = np.frombuffer(ref["bwt"], dtype=np.uint8)
        bad = np.nonzero(a != b)[0]
        raise AssertionError(f"{bad.size} BWT symbols differ, first at row {bad[0]}")
    assert np.array_equal(got["dollar_pos"], ref["dollar_pos"]), "dollar rows differ"
    assert np.array_equal(got["counts"], ref["counts"]), "counts differ"
    if sa:
        assert np.array_equal(got["sa_read"], ref["sa_read"]) and np.array_equal(got["sa_pos"], ref["sa_pos"])


def oracle_of(codes, lens):
    return oracle.bwt(oracle.Collection(codes, lens))


