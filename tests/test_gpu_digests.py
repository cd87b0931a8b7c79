"""The GPU results of the 10,000 x 100 bp and the genome-like 1M x 100 bp
workloads have the digests of the oracle's results, stored in
tests/golden/oracle_digests.json by tests/golden/make_oracle_digests.py.
A collection is compared only when the generator here draws the same one
(its input digest matches): numpy does not promise equal draws across its
releases."""
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
