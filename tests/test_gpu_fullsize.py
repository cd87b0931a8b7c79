"""Parity at the benchmark's full size: 1M genome-like reads x 100 bp
(101M suffixes), built exactly as bench.py builds it (device-resident input,
default tile shape).  Three independent checks:

* the suffix order the GPU returns is certified by the oracle: every suffix
  once, each strictly smaller than the next under the Section 2 order;
* the whole result equals the oracle's full sort, element by element;
* the size-independent invariants (counts, first n symbols, LF inversion).
"""
import os

import numpy as np
import pytest

import oracle
import pins
from gpu_helpers import assert_same, ctx, gpu_bwt  # noqa: F401
from paper_1401_7457_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def genome_like():
    codes, lens = synth.genome_like()
    return codes, lens, oracle.Collection(codes, lens)


@pytest.fixture(scope="module")
def gpu_result(ctx, genome_like):
    codes, lens, _ = genome_like
    return gpu_bwt(ctx, codes, lens, want_sa=True)


def test_certificate_of_gpu_suffix_order(genome_like, gpu_result):
    _, _, col = genome_like
    assert gpu_result["sa_read"].size == col.n_suffixes == 101_000_000
    assert oracle.check_sa(col, gpu_result["sa_read"], gpu_result["sa_pos"], threads=os.cpu_count()) == -1


def test_full_oracle_equality(genome_like, gpu_result):
    _, _, col = genome_like
    ref = oracle.bwt(col, threads=os.cpu_count())
    assert_same(gpu_result, ref, sa=True)


def test_invariants(genome_like, gpu_result):
    codes, lens, _ = genome_like
    pins.check_invariants(codes, lens, gpu_result["bwt"], gpu_result["dollar_pos"], gpu_result["counts"])


def test_sampled_ranks(genome_like, gpu_result):
    """A few suffixes ranked one by one by the oracle land at the GPU's rows."""
    _, _, col = genome_like
    rng = np.random.default_rng(11)
    for r in rng.integers(0, col.n_suffixes, size=8):
        i, k = int(gpu_result["sa_read"][r]), int(gpu_result["sa_pos"][r])
        assert oracle.rank(col, i, k, threads=os.cpu_count()) == r
