"""Failure handling without a GPU fault: a device-side wait that nothing
satisfies runs out after its limit, the build returns CXBWT_ETIMEOUT, and the
context keeps working.  Bad input is rejected on the host before any device
work; an exhausted budget gives CXBWT_ENOMEM."""
import numpy as np
import pytest

from gpu_helpers import assert_same, gpu_bwt, oracle_of  # noqa: F401
from paper_1401_7457_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_lookback_wait_runs_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7457_gb300 import binding
    codes, lens = synth.uniform_reads(20_000, 100, 51)
    words = binding.pack_codes(codes)
    with binding.Context(device=0, plan_flags=binding.Context.PLAN_TEST_STALL, wait_limit_ms=20) as c:
        with pytest.raises(binding.CxbwtError) as e:
            c.build(words, lens)
        assert e.value.status == -4  # CXBWT_ETIMEOUT
        assert "limit" in str(e.value)
        # The same context answers again (the same way: the hook stalls every build).
        with pytest.raises(binding.CxbwtError) as e:
            c.build(words, lens)
        assert e.value.status == -4
    # A fresh context on the same device, and builds after the timed-out one, work.
    with binding.Context(device=0) as c:
        assert_same(gpu_bwt(c, codes, lens), oracle_of(codes, lens))
