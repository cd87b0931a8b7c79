"""The pins catch plausible mistakes planted in the oracle.

Each case copies ``oracle/cx_oracle.cpp`` to a temporary directory, changes
one line the way a slip would (a reversed tie-break, a wrong sign, an index off
by one, a dropped compared symbol), builds it and runs the whole pin suite
against it in a separate process.  Every mutant must fail at least one pin.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cx_oracle.cpp")

MUTANTS = {
    "end_marker_order_reversed": ("return a.read < b.read;", "return a.read > b.read;"),
    "end_marker_above_bases": ("if (la != lb) return la < lb;", "if (la != lb) return la > lb;"),
    "alphabet_reversed": ("if (c != 0) return c < 0;", "if (c != 0) return c > 0;"),
    "last_symbol_not_compared": ("const uint32_t m = la < lb ? la : lb;",
                                 "const uint32_t m = la < lb ? (la ? la - 1 : 0) : (lb ? lb - 1 : 0);"),
    "preceding_symbol_off_by_one": ("R.seq[R.off[s.read] + s.pos - 1]", "R.seq[R.off[s.read] + s.pos]"),
    "dollar_at_wrong_end": ("s.pos == 0 ? '$'", "s.pos == R.len[s.read] ? '$'"),
    "rank_counts_equal_suffix": ("if (suffix_less(R, Suffix{uint64_t(i), k}, q)) ++count;",
                                 "if (!suffix_less(R, q, Suffix{uint64_t(i), k})) ++count;"),
    "certificate_skips_last_pair": ("for (int64_t r = 0; r < last; ++r) {", "for (int64_t r = 0; r < last - 1; ++r) {"),
    "bucket_symbol_order_reversed": ("code = code * 5 + s;", "code = code * 5 + (4 - s);"),
    "bucket_end_marker_above_bases": ("    uint64_t s = 0;\n    if (k + uint32_t(t) < len[i]) {",
                                      "    uint64_t s = 5;\n    if (k + uint32_t(t) < len[i]) {"),
    "range_drops_its_first_bucket": ("if (b >= bucket_lo && b < bucket_hi) mine.push_back",
                                     "if (b > bucket_lo && b < bucket_hi) mine.push_back"),
}

RUNNER = r"""
import json, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, pins
lib = oracle.load_library({lib!r})
print(json.dumps(pins.run_all_pins(lib, n_random=300)))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.cpp"
    mutated.write_text(src.replace(before, after))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-shared", "-fPIC", str(mutated), "-o", str(lib)])
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=str(lib))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    if p.returncode != 0:
        return  # the broken oracle crashed or raised inside a pin: caught
    failed = json.loads(p.stdout.strip().splitlines()[-1])
    assert failed, f"mutant {name} passed every pin"


def test_unmutated_oracle_passes_every_pin():
    import pins
    assert pins.run_all_pins() == []
