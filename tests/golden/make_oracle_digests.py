"""Writes ``oracle_digests.json``: the SHA-256 digest of the oracle's result
for seeded synthetic workloads, so that a parity test can check a GPU result
against the oracle's at full size from a stored value.

Only the oracle (``oracle/``) and the seeded input generators
(``paper_1401_7457_gb300/synth.py``, which hold none of the method's
arithmetic) are called.  From the repository root:

    python tests/golden/make_oracle_digests.py

The digest of a result (``result_digest`` in ``tests/pins.py``) is SHA-256
over the BWT as ASCII over "$ACGT" (N bytes), then the $ row of every read
(n little-endian uint64), then the counts of $, A, C, G, T (5 little-endian
uint64).  ``input_sha256`` (``input_digest``) identifies the collection the
digest belongs to: numpy does not promise the same draws from one seed across
its releases, so a test that regenerates the collection checks it first.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import pins  # noqa: E402
from paper_1401_7457_gb300 import synth  # noqa: E402

WORKLOADS = {
    "tiny": ("10,000 reads x 100 bp, i.i.d. uniform bases, seed 1", synth.tiny_uniform),
    "genome-like": ("1,000,000 reads x 100 bp from both strands of a 5 Mbp uniform genome, 1% substitutions, "
                    "seed 2", synth.genome_like),
}


def main():
    threads = os.cpu_count() or 1
    out = {}
    for name, (desc, make) in WORKLOADS.items():
        codes, lens = make()
        res = oracle.bwt(oracle.Collection(codes, lens), threads=threads)
        out[name] = {"workload": desc, "n_reads": int(lens.size), "n_symbols": len(res["bwt"]),
                     "input_sha256": pins.input_digest(codes, lens),
                     "sha256": pins.result_digest(res["bwt"], res["dollar_pos"], res["counts"])}
        print(name, out[name]["sha256"], flush=True)
    with open(os.path.join(HERE, "oracle_digests.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
