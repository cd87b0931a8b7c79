"""Writes ``oracle_digests.json``: the SHA-256 digest of the oracle's result
for seeded synthetic workloads, so that a parity test can check a GPU result
against the oracle's at full size from a stored value.

Only the oracle (``oracle/``) and the seeded input generators
(``paper_1401_7457_gb300/synth.py``, which hold none of the method's
arithmetic) are called.  From the repository root:

    python tests/golden/make_oracle_digests.py [workload ...]

(no name: every workload; the entries of the others already in the file are
kept).

Digests (``tests/pins.py``):

* ``sha256`` (``result_digest``): SHA-256 over the BWT as ASCII over "$ACGT"
  (N bytes), then the $ row of every read (n little-endian uint64), then the
  counts of $, A, C, G, T (5 little-endian uint64);
* ``packed_sha256`` (``packed_result_digest``): the same result with the BWT
  packed two bits per symbol by ``pins.pack_symbols`` (numpy, not the
  library), for the workloads whose ASCII BWT runs to gigabytes.

``input_sha256`` (``input_digest``) identifies the collection a digest belongs
to: numpy does not promise the same draws from one seed across its releases,
so a test that regenerates a collection checks it first.

The repeat-rich workload (5.05G suffixes) is sorted one range of 4-symbol
prefix buckets at a time (``oracle.sorted_ranges``), so that the host holds
one range's suffix list at a time; the batched and served workloads are
digested collection by collection.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import pins  # noqa: E402
from paper_1401_7457_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_digests.json")

WHOLE = {
    "tiny": ("10,000 reads x 100 bp, i.i.d. uniform bases, seed 1", synth.tiny_uniform),
    "genome-like": ("1,000,000 reads x 100 bp from both strands of a 5 Mbp uniform genome, 1% substitutions, "
                    "seed 2", synth.genome_like),
}
REPEAT_RICH = ("50,000,000 reads x 100 bp from both strands of a 100 Mbp genome with 5% in 10-copy 1 kb repeats "
               "at 0.5% divergence, 1% substitutions, seed 3")
BATCHED = "256 collections: n log-uniform in [10k, 2M], length from {36, 76, 100, 150}, genome-like reads, seed 4"
SERVED = "256 requests: n log-uniform in [50k, 5M], length from {100, 150}, i.i.d. uniform reads, seed 5"
NAMES = list(WHOLE) + ["repeat-rich", "batched", "served"]


def digest_whole(codes, lens, threads, ascii_too):
    res = oracle.bwt(oracle.Collection(codes, lens), threads=threads)
    out = {"n_reads": int(lens.size), "n_symbols": len(res["bwt"]), "input_sha256": pins.input_digest(codes, lens),
           "packed_sha256": pins.packed_result_digest(pins.pack_symbols(res["bwt"]), res["dollar_pos"],
                                                      res["counts"])}
    if ascii_too:
        out["sha256"] = pins.result_digest(res["bwt"], res["dollar_pos"], res["counts"])
    return out


def digest_ranged(codes, lens, threads, max_rows=500_000_000):
    """The packed digest of a collection too large for one suffix list."""
    in_sha = pins.input_digest(codes, lens)
    col = oracle.Collection(codes, lens)
    del codes
    N, n = col.n_suffixes, col.n
    sym = np.empty(N, dtype=np.uint8)
    dollar = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
    for row0, b, sr, sp in oracle.sorted_ranges(col, 4, max_rows, threads=threads):
        sym[row0:row0 + len(b)] = np.frombuffer(b, dtype=np.uint8)
        at = np.nonzero(sp == 0)[0]
        dollar[sr[at].astype(np.int64)] = (row0 + at).astype(np.uint64)
        print(f"  rows {row0:,} .. {row0 + len(b):,}", flush=True)
    counts = np.array([np.count_nonzero(sym == ord(c)) for c in "$ACGT"], dtype=np.uint64)
    return {"n_reads": n, "n_symbols": N, "input_sha256": in_sha,
            "packed_sha256": pins.packed_result_digest(pins.pack_symbols(sym), dollar, counts)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", choices=NAMES + [[]], default=[])
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    names = args.names or NAMES
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)

    def save():
        with open(OUT + ".tmp", "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        os.replace(OUT + ".tmp", OUT)

    for name in names:
        t0 = time.time()
        if name in WHOLE:
            desc, make = WHOLE[name]
            codes, lens = make()
            out[name] = {"workload": desc, **digest_whole(codes, lens, args.threads, ascii_too=True)}
        elif name == "repeat-rich":
            codes, lens = synth.repeat_rich()
            out[name] = {"workload": REPEAT_RICH, **digest_ranged(codes, lens, args.threads)}
        else:
            items = []
            specs = synth.batch_specs() if name == "batched" else synth.serve_requests()
            for j, sp in enumerate(specs):
                codes, lens = synth.batch_collection(sp) if name == "batched" else synth.request_reads(sp)
                items.append({"n_reads": int(lens.size), "length": int(lens[0]), "seed": sp["seed"],
                              **digest_whole(codes, lens, args.threads, ascii_too=False)})
                print(f"  {name} {j}: {lens.size:,} x {lens[0]}", flush=True)
            out[name] = {"workload": BATCHED if name == "batched" else SERVED, "items": items}
        save()
        print(name, f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
