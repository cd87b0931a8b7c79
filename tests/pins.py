"""Checks that pin the oracle to something other than itself.

Each check is independent of ``oracle/cx_oracle.cpp``:

* ``rotation_bwt`` - the textbook BWT by sorting rotations (Burrows & Wheeler
  1994) of the concatenation S_0 $_0 S_1 $_1 ... S_{n-1} $_{n-1} over an
  integer alphabet in which $_i = i and the bases follow as n..n+3.  Because
  every end marker is a distinct symbol, comparing two rotations always stops at
  or before the first marker, which is exactly the order of Section 2.  Python
  list comparison does the sorting; nothing is shared with the oracle's
  comparator.
* ``rotation_rows`` - the same rotation sort, returning the suffix of each
  row: pins the oracle's rank and sortedness certificate (the two checks the
  GPU tests use at sizes the full sort cannot reach).
* worked examples (Figure 1) and hand-derived cases under ``tests/golden/``.
* closed forms: one read is the plain BWT of S$; n identical reads repeat each
  symbol of that BWT n times.
* invariants at any size: symbol counts equal the input composition plus n $;
  the first n symbols are the last bases of reads 0..n-1; LF-mapping inversion
  (Ferragina & Manzini 2000) started at row i recovers read i exactly and ends
  at that read's $ row.

The same invariants double as the full-size property checks of the GPU path.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SYMS = "$ACGT"


def rotation_bwt(reads):
    """BWT of a collection by brute-force rotation sorting (integer alphabet)."""
    n = len(reads)
    T = []
    owner = []
    for i, r in enumerate(reads):
        T.extend(n + "ACGT".index(c) for c in r)
        T.append(i)  # $_i
    total = len(T)
    rots = sorted(range(total), key=lambda p: T[p:] + T[:p])
    out = []
    for p in rots:
        prev = T[p - 1]  # cyclic: T[-1] is $_{n-1}
        out.append("$" if prev < n else "ACGT"[prev - n])
    return "".join(out)


def rotation_rows(reads):
    """(read, offset) of each rotation of the same concatenation, in sorted
    order: the suffix order of Section 2 by brute force (offset L_i names the
    rotation starting at $_i, the terminator-only suffix)."""
    n = len(reads)
    T, where = [], []
    for i, r in enumerate(reads):
        for k, c in enumerate(r):
            T.append(n + "ACGT".index(c))
            where.append((i, k))
        T.append(i)
        where.append((i, len(r)))
    rots = sorted(range(len(T)), key=lambda p: T[p:] + T[:p])
    return [where[p] for p in rots]


def result_digest(bwt_ascii: bytes, dollar_pos, counts) -> str:
    """SHA-256 of a result: the ASCII BWT, then the $ rows and the five counts
    as little-endian uint64."""
    import hashlib
    h = hashlib.sha256()
    h.update(bytes(bwt_ascii))
    h.update(np.ascontiguousarray(dollar_pos, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(counts, dtype="<u8").tobytes())
    return h.hexdigest()


def pack_symbols(bwt_ascii, chunk_words: int = 1 << 24) -> np.ndarray:
    """A BWT over "$ACGT" in the library's packed layout, written here with
    numpy (not the library's packer): codes A=0, C=1, G=2, T=3 and 0 at a $
    row, symbol r in bits [31-2(r%16) .. 30-2(r%16)] of word r/16, the bits
    past the last symbol 0."""
    sym = np.frombuffer(bwt_ascii, dtype=np.uint8) if not isinstance(bwt_ascii, np.ndarray) else bwt_ascii
    lut = np.zeros(256, dtype=np.uint32)
    for code, ch in enumerate("ACGT"):
        lut[ord(ch)] = code
    n_words = (sym.size + 15) // 16
    out = np.empty(n_words, dtype=np.uint32)
    shifts = (30 - 2 * np.arange(16, dtype=np.uint32)).astype(np.uint32)
    for w0 in range(0, n_words, chunk_words):
        w1 = min(n_words, w0 + chunk_words)
        part = sym[w0 * 16:w1 * 16]
        codes = np.zeros((w1 - w0) * 16, dtype=np.uint32)
        codes[:part.size] = lut[part]
        out[w0:w1] = np.bitwise_or.reduce(codes.reshape(-1, 16) << shifts, axis=1)
    return out


def packed_result_digest(words, dollar_pos, counts) -> str:
    """SHA-256 of a result in packed form: the BWT words (as ``pack_symbols``
    lays them out) as little-endian uint32, then the $ rows and the five
    counts as little-endian uint64.  Cheaper than ``result_digest`` at sizes
    where the ASCII BWT runs to gigabytes."""
    import hashlib
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(words, dtype="<u4")).cast("B"))
    h.update(np.ascontiguousarray(dollar_pos, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(counts, dtype="<u8").tobytes())
    return h.hexdigest()


def input_digest(codes, lens) -> str:
    """SHA-256 of a collection: its base codes (uint8), then its lengths as
    little-endian uint32."""
    import hashlib
    h = hashlib.sha256()
    h.update(memoryview(np.ascontiguousarray(codes, dtype=np.uint8)).cast("B"))
    h.update(np.ascontiguousarray(lens, dtype="<u4").tobytes())
    return h.hexdigest()


def read_oracle_digests():
    import json
    with open(os.path.join(GOLDEN, "oracle_digests.json")) as f:
        return json.load(f)


def read_figure1():
    with open(os.path.join(GOLDEN, "figure1.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    d = {r[0]: r[1:] for r in rows}
    return d["reads"], d["sorted_suffixes"], d["bwt"][0]


def read_hand_examples():
    out = []
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            reads, want = (x.strip() for x in ln.split("->"))
            out.append((reads.split(","), want))
    return out


def lf_walk(bwt: bytes, n: int, max_len: int):
    """LF walks from rows 0..n-1: an (n, max_len) matrix of the base codes met
    (read i last base first), -1 after the walk met $, and the $ rows."""
    rev, end_rows, M = _lf(bwt, n, max_len)
    return M, end_rows


def lf_invert(bwt: bytes, n: int, max_len: int):
    rev, end_rows, _ = _lf(bwt, n, max_len)
    return rev, end_rows


def _lf(bwt: bytes, n: int, max_len: int):
    """Recover every read from the BWT by LF-mapping, LF(r) = C[c] + rank_c(r).

    Returns ``(reads_reversed, end_rows, M)``: for each read i (when n is
    small) its bases in reverse order, the row at which the walk met $, and the
    int8 walk matrix.  Raises if a walk does not meet $ within ``max_len + 1``
    steps.
    """
    B = np.frombuffer(bwt, dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    for s, ch in enumerate(SYMS):
        lut[ord(ch)] = s
    sym = lut[B]
    if np.any(sym == 255):
        raise ValueError("BWT holds a symbol outside $ACGT")
    N = sym.size
    cnt = np.bincount(sym, minlength=5).astype(np.int64)
    C = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    occ = np.empty(N, dtype=np.int64)
    for s in range(5):
        m = sym == s
        occ[m] = np.arange(int(cnt[s]), dtype=np.int64)
    LF = C[sym] + occ
    rows = np.arange(n, dtype=np.int64)
    active = np.ones(n, dtype=bool)
    collected = []
    end_rows = np.full(n, -1, dtype=np.int64)
    for _ in range(max_len + 1):
        s = sym[rows]
        done = active & (s == 0)
        end_rows[done] = rows[done]
        active &= s != 0
        if not active.any():
            break
        step = np.where(active, s.astype(np.int8) - 1, -1).astype(np.int8)
        collected.append(step)
        rows = np.where(active, LF[rows], rows)
    if active.any():
        raise AssertionError("LF walk did not reach $ for some read")
    M = np.full((n, max_len), -1, dtype=np.int8)
    if collected:
        C2 = np.stack(collected, axis=1)
        M[:, :C2.shape[1]] = C2
    reads_rev = None if n > 10_000 else [M[i][M[i] >= 0].astype(np.uint8) for i in range(n)]
    return reads_rev, end_rows, M


def check_invariants(codes: np.ndarray, lens: np.ndarray, bwt: bytes, dollar_pos=None, counts=None):
    """Assert the size-independent properties of a multi-string BWT."""
    codes = np.asarray(codes, dtype=np.uint8)
    lens = np.asarray(lens, dtype=np.int64)
    n = lens.size
    N = int(lens.sum()) + n
    assert len(bwt) == N, f"BWT length {len(bwt)} != {N}"
    B = np.frombuffer(bwt, dtype=np.uint8)
    want_counts = np.concatenate([[n], np.bincount(codes, minlength=4)]).astype(np.int64)
    got_counts = np.array([np.count_nonzero(B == ord(c)) for c in SYMS], dtype=np.int64)
    assert np.array_equal(got_counts, want_counts), f"counts {got_counts} != {want_counts}"
    if counts is not None:
        assert np.array_equal(np.asarray(counts, dtype=np.int64), want_counts)
    # The n terminator-only suffixes are the n smallest, in read order; each is
    # preceded by the last base of its read.
    ends = np.cumsum(lens) - 1
    last = np.frombuffer(b"ACGT", dtype=np.uint8)[codes[ends]]
    assert np.array_equal(B[:n], last), "first n symbols are not the last bases of the reads"
    M, end_rows = lf_walk(bwt, n, int(lens.max()))
    # Expected walk of read i: its bases last to first, then -1 padding.
    off = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    want = np.full(M.shape, -1, dtype=np.int8)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    t = np.arange(rows.size, dtype=np.int64) - np.repeat(off, lens)
    want[rows, t] = codes[np.repeat(off + lens - 1, lens) - t].astype(np.int8)
    if not np.array_equal(M, want):
        bad = int(np.nonzero((M != want).any(axis=1))[0][0])
        raise AssertionError(f"LF inversion of read {bad} does not give the read back")
    if dollar_pos is not None:
        assert np.array_equal(np.asarray(dollar_pos, dtype=np.int64), end_rows), "dollar positions differ from LF walk"


# ---------------------------------------------------------------------------
# Whole pin suite against an oracle library (used by the mutant test, which
# runs it in a subprocess against deliberately broken oracle builds).
# ---------------------------------------------------------------------------

def run_all_pins(lib=None, n_random=300, seed=7):
    """Run every pin against an oracle library; returns the list of failed pin names."""
    import oracle
    from paper_1401_7457_gb300 import synth

    failed = []

    def bwt_of(reads):
        return oracle.bwt(oracle.Collection.from_strings(reads), lib=lib)["bwt"].decode()

    reads, _, want = read_figure1()
    if bwt_of(reads) != want:
        failed.append("figure1")
    for reads, want in read_hand_examples():
        if bwt_of(reads) != want:
            failed.append("hand:" + ",".join(reads))
            break
    rng = np.random.default_rng(seed)
    for _ in range(n_random):
        k = int(rng.integers(1, 6))
        alpha = "ACGT"[: int(rng.integers(1, 5))]
        reads = ["".join(rng.choice(list(alpha), size=int(rng.integers(1, 9)))) for _ in range(k)]
        if bwt_of(reads) != rotation_bwt(reads):
            failed.append("brute_force")
            break
    base = "GATTACAGATTACA"
    one = bwt_of([base])
    if bwt_of([base] * 3) != "".join(c * 3 for c in one):
        failed.append("identical_reads")
    codes, lens = synth.uniform_reads(300, 30, 11)
    col = oracle.Collection(codes, lens)
    res = oracle.bwt(col, lib=lib)
    try:
        check_invariants(codes, lens, res["bwt"], res["dollar_pos"], res["counts"])
    except AssertionError:
        failed.append("invariants")
    # Rank and certificate against the brute-force order of all rotations:
    # the rank of the suffix in row r is r, the rotation order passes the
    # certificate, and a swap of the first or the last two rows fails it there.
    reads = ["ACGTTG", "ACG", "TTGA", "ACGTTG", "G"]
    rows = rotation_rows(reads)
    col = oracle.Collection.from_strings(reads)
    sa_r = np.array([i for i, _ in rows], dtype=np.uint64)
    sa_p = np.array([k for _, k in rows], dtype=np.uint32)
    N = len(rows)
    ok = all(oracle.rank(col, i, k, lib=lib) == r for r, (i, k) in enumerate(rows))
    ok = ok and oracle.check_sa(col, sa_r, sa_p, lib=lib) == -1
    for a in (0, N - 2):
        sr, sp = sa_r.copy(), sa_p.copy()
        sr[[a, a + 1]], sp[[a, a + 1]] = sr[[a + 1, a]], sp[[a + 1, a]]
        ok = ok and oracle.check_sa(col, sr, sp, lib=lib) == a
    if not ok:
        failed.append("rank_and_certificate")
    # The sort one range of prefix buckets at a time (Section 3.1's
    # partition), concatenated, against the brute-force rotation order.
    rng = np.random.default_rng(seed + 1)
    for _ in range(max(n_random // 10, 5)):
        k = int(rng.integers(1, 6))
        alpha = "ACGT"[: int(rng.integers(1, 5))]
        reads = ["".join(rng.choice(list(alpha), size=int(rng.integers(1, 9)))) for _ in range(k)]
        if not prefix_ranges_match(reads, int(rng.integers(1, 4)), int(rng.integers(1, 8)), lib):
            failed.append("prefix_ranges")
            break
    return failed


def prefix_ranges_match(reads, p, max_rows, lib=None) -> bool:
    """The oracle's bucket-range sort, concatenated in bucket order, gives the
    rotation order and the rotation BWT, with each range starting at the rank
    of its first suffix."""
    import oracle
    col = oracle.Collection.from_strings(reads)
    try:
        parts = list(oracle.sorted_ranges(col, p, max_rows, threads=1, lib=lib))
    except RuntimeError:
        return False
    rows = [(int(i), int(k)) for _, _, sr, sp in parts for i, k in zip(sr, sp)]
    starts = [r0 for r0, _, _, _ in parts]
    sizes = [len(b) for _, b, _, _ in parts]
    if starts != [sum(sizes[:j]) for j in range(len(sizes))]:
        return False
    return rows == rotation_rows(reads) and b"".join(b for _, b, _, _ in parts).decode() == rotation_bwt(reads)
