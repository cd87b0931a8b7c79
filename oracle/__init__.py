"""CPU oracle for the multi-string BWT (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path
(``paper_1401_7457_gb300``) never imports it and shares no code with it.

It computes the definition of the BWT of a read collection in Section 2 of
Liu, Luo & Lam (arXiv 1401.7457): every suffix of every read, the
terminator-only ones included, sorted with $ below every base and
$_i < $_j for i < j; B_R[r] is the symbol before the r-th suffix, or $ when
that suffix starts at position 0.  The arithmetic lives in ``cx_oracle.cpp``
(a plain comparator handed to a library sort); this module converts inputs
and derives the per-read $ positions and the symbol counts from its result.

Inputs are base codes 0..3 (A, C, G, T) in one concatenated ``uint8`` array
plus ``uint32`` read lengths, exactly what the seeded generators produce.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cx_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcxoracle.so")
_lock = threading.Lock()
_lib = None

ALPHABET = b"ACGT"  # code c -> ASCII; A < C < G < T (Section 2 alphabet order)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (OpenMP for the parallel sort)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.cxo_sort.restype = ctypes.c_int64
    lib.cxo_sort.argtypes = [ctypes.c_char_p, u64p, u32p, ctypes.c_uint64, u64p, u32p,
                             ctypes.c_char_p, ctypes.c_int]
    lib.cxo_rank.restype = ctypes.c_int64
    lib.cxo_rank.argtypes = [ctypes.c_char_p, u64p, u32p, ctypes.c_uint64, ctypes.c_uint64,
                             ctypes.c_uint32, ctypes.c_int]
    lib.cxo_check_sa.restype = ctypes.c_int64
    lib.cxo_check_sa.argtypes = [ctypes.c_char_p, u64p, u32p, ctypes.c_uint64, u64p, u32p,
                                 ctypes.c_uint64, ctypes.c_int]
    if hasattr(lib, "cxo_sort_range"):
        lib.cxo_prefix_counts.restype = ctypes.c_int64
        lib.cxo_prefix_counts.argtypes = [ctypes.c_char_p, u64p, u32p, ctypes.c_uint64, ctypes.c_int, u64p,
                                          ctypes.c_int]
        lib.cxo_sort_range.restype = ctypes.c_int64
        lib.cxo_sort_range.argtypes = [ctypes.c_char_p, u64p, u32p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_uint64, u64p, u32p, ctypes.c_char_p, ctypes.c_int]
    return lib


def load_library(path: str):
    """Load an oracle library built from ``cx_oracle.cpp`` at ``path`` (tests load
    deliberately broken copies this way to show that the pins catch them)."""
    return _bind(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Collection:
    """A read collection in the oracle's own form: ASCII bases + offsets + lengths."""

    def __init__(self, codes: np.ndarray, lens: np.ndarray):
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        self.lens = np.ascontiguousarray(lens, dtype=np.uint32)
        if codes.size != int(self.lens.sum(dtype=np.uint64)):
            raise ValueError("codes length does not match sum(lens)")
        if codes.size and int(codes.max()) > 3:
            raise ValueError("base codes must be 0..3")
        self.seq = np.frombuffer(ALPHABET, dtype=np.uint8)[codes].tobytes()
        self.off = np.zeros(self.lens.size, dtype=np.uint64)
        if self.lens.size > 1:
            np.cumsum(self.lens[:-1], dtype=np.uint64, out=self.off[1:])
        self.n = int(self.lens.size)
        self.n_suffixes = int(self.lens.sum(dtype=np.uint64)) + self.n

    @classmethod
    def from_strings(cls, reads):
        """Reads as Python strings over ACGT (tests and worked examples)."""
        table = {"A": 0, "C": 1, "G": 2, "T": 3}
        codes = np.array([table[c] for r in reads for c in r], dtype=np.uint8)
        lens = np.array([len(r) for r in reads], dtype=np.uint32)
        return cls(codes, lens)


def sort(col: Collection, threads: int = 1, lib=None):
    """Sorted suffix list and BWT.

    Returns ``(bwt, sa_read, sa_pos)``: ``bwt`` is an ASCII ``bytes`` of length
    N over ``$ACGT``; ``(sa_read[r], sa_pos[r])`` is the suffix of rank r.
    """
    lib = lib or _load()
    N = col.n_suffixes
    sa_read = np.empty(N, dtype=np.uint64)
    sa_pos = np.empty(N, dtype=np.uint32)
    out = ctypes.create_string_buffer(max(N, 1))
    got = lib.cxo_sort(col.seq, _ptr(col.off, ctypes.c_uint64), _ptr(col.lens, ctypes.c_uint32), col.n,
                       _ptr(sa_read, ctypes.c_uint64), _ptr(sa_pos, ctypes.c_uint32), out, int(threads))
    if got != N:
        raise RuntimeError(f"cxo_sort returned {got}, expected {N}")
    return out.raw[:N], sa_read, sa_pos


def bwt(col: Collection, threads: int = 1, lib=None):
    """The BWT and the quantities derived from it.

    Returns a dict with
      ``bwt``        ASCII bytes over ``$ACGT`` (length N),
      ``dollar_pos`` uint64[n]: row of the $ that precedes read i's whole suffix,
                     i.e. the rank of suffix (i, 0),
      ``counts``     uint64[5]: occurrences of $, A, C, G, T,
      ``sa_read``, ``sa_pos``: the sorted suffix list.
    """
    b, sa_read, sa_pos = sort(col, threads, lib)
    return {"bwt": b, "sa_read": sa_read, "sa_pos": sa_pos,
            "dollar_pos": dollar_positions(sa_read, sa_pos, col.n), "counts": counts(b)}


def dollar_positions(sa_read: np.ndarray, sa_pos: np.ndarray, n: int) -> np.ndarray:
    """For each read i, the rank of its whole suffix (i, 0): where its $ lands in B_R."""
    rows = np.nonzero(sa_pos == 0)[0]
    out = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
    out[sa_read[rows].astype(np.int64)] = rows.astype(np.uint64)
    return out


def counts(b: bytes) -> np.ndarray:
    """Occurrences of $, A, C, G, T in an ASCII BWT."""
    arr = np.frombuffer(b, dtype=np.uint8)
    return np.array([np.count_nonzero(arr == ord(c)) for c in "$ACGT"], dtype=np.uint64)


def rank(col: Collection, read: int, pos: int, threads: int = 0, lib=None) -> int:
    """Number of suffixes strictly smaller than suffix (read, pos): its row in the sorted list."""
    r = (lib or _load()).cxo_rank(col.seq, _ptr(col.off, ctypes.c_uint64), _ptr(col.lens, ctypes.c_uint32), col.n,
                         int(read), int(pos), int(threads))
    if r < 0:
        raise ValueError("bad suffix")
    return int(r)


def check_sa(col: Collection, sa_read: np.ndarray, sa_pos: np.ndarray, threads: int = 0, lib=None) -> int:
    """-1 if (sa_read, sa_pos) lists every suffix once in strictly increasing order,
    else the first failing rank (-2: wrong length)."""
    sa_read = np.ascontiguousarray(sa_read, dtype=np.uint64)
    sa_pos = np.ascontiguousarray(sa_pos, dtype=np.uint32)
    return int((lib or _load()).cxo_check_sa(col.seq, _ptr(col.off, ctypes.c_uint64), _ptr(col.lens, ctypes.c_uint32),
                                    col.n, _ptr(sa_read, ctypes.c_uint64), _ptr(sa_pos, ctypes.c_uint32),
                                    sa_read.size, int(threads)))


def prefix_counts(col: Collection, p: int, threads: int = 0, lib=None) -> np.ndarray:
    """Suffixes per bucket of their first p symbols over $ < A < C < G < T
    (5**p buckets, base 5, first symbol most significant; positions from the
    $ on read as $): the partition of Section 3.1."""
    out = np.zeros(5 ** p, dtype=np.uint64)
    got = (lib or _load()).cxo_prefix_counts(col.seq, _ptr(col.off, ctypes.c_uint64), _ptr(col.lens, ctypes.c_uint32),
                                             col.n, int(p), _ptr(out, ctypes.c_uint64), int(threads))
    if got != col.n_suffixes:
        raise RuntimeError(f"cxo_prefix_counts returned {got}, expected {col.n_suffixes}")
    return out


def sort_range(col: Collection, p: int, lo: int, hi: int, rows: int, threads: int = 1, lib=None):
    """The sorted suffixes of buckets [lo, hi) (``rows`` of them, from
    ``prefix_counts``): ``(bwt, sa_read, sa_pos)`` as ``sort`` returns them
    for those rows of the whole order."""
    sa_read = np.empty(rows, dtype=np.uint64)
    sa_pos = np.empty(rows, dtype=np.uint32)
    out = ctypes.create_string_buffer(max(rows, 1))
    got = (lib or _load()).cxo_sort_range(col.seq, _ptr(col.off, ctypes.c_uint64), _ptr(col.lens, ctypes.c_uint32),
                                          col.n, int(p), int(lo), int(hi), int(rows), _ptr(sa_read, ctypes.c_uint64),
                                          _ptr(sa_pos, ctypes.c_uint32), out, int(threads))
    if got != rows:
        raise RuntimeError(f"cxo_sort_range returned {got}, expected {rows}")
    return out.raw[:rows], sa_read, sa_pos


def sorted_ranges(col: Collection, p: int = 4, max_rows: int = 500_000_000, threads: int = 1, lib=None):
    """The whole sorted suffix list, one range of consecutive prefix buckets at
    a time (each of at most ``max_rows`` suffixes unless one bucket alone is
    larger): yields ``(row0, bwt, sa_read, sa_pos)`` with row0 the rank of
    the range's first suffix.  Concatenated, the ranges are ``sort``'s
    result."""
    counts = prefix_counts(col, p, threads, lib)
    row0 = 0
    b = 0
    nb = counts.size
    while b < nb:
        e, rows = b, 0
        while e < nb and (e == b or rows + int(counts[e]) <= max_rows):
            rows += int(counts[e])
            e += 1
        if rows:
            bwt_r, sr, sp = sort_range(col, p, b, e, rows, threads, lib)
            yield row0, bwt_r, sr, sp
        row0 += rows
        b = e
