"""ctypes binding of libcxbwt (include/cxbwt.h): argument marshalling only.

Every step of a build runs in the CUDA library; this module only turns numpy
arrays and torch tensors into pointers, allocates outputs when the caller
does not pass them, and raises ``CxbwtError`` on a negative status.  If the
library has not been built, importing the functions below raises: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcxbwt.so")

_lock = threading.Lock()
_lib = None

STATUS = {0: "CXBWT_OK", -1: "CXBWT_EINVAL", -2: "CXBWT_ENOMEM", -3: "CXBWT_ECUDA", -4: "CXBWT_ETIMEOUT",
          -5: "CXBWT_EUNSUPPORTED", -6: "CXBWT_EBUSY", -7: "CXBWT_EINTERNAL"}


class CxbwtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("device", ctypes.c_int), ("prefix_len", ctypes.c_int),
                ("digit_bits", ctypes.c_int), ("tile_items", ctypes.c_int), ("async_", ctypes.c_int),
                ("timing", ctypes.c_int), ("algorithm", ctypes.c_int), ("plan_flags", ctypes.c_int),
                ("batch_workers", ctypes.c_int), ("batch_small_mrows", ctypes.c_int), ("wait_limit_ms", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class Stats(ctypes.Structure):
    _fields_ = [("builds", ctypes.c_uint64), ("bases", ctypes.c_uint64), ("suffixes", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("sort_pass_launches", ctypes.c_uint64),
                ("sort_pass_items", ctypes.c_uint64), ("sort_pass_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("device_bytes_held", ctypes.c_uint64), ("group_ms", ctypes.c_double), ("emit_ms", ctypes.c_double),
                ("slices", ctypes.c_uint64), ("cta_groups", ctypes.c_uint64), ("big_groups", ctypes.c_uint64),
                ("carried_pass_launches", ctypes.c_uint64), ("carried_pass_items", ctypes.c_uint64),
                ("carried_pass_ms", ctypes.c_double), ("reserved", ctypes.c_uint64 * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


# Every entry point of include/cxbwt.h with its ctypes signature.
_VP, _U64, _U32P, _U64P = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p
SIGNATURES = {
    "cxbwt_abi_version": (ctypes.c_int, []),
    "cxbwt_default_options": (None, [ctypes.POINTER(Options)]),
    "cxbwt_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Options)]),
    "cxbwt_destroy": (None, [_VP]),
    "cxbwt_last_error": (ctypes.c_char_p, [_VP]),
    "cxbwt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cxbwt_output_size": (ctypes.c_int, [_U64, _VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "cxbwt_build": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP]),
    "cxbwt_build_sa": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP, _VP]),
    "cxbwt_sync": (ctypes.c_int, [_VP]),
    "cxbwt_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(Stats)]),
    "cxbwt_reset_stats": (ctypes.c_int, [_VP]),
    "cxbwt_pack_codes": (ctypes.c_int, [_VP, _U64, _VP]),
    "cxbwt_pack_ascii": (ctypes.c_int, [ctypes.c_char_p, _U64, _VP]),
    "cxbwt_unpack_ascii": (ctypes.c_int, [_VP, _VP, _U64, _U64, _VP]),
    "cxbwt_build_noalloc": (ctypes.c_int, [_VP, _U64, _VP, _VP, _VP, _VP, _VP]),
    "cxbwt_build_batch": (ctypes.c_int, [_VP, _VP, _U64, _VP]),
    "cxbwt_autotune": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP]),
    "cxbwt_bucket_counts": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "cxbwt_split_parts": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, _VP, _VP]),
    "cxbwt_build_part": (ctypes.c_int, [_VP, _VP, _U64, _VP, ctypes.c_uint32, ctypes.c_uint32, _VP, _VP, _VP, _VP,
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _VP]),
    "cxbwt_merge_part": (ctypes.c_int, [_VP, _U64, _VP, _U64, _U64]),
    "cxbwt_default_server_options": (None, [_VP]),
    "cxbwt_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _VP]),
    "cxbwt_server_destroy": (None, [_VP]),
    "cxbwt_submit": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    "cxbwt_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "cxbwt_wait": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "cxbwt_ticket_times": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "cxbwt_server_counters": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint64)]),
}


class Tuning(ctypes.Structure):
    _fields_ = [("tile_items", ctypes.c_int), ("algorithm", ctypes.c_int), ("digit_bits", ctypes.c_int),
                ("best_ms", ctypes.c_float), ("prefix_len", ctypes.c_int)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("device", ctypes.c_int), ("workers", ctypes.c_int),
                ("max_pack_suffixes", ctypes.c_uint64), ("reserved", ctypes.c_int * 8)]


class Request(ctypes.Structure):
    """cxbwt_request."""
    _fields_ = [("reads_2bit", ctypes.c_void_p), ("n_reads", ctypes.c_uint64), ("lens", ctypes.c_void_p),
                ("out_bwt", ctypes.c_void_p), ("out_dollar_pos", ctypes.c_void_p), ("out_counts", ctypes.c_void_p)]


class Server:
    """cxbwt_server: continuous batching of host-memory build requests."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, workers: int = 0, max_pack_suffixes: int = 0):
        L = lib()
        opt = ServerOptions()
        L.cxbwt_default_server_options(ctypes.byref(opt))
        opt.device = device
        opt.device_budget_bytes = budget_bytes
        if workers:
            opt.workers = workers
        opt.max_pack_suffixes = max_pack_suffixes
        h = ctypes.c_void_p()
        _check(L.cxbwt_server_create(ctypes.byref(h), ctypes.byref(opt)))
        self._h = h
        self._keep = {}

    def submit(self, reads_2bit, lens, out_bwt, out_dollar_pos=None, out_counts=None) -> int:
        """Queue a request (host arrays, kept alive here until it is done); returns its ticket."""
        _need(4, reads_2bit=reads_2bit, lens=lens, out_bwt=out_bwt)
        _need(8, out_dollar_pos=out_dollar_pos, out_counts=out_counts)
        lens_n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
        req = Request(_ptr(reads_2bit), lens_n, _ptr(lens), _ptr(out_bwt), _ptr(out_dollar_pos), _ptr(out_counts))
        t = ctypes.c_uint64()
        _check(lib().cxbwt_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (reads_2bit, lens, out_bwt, out_dollar_pos, out_counts)
        return t.value

    def poll(self, ticket: int) -> bool:
        done = ctypes.c_int()
        _check(lib().cxbwt_poll(self._h, ticket, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, ticket: int):
        _check(lib().cxbwt_wait(self._h, ticket))

    def times(self, ticket: int):
        """(queued_ms, latency_ms) of a finished request."""
        q, l = ctypes.c_double(), ctypes.c_double()
        _check(lib().cxbwt_ticket_times(self._h, ticket, ctypes.byref(q), ctypes.byref(l)))
        return q.value, l.value

    def counters(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().cxbwt_server_counters(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"completed": a.value, "packs": b.value, "bases": c.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().cxbwt_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Collection(ctypes.Structure):
    """cxbwt_collection."""
    _fields_ = [("reads_2bit", ctypes.c_void_p), ("n_reads", ctypes.c_uint64), ("lens", ctypes.c_void_p),
                ("out_bwt", ctypes.c_void_p), ("out_dollar_pos", ctypes.c_void_p), ("out_counts", ctypes.c_void_p)]

NOALLOC_MAX_SUFFIXES = 1 << 21
NOALLOC_MAX_READ_LEN = 272


def build_noalloc(reads_2bit, lens_host, out_bwt, out_dollar_pos, out_counts, stream=None):
    """cxbwt_build_noalloc: device reads and outputs (torch CUDA tensors),
    host lengths (numpy uint32).  Allocates nothing; raises CxbwtError on a
    negative status."""
    _need(4, reads_2bit=reads_2bit, out_bwt=out_bwt)
    _need(8, out_dollar_pos=out_dollar_pos, out_counts=out_counts)
    lens_host = np.ascontiguousarray(lens_host, dtype=np.uint32)
    st = lib().cxbwt_build_noalloc(_ptr(reads_2bit), lens_host.size, lens_host.ctypes.data, _ptr(out_bwt),
                                   _ptr(out_dollar_pos), _ptr(out_counts), _stream_ptr(stream))
    if st != 0:
        raise CxbwtError(st, "cxbwt_build_noalloc")


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libcxbwt is not built ({LIB_PATH} missing): run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _is_tensor(x):
    try:
        import torch
    except ImportError:
        return False
    return isinstance(x, torch.Tensor)


def _ptr(x):
    """Pointer of a numpy array or torch tensor (must be contiguous)."""
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"expected numpy array or torch tensor, got {type(x)}")


def _nbytes(x):
    return x.numel() * x.element_size() if _is_tensor(x) else x.nbytes


def _need(size: int, **arrays):
    """Raise TypeError unless every given array or tensor (None: skipped) has
    elements of `size` bytes: the library reads packed words and lengths as
    uint32 and writes $ rows, counts and suffix entries as uint64, so an
    int64 length array, say, would otherwise be read as other lengths."""
    for name, x in arrays.items():
        if x is None or not (_is_tensor(x) or isinstance(x, np.ndarray)):
            continue
        got = x.element_size() if _is_tensor(x) else x.itemsize
        if got != size:
            raise TypeError(f"{name} needs {size}-byte elements ({'uint32' if size == 4 else 'uint64'}), "
                            f"got {x.dtype}")


def _check(status: int, ctx=None):
    if status != 0:
        msg = lib().cxbwt_last_error(ctx)
        raise CxbwtError(status, msg.decode() if msg else "")


# ---- host helpers -----------------------------------------------------------

def pack_codes(codes: np.ndarray) -> np.ndarray:
    """Base codes (uint8, 0..3) -> packed 2-bit words (uint32, ABI layout)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.zeros((codes.size + 15) // 16, dtype=np.uint32)
    _check(lib().cxbwt_pack_codes(codes.ctypes.data, codes.size, out.ctypes.data))
    return out


def pack_ascii(s: str | bytes) -> np.ndarray:
    b = s.encode() if isinstance(s, str) else bytes(s)
    out = np.zeros((len(b) + 15) // 16, dtype=np.uint32)
    _check(lib().cxbwt_pack_ascii(b, len(b), out.ctypes.data))
    return out


def unpack_ascii(words, dollar_pos, n_symbols: int) -> bytes:
    """Packed BWT + $ rows -> ASCII bytes over $ACGT."""
    words = np.ascontiguousarray(_to_numpy(words).view(np.uint32))
    dp = np.ascontiguousarray(_to_numpy(dollar_pos).view(np.uint64))
    out = ctypes.create_string_buffer(max(int(n_symbols), 1))
    _check(lib().cxbwt_unpack_ascii(words.ctypes.data, dp.ctypes.data, int(n_symbols), dp.size, out))
    return out.raw[:int(n_symbols)]


def output_size(lens) -> tuple[int, int]:
    lens = np.ascontiguousarray(_to_numpy(lens).view(np.uint32))
    n_sym, words = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().cxbwt_output_size(lens.size, lens.ctypes.data, ctypes.byref(n_sym), ctypes.byref(words)))
    return int(n_sym.value), int(words.value)


BUCKETS = 65536  # 8-base buckets of the bucket-range parts


def split_parts(counts, n_parts: int) -> tuple[np.ndarray, np.ndarray]:
    """Bucket and row bounds (n_parts + 1 each) of n_parts ranges of about
    equal suffix counts (cxbwt_split_parts; host only)."""
    c = np.ascontiguousarray(_to_numpy(counts), dtype=np.uint64)
    bb = np.zeros(n_parts + 1, dtype=np.uint32)
    rb = np.zeros(n_parts + 1, dtype=np.uint64)
    _check(lib().cxbwt_split_parts(c.ctypes.data, c.size, n_parts, bb.ctypes.data, rb.ctypes.data))
    return bb, rb


def part_words(row0: int, rows: int) -> int:
    """Words of a part's output (rows [row0, row0 + rows))."""
    return (row0 % 16 + rows + 15) // 16 if rows else 0


def merge_part(bwt_words: np.ndarray, part: np.ndarray, row0: int, rows: int) -> None:
    """OR a part's words into a zero-initialised host B_R (cxbwt_merge_part)."""
    assert bwt_words.dtype == np.uint32 and bwt_words.flags.c_contiguous
    p = np.ascontiguousarray(_to_numpy(part)).view(np.uint32)
    _check(lib().cxbwt_merge_part(bwt_words.ctypes.data, bwt_words.size, p.ctypes.data if p.size else None,
                                  row0, rows))


def _to_numpy(x):
    if _is_tensor(x):
        return x.detach().cpu().numpy()
    return np.asarray(x)


# ---- context ----------------------------------------------------------------

class Context:
    """One cxbwt context (device workspace + bookkeeping) on one device."""

    ALGO_AUTO, ALGO_LSD, ALGO_GROUPS = 0, 1, 2
    PLAN_ID64, PLAN_READ_MAJOR, PLAN_TEST_STALL, PLAN_CARRY_BASE, PLAN_NO_PREFETCH = 1, 2, 4, 8, 16
    PLAN_DIGIT_LISTING = 32

    def __init__(self, device: int = 0, budget_bytes: int = 0, async_: bool = False, timing: bool = False,
                 tile_items: int = 0, algorithm: int = 0, plan_flags: int = 0, batch_workers: int = 0,
                 batch_small_mrows: int = 0, wait_limit_ms: int = 0, prefix_len: int = 0):
        L = lib()
        opt = Options()
        L.cxbwt_default_options(ctypes.byref(opt))
        opt.device = device
        opt.device_budget_bytes = budget_bytes
        opt.async_ = 1 if async_ else 0
        opt.timing = 1 if timing else 0
        opt.tile_items = tile_items
        opt.algorithm = algorithm
        opt.plan_flags = plan_flags
        opt.batch_workers = batch_workers
        opt.batch_small_mrows = batch_small_mrows
        opt.wait_limit_ms = wait_limit_ms
        opt.prefix_len = prefix_len
        h = ctypes.c_void_p()
        st = L.cxbwt_create(ctypes.byref(h), ctypes.byref(opt))
        if st != 0:
            raise CxbwtError(st, (L.cxbwt_last_error(None) or b"").decode())
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().cxbwt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def build(self, reads_2bit, lens, out_bwt=None, out_dollar_pos=None, out_counts=None, out_sa=None,
              stream=None, want_sa: bool = False):
        """Build the BWT.  Inputs may be numpy arrays (host) or torch tensors
        (host or CUDA); missing outputs are allocated on the inputs' side.
        Returns ``(bwt_words, dollar_pos, counts[, sa])``."""
        n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
        on_dev = _is_tensor(reads_2bit) and reads_2bit.is_cuda
        if out_bwt is None or out_dollar_pos is None or out_counts is None or (want_sa and out_sa is None):
            if _is_tensor(lens) and lens.is_cuda:
                total = int(lens.to(dtype=_torch().int64).sum().item()) + n
            else:
                total = int(np.asarray(_to_numpy(lens), dtype=np.uint64).sum()) + n
            words = (total + 15) // 16
            if on_dev:
                torch = _torch()
                dev = reads_2bit.device
                if out_bwt is None:
                    out_bwt = torch.empty(words, dtype=torch.int32, device=dev)
                if out_dollar_pos is None:
                    out_dollar_pos = torch.empty(n, dtype=torch.int64, device=dev)
                if out_counts is None:
                    out_counts = torch.zeros(5, dtype=torch.int64, device=dev)
                if want_sa and out_sa is None:
                    out_sa = torch.empty(total, dtype=torch.int64, device=dev)
            else:
                if out_bwt is None:
                    out_bwt = np.zeros(words, dtype=np.uint32)
                if out_dollar_pos is None:
                    out_dollar_pos = np.zeros(n, dtype=np.uint64)
                if out_counts is None:
                    out_counts = np.zeros(5, dtype=np.uint64)
                if want_sa and out_sa is None:
                    out_sa = np.zeros(total, dtype=np.uint64)
        _need(4, reads_2bit=reads_2bit, lens=lens, out_bwt=out_bwt)
        _need(8, out_dollar_pos=out_dollar_pos, out_counts=out_counts, out_sa=out_sa)
        st = _stream_ptr(stream)
        L = lib()
        if want_sa or out_sa is not None:
            status = L.cxbwt_build_sa(self._h, _ptr(reads_2bit), n, _ptr(lens), _ptr(out_bwt), _ptr(out_dollar_pos),
                                      _ptr(out_counts), _ptr(out_sa), st)
            _check(status, self._h)
            return out_bwt, out_dollar_pos, out_counts, out_sa
        status = L.cxbwt_build(self._h, _ptr(reads_2bit), n, _ptr(lens), _ptr(out_bwt), _ptr(out_dollar_pos),
                               _ptr(out_counts), st)
        _check(status, self._h)
        return out_bwt, out_dollar_pos, out_counts

    def bucket_counts(self, reads_2bit, lens, stream=None) -> np.ndarray:
        """Suffixes per 8-base bucket (BUCKETS entries; reads of one length)."""
        _need(4, reads_2bit=reads_2bit, lens=lens)
        n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
        out = np.zeros(BUCKETS, dtype=np.uint64)
        _check(lib().cxbwt_bucket_counts(self._h, _ptr(reads_2bit), n, _ptr(lens), out.ctypes.data,
                                         _stream_ptr(stream)), self._h)
        return out

    def build_part(self, reads_2bit, lens, bucket_lo: int, bucket_hi: int, row0: int, rows: int,
                   out_words=None, out_dollar_pos=None, out_counts=None, stream=None, bucket_counts=None):
        """Build the part of B_R of buckets [bucket_lo, bucket_hi), whose rows
        are [row0, row0 + rows) (from bucket_counts / split_parts; passing
        those counts spares the device a count of every suffix).  Missing
        outputs are allocated on the inputs' side.  Returns
        ``(words, dollar_pos, counts)``."""
        bc = None
        if bucket_counts is not None:
            bc = np.ascontiguousarray(_to_numpy(bucket_counts), dtype=np.uint64)
            if bc.size != BUCKETS:
                raise ValueError(f"bucket_counts needs {BUCKETS} entries")
        n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
        nw = max(part_words(row0, rows), 1)
        if _is_tensor(reads_2bit) and reads_2bit.is_cuda:
            torch = _torch()
            dev = reads_2bit.device
            if out_words is None:
                out_words = torch.empty(nw, dtype=torch.int32, device=dev)
            if out_dollar_pos is None:
                out_dollar_pos = torch.empty(n, dtype=torch.int64, device=dev)
            if out_counts is None:
                out_counts = torch.zeros(5, dtype=torch.int64, device=dev)
        else:
            if out_words is None:
                out_words = np.zeros(nw, dtype=np.uint32)
            if out_dollar_pos is None:
                out_dollar_pos = np.zeros(n, dtype=np.uint64)
            if out_counts is None:
                out_counts = np.zeros(5, dtype=np.uint64)
        _need(4, reads_2bit=reads_2bit, lens=lens, out_words=out_words)
        _need(8, out_dollar_pos=out_dollar_pos, out_counts=out_counts)
        if _nbytes(out_words) < 4 * part_words(row0, rows):
            raise ValueError("out_words holds fewer words than the part needs")
        r0, nr = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().cxbwt_build_part(self._h, _ptr(reads_2bit), n, _ptr(lens), bucket_lo, bucket_hi,
                                      None if bc is None else bc.ctypes.data,
                                      _ptr(out_words), _ptr(out_dollar_pos), _ptr(out_counts), ctypes.byref(r0),
                                      ctypes.byref(nr), _stream_ptr(stream)), self._h)
        if (int(r0.value), int(nr.value)) != (row0, rows):
            raise CxbwtError(-7, f"part rows [{r0.value}, +{nr.value}) differ from the plan's [{row0}, +{rows})")
        return out_words, out_dollar_pos, out_counts

    def build_batch(self, collections, stream=None):
        """collections: list of (reads_2bit, lens, out_bwt, out_dollar_pos, out_counts) arrays/tensors
        (outputs required).  Builds every BWT; returns nothing (outputs are filled)."""
        arr = (Collection * len(collections))()
        keep = []
        for i, (words, lens, bwt, dpos, cnt) in enumerate(collections):
            _need(4, reads_2bit=words, lens=lens, out_bwt=bwt)
            _need(8, out_dollar_pos=dpos, out_counts=cnt)
            n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
            arr[i] = Collection(_ptr(words), n, _ptr(lens), _ptr(bwt), _ptr(dpos), _ptr(cnt))
            keep.append((words, lens, bwt, dpos, cnt))
        _check(lib().cxbwt_build_batch(self._h, ctypes.cast(arr, ctypes.c_void_p), len(collections),
                                       _stream_ptr(stream)), self._h)

    def autotune(self, reads_2bit, lens, scratch_bwt, scratch_dollar_pos=None, stream=None) -> dict:
        """Time the candidate plans on this collection; later builds of its size class use the fastest."""
        _need(4, reads_2bit=reads_2bit, lens=lens, scratch_bwt=scratch_bwt)
        _need(8, scratch_dollar_pos=scratch_dollar_pos)
        n = int(lens.numel() if _is_tensor(lens) else np.asarray(lens).size)
        t = Tuning()
        _check(lib().cxbwt_autotune(self._h, _ptr(reads_2bit), n, _ptr(lens), _ptr(scratch_bwt),
                                    _ptr(scratch_dollar_pos), _stream_ptr(stream), ctypes.byref(t)), self._h)
        return {"tile_items": t.tile_items, "algorithm": t.algorithm, "digit_bits": t.digit_bits,
                "best_ms": t.best_ms, "prefix_len": t.prefix_len}

    def sync(self):
        _check(lib().cxbwt_sync(self._h), self._h)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().cxbwt_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def reset_stats(self):
        _check(lib().cxbwt_reset_stats(self._h), self._h)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def decode_sa(sa) -> tuple[np.ndarray, np.ndarray]:
    """(i << 16) | k entries -> (read, offset) arrays."""
    a = _to_numpy(sa).view(np.uint64)
    return a >> np.uint64(16), (a & np.uint64(0xFFFF)).astype(np.uint32)
