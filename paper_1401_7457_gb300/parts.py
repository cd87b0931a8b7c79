"""Bucket-range parts of one BWT build.

Section 3.3 of the paper splits the suffixes by their l-prefix into bucket
ranges holding about equal numbers of suffixes and sorts each range on its own
node; Section 3.1 sorts such ranges one after another when memory is bounded
("rounds"), writing each range's piece of B_R out before the next.  Both rest
on one fact: every suffix of a lower bucket sorts before every suffix of a
higher one, so B_R is the concatenation of the ranges' pieces in bucket order.

Here a bucket is the first 8 bases of a suffix (A-padded past the read end)
and a part is a range of whole buckets, built on the device by
``cxbwt_build_part``.  This module adds the host side:

* ``build_sharded``: one part per rank of a ``torch.distributed`` group.  Each
  rank computes the bucket counts itself (no exchange needed for the plan),
  builds its part, and the parts are gathered to rank 0 and merged: the only
  exchange is that ordered gather, as tensors (the symbol counts add, the
  ``$`` rows merge by element-wise minimum, the packed words by OR).
* ``build_rounds``: the parts one after another into files (the packed B_R
  and the ``$`` rows, as memory maps, so host memory holds one part at a
  time), with a checkpoint after every part: an interrupted build resumes at
  the first part not yet written.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass

import numpy as np

from . import binding

NO_ROW = np.uint64(0xFFFFFFFFFFFFFFFF)  # $ row of a read whose $ lies in another part


@dataclass(frozen=True)
class Part:
    lo: int      # first bucket
    hi: int      # one past the last bucket
    row0: int    # first global row of B_R
    rows: int    # rows of the part


def plan_parts(bucket_counts, n_parts: int) -> list[Part]:
    """n_parts consecutive bucket ranges of about equal suffix counts."""
    bb, rb = binding.split_parts(bucket_counts, n_parts)
    return [Part(int(bb[j]), int(bb[j + 1]), int(rb[j]), int(rb[j + 1] - rb[j])) for j in range(n_parts)]


def empty_result(n_symbols: int, n_reads: int):
    """Zeroed B_R words, unset $ rows and zero counts, ready for merge_into."""
    return (np.zeros((n_symbols + 15) // 16, dtype=np.uint32), np.full(n_reads, NO_ROW, dtype=np.uint64),
            np.zeros(5, dtype=np.uint64))


def merge_into(result, part: Part, words, dollar_pos, counts) -> None:
    """Merge one part's outputs (host arrays) into a full result."""
    bwt, dpos, cnt = result
    if part.rows:
        binding.merge_part(bwt, np.asarray(words), part.row0, part.rows)
    d = np.asarray(dollar_pos).view(np.uint64)
    np.minimum(dpos, d, out=dpos)
    cnt += np.asarray(counts).view(np.uint64)


def _host(x):
    return binding._to_numpy(x)


def build_part_host(ctx, reads_2bit, lens, part: Part, stream=None, bucket_counts=None):
    """Build one part; its outputs come back as host arrays.  bucket_counts
    (the collection's, when the caller has them) spares the device a count."""
    if part.rows == 0:
        n = int(lens.numel() if binding._is_tensor(lens) else np.asarray(lens).size)
        return np.zeros(0, dtype=np.uint32), np.full(n, NO_ROW, dtype=np.uint64), np.zeros(5, dtype=np.uint64)
    w, d, c = ctx.build_part(reads_2bit, lens, part.lo, part.hi, part.row0, part.rows, stream=stream,
                             bucket_counts=bucket_counts)
    return (_host(w).view(np.uint32)[: binding.part_words(part.row0, part.rows)], _host(d).view(np.uint64),
            _host(c).view(np.uint64))


def gather_parts(local, part: Part, n_symbols: int, n_reads: int, plan=None, group=None):
    """Gather every rank's part outputs (words, dollar_pos, counts) to rank 0
    and merge them there; returns the full (bwt, dollar_pos, counts) on rank 0,
    None on the other ranks.  This is the only exchange of a sharded build,
    and it moves tensors (on the GPU under NCCL, on the host under gloo):

    * the $ rows by an element-wise MIN reduction (a read's row is set in the
      one part that holds it; the others hold no row, sent as the largest
      int64),
    * the symbol counts by a SUM reduction,
    * each part's packed words by a send to rank 0, whose sizes rank 0 knows
      from the plan (``plan``: every rank's Part, as ``plan_parts`` gives it;
      without it the sizes are exchanged first).
    """
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    dst = dist.get_global_rank(group, 0) if group is not None else 0
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    words, dollar_pos, counts = local
    d = np.asarray(dollar_pos).view(np.uint64).copy()
    big = np.uint64(np.iinfo(np.int64).max)
    d[d == NO_ROW] = big
    dt = torch.from_numpy(d.view(np.int64)).to(dev)
    dist.reduce(dt, dst=dst, op=dist.ReduceOp.MIN, group=group)
    ct = torch.from_numpy(np.asarray(counts).view(np.uint64).astype(np.int64)).to(dev)
    dist.reduce(ct, dst=dst, op=dist.ReduceOp.SUM, group=group)
    if plan is None:
        # Every rank's (row0, rows), so that rank 0 can size its receives.
        mine = torch.tensor([part.lo, part.hi, part.row0, part.rows], dtype=torch.int64, device=dev)
        allp = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(allp, mine, group=group)
        plan = [Part(*(int(x) for x in t.cpu().tolist())) for t in allp]
    if rank != 0:
        if part.rows:
            w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32)[: binding.part_words(part.row0, part.rows)])
            dist.send(torch.from_numpy(w.view(np.int32)).to(dev), dst=dst, group=group)
        return None
    result = empty_result(n_symbols, n_reads)
    bwt = result[0]
    if part.rows:
        binding.merge_part(bwt, np.asarray(words, dtype=np.uint32), part.row0, part.rows)
    for r in range(1, world):
        p = plan[r]
        if not p.rows:
            continue
        buf = torch.empty(binding.part_words(p.row0, p.rows), dtype=torch.int32, device=dev)
        src = dist.get_global_rank(group, r) if group is not None else r
        dist.recv(buf, src=src, group=group)
        binding.merge_part(bwt, buf.cpu().numpy().view(np.uint32), p.row0, p.rows)
    dm = dt.cpu().numpy().view(np.uint64).copy()
    dm[dm == big] = NO_ROW
    result[1][:] = dm
    result[2][:] = ct.cpu().numpy().astype(np.uint64)
    return result


def build_sharded(ctx, reads_2bit, lens, group=None, stream=None):
    """One part per rank of `group` (default: the whole world).  Every rank
    returns; rank 0 gets the full (bwt, dollar_pos, counts), the others None."""
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    counts = ctx.bucket_counts(reads_2bit, lens, stream=stream)
    parts = plan_parts(counts, world)
    n_symbols = int(counts.sum())
    n_reads = int(lens.numel() if binding._is_tensor(lens) else np.asarray(lens).size)
    local = build_part_host(ctx, reads_2bit, lens, parts[rank], stream=stream, bucket_counts=counts)
    return gather_parts(local, parts[rank], n_symbols, n_reads, plan=parts, group=group)


def _fingerprint(bucket_counts, n_reads: int, n_rounds: int) -> str:
    h = hashlib.blake2b(digest_size=16)
    h.update(np.ascontiguousarray(bucket_counts, dtype=np.uint64).tobytes())
    h.update(np.array([n_reads, n_rounds], dtype=np.uint64).tobytes())
    return h.hexdigest()


def rounds_for_host_budget(n_symbols: int, host_bytes: int) -> int:
    """Rounds whose parts' packed words (a quarter byte per row) fit host_bytes."""
    per_round = max(host_bytes, 64) * 4  # rows per round
    return max(1, -(-n_symbols // per_round))


def build_rounds(ctx, reads_2bit, lens, n_rounds: int, out_dir: str, stop_after: int | None = None,
                 builder=None, bucket_counts=None) -> dict:
    """Build B_R in n_rounds parts, one after another, into out_dir:

    * ``bwt.u32``: the packed words of B_R (as cxbwt_build's out_bwt),
    * ``dollar.u64``: the $ row of every read (as out_dollar_pos),
    * ``state.json``: the checkpoint: the plan's fingerprint, the next part
      to build and the symbol counts so far.

    Each part is merged into the memory-mapped files and flushed before the
    checkpoint names the next part, so a build stopped at any point (here:
    ``stop_after`` parts, for tests) resumes at the first unwritten part when
    called again with the same collection and n_rounds.  ``builder(part)``
    (default: build_part_host on ctx) and ``bucket_counts`` (default: the
    device's) are the two steps that touch the device.  Returns the state."""
    n_reads = int(lens.numel() if binding._is_tensor(lens) else np.asarray(lens).size)
    if bucket_counts is None:
        bucket_counts = ctx.bucket_counts(reads_2bit, lens)
    bucket_counts = np.asarray(bucket_counts, dtype=np.uint64)
    if builder is None:
        def builder(p):
            return build_part_host(ctx, reads_2bit, lens, p, bucket_counts=bucket_counts)
    parts = plan_parts(bucket_counts, n_rounds)
    n_symbols = int(bucket_counts.sum())
    n_words = (n_symbols + 15) // 16
    fp = _fingerprint(bucket_counts, n_reads, n_rounds)
    os.makedirs(out_dir, exist_ok=True)
    state_path = os.path.join(out_dir, "state.json")
    bwt_path = os.path.join(out_dir, "bwt.u32")
    dollar_path = os.path.join(out_dir, "dollar.u64")
    state = None
    if os.path.exists(state_path):
        with open(state_path) as f:
            state = json.load(f)
        if state.get("fingerprint") != fp:
            raise ValueError(f"{state_path} belongs to another collection or round count")
    if state is None:
        with open(bwt_path, "wb") as f:
            f.truncate(n_words * 4)
        np.full(n_reads, NO_ROW, dtype=np.uint64).tofile(dollar_path)
        state = {"fingerprint": fp, "n_rounds": n_rounds, "n_symbols": n_symbols, "n_reads": n_reads,
                 "next": 0, "counts": [0] * 5, "done": False}
        _write_state(state_path, state)
    bwt = np.memmap(bwt_path, dtype=np.uint32, mode="r+", shape=(n_words,))
    dpos = np.memmap(dollar_path, dtype=np.uint64, mode="r+", shape=(n_reads,))
    built = 0
    try:
        while state["next"] < n_rounds:
            if stop_after is not None and built >= stop_after:
                break
            j = state["next"]
            p = parts[j]
            words, dollar_pos, counts = builder(p)
            if p.rows:
                w0 = p.row0 // 16
                nw = binding.part_words(p.row0, p.rows)
                region = np.array(bwt[w0:w0 + nw])
                region |= np.asarray(words, dtype=np.uint32)[:nw]
                bwt[w0:w0 + nw] = region
            d = np.asarray(dollar_pos).view(np.uint64)
            mine = d != NO_ROW
            dpos[mine] = d[mine]
            bwt.flush()
            dpos.flush()
            state["counts"] = [int(a) + int(b) for a, b in zip(state["counts"], np.asarray(counts).view(np.uint64))]
            state["next"] = j + 1
            state["done"] = state["next"] == n_rounds
            _write_state(state_path, state)
            built += 1
    finally:
        del bwt, dpos
    return state


def _write_state(path: str, state: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(state, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)
