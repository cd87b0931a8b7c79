"""The bench's multi-GPU path on CPU ranks (gloo, world size 2): each rank
builds its own independent collection (weak scaling, no data-path
collective); the whole-job throughput divides all ranks' bases by the
slowest rank's time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1401_7457_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # Ranks draw different collections of the same shape.
    _, codes, lens = bench.load_workload("tiny", rank, 200)
    local_ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    value, total = bench.aggregate(dist, local_ms, int(lens.sum()), world, 5)
    q.put((rank, value, total, int(codes[:64].sum())))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, v0, t0, s0), (_, v1, t1, s1) = out
    assert t0 == t1 == 200.0  # the slowest rank's time on every rank
    bases = 200 * 100
    assert v0 == v1 == pytest.approx(bases * 2 * 5 / 0.2 / 1e9)
    assert s0 != s1  # independent collections per rank
