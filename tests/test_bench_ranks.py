"""Host logic of the multi-GPU benchmark (independent replicas) on CPU:
two gloo ranks combine their figures -- evaluations are summed, times are
the slowest rank's -- without any GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    out = bench.combine_ranks(100 * (rank + 1), 10.0 + rank, 7 * (rank + 1), 3.0 - rank, ws, torch.device("cpu"))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_sum_units_and_take_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        evals, ms, e2e_evals, e2e_ms = res[r]
        assert evals == 300 and ms == 11.0 and e2e_evals == 21 and e2e_ms == 3.0


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5, 2.5, 3, 1.5, 1, None) == (5.0, 2.5, 3.0, 1.5)
