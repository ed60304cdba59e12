"""The multi-process path of bench.py on CPU (gloo, two ranks): whole-job units are summed
over the ranks and the timed seconds are the slowest rank's, as the GPU run does over
NCCL.  Each rank owns independent RVEs, so this reduction is the only collective."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [0.5, 2.0][rank]
    units = [16, 15][rank]          # rank 1 had one failed increment
    applies = [10000, 9000][rank]
    t, u, a = bench.combine_ranks(torch, dist, t_local, units, applies, "cpu")
    q.put((rank, t, u, a))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_combine_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, a in res:
        assert t == 2.0 and u == 31 and a == 19000


def test_combine_ranks_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(torch, None, 1.5, 16, 700, "cpu") == (1.5, 16, 700)
