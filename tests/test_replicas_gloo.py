"""The multi-GPU form is independent replicas (one problem per rank, no data-path
collective); bench.py reports whole-job eigenpairs over the slowest rank's time.  The
reduction runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    found, ms = bench.reduce_over_ranks(105 - rank, 1000.0 + 250.0 * rank, world, device="cpu")
    out[rank] = (found, ms)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_sum_eigenpairs_and_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    assert out[0] == out[1] == (209, 1250.0)
    assert __import__("bench").reduce_over_ranks(7, 3.5, 1) == (7, 3.5)
