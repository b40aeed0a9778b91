"""Pole sharding (the paper's first parallel level, Sec. 2.3): each rank filters with its
share of the pole table (slrf.pole_shard) and one sum all-reduce of the partial blocks
gives the filtered block of the whole table.  Two gloo ranks on the CPU run the FP64
oracle's filter apply on their shares, zero-guess and warm-started (the warm start
Y_j = x/(theta - sigma_j) + correction splits by pole too); the reduced block equals the
single-rank block to rounding, and the shards partition the poles."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    sys.path.insert(0, ROOT)
    import slrf_inputs as si
    from oracle import slrf_oracle as orc

    p = si.q1_scalar((6, 5, 4), shift=1e-3)
    gamma = 120.0
    sig, w = orc.slrf_poles(8, gamma)
    V = si.start_block(p.n, 6, 3)
    theta = np.linspace(0.1, 1.2, 6) * gamma
    return p, gamma, sig, w, V, theta


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from oracle import slrf_oracle as orc
    from paper_2510_17334_gb300.slrf import pole_shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, gamma, sig, w, V, theta = _case()
    mine = pole_shard(len(sig), world, rank)
    res = []
    for th in (None, theta):
        U, _ = orc.filter_apply(p.A(), p.B(), V, th, sig[mine], w[mine], 30, 1e-12)
        t = torch.from_numpy(U)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        res.append(t.numpy().copy())
    out[rank] = (mine, res)
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_pole_sharded_filter_equals_the_single_rank_filter():
    sys.path.insert(0, ROOT)
    from oracle import slrf_oracle as orc
    from paper_2510_17334_gb300.slrf import pole_shard

    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(150)
        assert q.exitcode == 0
    assert sorted(out[0][0] + out[1][0]) == list(range(8))
    p, gamma, sig, w, V, theta = _case()
    for i, th in enumerate((None, theta)):
        Uref, _ = orc.filter_apply(p.A(), p.B(), V, th, sig, w, 30, 1e-12)
        for r in range(2):
            assert np.abs(out[r][1][i] - Uref).max() <= 1e-12 * np.abs(Uref).max()
    for world in (1, 3, 8, 11):
        parts = [pole_shard(8, world, r) for r in range(world)]
        assert sorted(sum(parts, [])) == list(range(8))
