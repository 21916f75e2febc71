"""The N > 1 layout on CPU with gloo (world size 2): shards cover the points exactly
once, the sharded adjoint plus one all-reduce equals the full adjoint, and the
sharded forward needs no exchange.  The per-shard transform here is the oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1809_10786_gb300 import distributed as sd
from paper_1809_10786_gb300 import inputs


def test_shards_partition_the_points():
    for M in (0, 1, 7, 1000, 1001):
        for W in (1, 2, 3, 8):
            seen = []
            for r in range(W):
                s, c = sd.shard(M, r, W)
                seen.extend(range(s, s + c))
            assert seen == list(range(M))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import direct
    B, M = 6, 301
    x = inputs.points_gaussian(M, 11)
    y = inputs.values(M, 12)
    c = inputs.coefficients(B, 13)

    def adj(xs, ys):
        a, _ = direct.adjoint(B, xs, ys, nthreads=1)
        return torch.from_numpy(a)

    coef = sd.sharded_adjoint(adj, x, y, rank, world)
    s, n = sd.shard(M, rank, world)
    f_part, _ = direct.forward(B, x[s:s + n], c, nthreads=1)
    tmax = sd.max_over_ranks(float(rank + 1))
    out[rank] = (coef.numpy().copy(), s, f_part, tmax)
    dist.destroy_process_group()


def test_sharded_adjoint_and_forward_with_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    from oracle import direct
    B, M = 6, 301
    x = inputs.points_gaussian(M, 11)
    y = inputs.values(M, 12)
    c = inputs.coefficients(B, 13)
    a_ref, _ = direct.adjoint(B, x, y)
    f_ref, _ = direct.forward(B, x, c)
    for r in range(world):
        coef, s, f_part, tmax = out[r]
        assert np.abs(coef - a_ref).max() <= 1e-12 * np.abs(a_ref).max()
        assert np.array_equal(f_part, f_ref[s:s + len(f_part)])
        assert tmax == float(world)
