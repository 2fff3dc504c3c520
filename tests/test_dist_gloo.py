"""The multi-rank path of the benchmark on the CPU: world size 2 over gloo.

The solve shards by node with no exchange, so what several ranks share is only
the timing protocol: a barrier on both sides of the timed steps, the slowest
rank's time, counts added over ranks, and inputs drawn from per-rank seeds.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2601_00976_gb300 import dist, synthetic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    g = dist.Group()   # gloo on the CPU
    assert (g.ws, g.rank) == (world, rank)
    g.barrier()
    slow = g.allmax(10.0 + rank)               # the slowest rank's time
    total = g.allsum(100 + rank)               # units over all ranks
    seed = dist.workload_seed(rank, 0)
    eps = np.linspace(1.0, 100.0, 8)
    inp = synthetic.make_inputs("profile", 4, eps, 2, seed=seed)
    first = g.allsum(int(inp["rho"][0] * 1e-3) % 1000003)   # fingerprints of the two workloads
    g.barrier()
    g.close()
    out.put((rank, slow, total, seed, int(inp["rho"][0] * 1e-3) % 1000003, first))


def test_two_gloo_ranks_share_only_the_timing_protocol():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, slow0, tot0, seed0, fp0, first0), (r1, slow1, tot1, seed1, fp1, first1) = res
    assert slow0 == slow1 == 11.0
    assert tot0 == tot1 == 201
    assert seed0 != seed1 and fp0 != fp1          # each rank draws its own nodes
    assert first0 == first1 == fp0 + fp1
    assert dist.weak_scaling_value(2 * 65536, 5, 1000.0) == pytest.approx(2 * 65536 * 5)


def test_single_rank_group_is_a_no_op(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    g = dist.Group()
    assert g.ws == 1 and g.allmax(3.5) == 3.5 and g.allsum(7) == 7
    g.barrier()
    g.close()
