"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Each rank advances its own independent world (weak scaling; no collective
on the data path).  Checked here without a GPU: the ranks get distinct
worlds of identical shape, the timing reduction takes the slowest rank's
time and the sum of the ranks' agent-steps, and a second rank's world is an
ordinary world (its oracle step conserves the ledgers).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle

    class A:
        workload = "small"
        precision = None
        side = slots = founders = None

    envs = bench.make_workloads(A, rank)
    w = envs[0]
    o = oracle.Oracle(w)
    o.reset()
    agent_steps = 0
    for _ in range(3):
        _, st, _ = o.step_once()
        agent_steps += st["agent_steps"]
    # pretend per-rank device times that differ
    t = [10.0 + rank, 20.0 - rank]
    res = bench.reduce_over_ranks(dist, t, [agent_steps, 7])
    out.put((rank, w["seed"], w["side"], agent_steps, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    (r0, seed0, side0, as0, res0), (r1, seed1, side1, as1, res1) = got
    assert seed0 != seed1 and side0 == side1
    assert res0 == res1
    assert res0[0] == 11.0 and res0[1] == 20.0          # max over ranks
    assert res0[2] == as0 + as1 and res0[3] == 14        # sum over ranks
