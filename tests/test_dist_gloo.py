"""The multi-process path of the benchmark on CPU, world size 2 over gloo: each rank solves its own
problems with the seed-counter offset of its shard and the job time is the slowest rank's. The
counter-based seeds make the sharded solve identical to one process solving all the problems;
the problems themselves are independent, so no collective touches the data path (the gather here
only brings the results to rank 0 for the check)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O
from paper_2607_11340_gb300 import synth

SPEC = synth.ROBOT_3SEG
P_PER_RANK = 5


def _cfg(p0):
    return O.IkConfig(S=16, n_final=2, k_init=8, k_final=6, seed=11, p0=p0)


def _problem():
    rb = O.make_robot(list(SPEC.L), SPEC.rc, SPEC.umax, nb=SPEC.nb)
    W = O.make_weights(**synth.WEIGHTS.as_dict())
    tg, _ = synth.ik_workload(SPEC, 2 * P_PER_RANK, "pose", lambda u: O.fk(rb, u)[0], seed=5)
    return rb, W, tg


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rb, W, tg = _problem()
        P = P_PER_RANK
        shard = tg[rank * P:(rank + 1) * P]
        r = O.solve_ik(rb, W, None, O.IK6, shard, _cfg(bench.shard_p0(rank, P)), threads=1)
        u = torch.as_tensor(r["u"])
        parts = [torch.zeros_like(u) for _ in range(world)]
        dist.all_gather(parts, u)
        t = bench.max_over_ranks(torch, dist, world, 10.0 + 7.5 * rank, "cpu")
        if rank == 0:
            q.put((torch.cat(parts).numpy(), t))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_solve_equals_one_process_and_max_time(orc):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        U, t = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    rb, W, tg = _problem()
    full = O.solve_ik(rb, W, None, O.IK6, tg, _cfg(0), threads=1)
    np.testing.assert_array_equal(U, full["u"])
    assert t == 17.5  # the slower rank's time
    assert bench.job_rate(world, P_PER_RANK, t) == world * P_PER_RANK / (t / 1e3)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(torch, None, 1, 12.5, "cpu") == 12.5
    assert bench.shard_p0(0, 4096) == 0 and bench.shard_p0(3, 4096) == 3 * 4096
