"""The multi-process path of the benchmark on CPU, world size 2 over gloo: each rank solves its own
problems with the seed-counter offset of its shard and the job time is the slowest rank's. The
counter-based seeds make the sharded solve identical to one process solving all the problems;
the problems themselves are independent, so no collective touches the data path (the gather here
only brings the results to rank 0 for the check)."""
import os
import socket

import numpy as np
import pytest
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


# ---- the ragged batch split over processes by estimated cost ----

def _ragged_case():
    """A small ragged batch (IK items and short paths of 1-3 segments, few seeds) with its targets and
    spheres, item-packed as the batch takes them."""
    rng = np.random.default_rng(44)
    N = 10
    items = np.zeros((N, 5), dtype=np.int64)
    items[:, 0] = rng.integers(0, 2, N)
    items[:, 1] = rng.integers(1, 4, N)
    items[:, 2] = np.where(items[:, 0] == 1, rng.integers(2, 5, N), 1)
    items[:, 3] = rng.integers(8, 17, N)
    items[:, 4] = rng.integers(0, 3, N)
    fam = synth.ROBOT_FAMILY

    def fkb(n, U):
        rb = O.make_robot(list(fam.L[:n]), fam.rc, fam.umax, nb=fam.nb)
        return O.fk(rb, U, backbone=True)

    items, targets, spheres, _ = synth.ragged_workload(N, fkb, seed=44, items=items)
    return fam, items, targets, spheres


def _solve_items(fam, items, targets, spheres, lo, hi, p0):
    """The oracle's solve of items [lo, hi) (IK: Algorithm 1; path: the path pipeline), item i drawing
    its seeds as problem p0 + (i - lo): a list of (u, success) per item."""
    ik = synth.IkSpec(S=16, n_final=2, k_init=6, k_final=6)
    w0 = np.concatenate([[0], np.cumsum(items[:, 2])])
    o0 = np.concatenate([[0], np.cumsum(items[:, 4])])
    W = O.make_weights(**synth.WEIGHTS.as_dict())
    out = []
    for i in range(lo, hi):
        kind, n, H, S, no = (int(v) for v in items[i])
        rb = O.make_robot(list(fam.L[:n]), fam.rc, fam.umax, nb=fam.nb)
        tg = targets[w0[i]:w0[i] + H]
        sp = spheres[o0[i]:o0[i] + no] if no else None
        cfg = O.IkConfig(S=S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, seed=3, p0=p0 + (i - lo))
        if kind == 1:
            o = O.solve_path(rb, W, None if sp is None else sp[None], tg[None], cfg, 3, 3, threads=1)
            out.append((o["x"][0], bool(o["lim_ok"][0] and o["col_ok"][0])))
        else:
            o = O.solve_ik(rb, W, sp, O.IK6, tg, cfg, threads=1)
            out.append((o["u"][0], bool(o["success"][0])))
    return out


def _partition(items, parts):
    from paper_2607_11340_gb300 import lib

    prm = lib.cr_batch_params()
    prm.ik.n_final, prm.ik.k_init, prm.ik.k_final = 2, 6, 6
    prm.k_warm, prm.k_joint = 3, 3
    return lib.cr_batch_partition(lib._batch_items(items), prm, parts)


def _ragged_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        fam, items, targets, spheres = _ragged_case()
        b = _partition(items, world)
        mine = _solve_items(fam, items, targets, spheres, b[rank], b[rank + 1], p0=b[rank])
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        if rank == 0:
            q.put((b, [r for p in parts for r in p]))
    finally:
        dist.destroy_process_group()


def test_ragged_partition_by_cost_equals_one_process():
    """Two gloo processes each take their contiguous, cost-balanced range of a ragged batch (the
    library's partitioner), solve it with the range start as their seed-counter offset and gather:
    every item's result equals the one-process solve of the whole batch."""
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ragged_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        b, got = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    fam, items, targets, spheres = _ragged_case()
    assert b[0] == 0 and b[-1] == len(items) and all(x <= y for x, y in zip(b, b[1:]))
    assert 0 < b[1] < len(items)  # both processes get work
    full = _solve_items(fam, items, targets, spheres, 0, len(items), p0=0)
    assert len(got) == len(full)
    for (u1, s1), (u2, s2) in zip(got, full):
        np.testing.assert_array_equal(u1, u2)
        assert s1 == s2


def test_partition_bounds():
    """The partitioner's bounds: equal items split evenly; one item far costlier than the rest gets
    (nearly) a part of its own; parts = 1 takes everything; bad input is refused."""
    from paper_2607_11340_gb300 import build_lib, lib

    build_lib.build()
    ik_item = [0, 3, 1, 64, 0]
    assert _partition(np.array([ik_item] * 12), 4) == [0, 3, 6, 9, 12]
    assert _partition(np.array([ik_item] * 12), 1) == [0, 12]
    heavy = [1, 6, 128, 256, 64]
    b = _partition(np.array([heavy] + [ik_item] * 11), 2)
    assert b[1] <= 1  # the path of 128 waypoints outweighs the 11 IK items
    with pytest.raises(lib.CrError):
        _partition(np.array([[0, 3, 2, 64, 0]]), 2)  # an IK item with H = 2


# ---- calibration with the poses spread over processes ----

def _calib_case():
    spec = synth.ROBOT_3SEG

    def fkp(U, L, rc):
        return O.fk(O.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    U, Pm, true, nom = synth.calib_workload(spec, 96, fkp, seed=8)
    rb = O.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    return spec, rb, U, Pm, nom


class _OracleCalibShard:
    """The four pieces of a sharded calibration iteration on the host for one share of the poses: the
    sums from the oracle's residual and complex-step Jacobian; the trial step and the rule as the LM
    rule states them (Marquardt damping of the diagonal, Cholesky, gain ratio, Nielsen update) on the
    all-reduced sums. Stands in for the library's cr_calib_* calls where there is no GPU."""

    def __init__(self, rb, U, Pm):
        self.rb, self.U, self.Pm = rb, U, Pm

    def sums(self, theta):
        th = theta.numpy()
        r = O.calib_residual(self.rb, self.U, self.Pm, th)
        J = O.calib_jacobian(self.rb, self.U, self.Pm, th)
        A = J.T @ J
        tri = [A[i, j] for i in range(len(th)) for j in range(i + 1)]
        return torch.tensor(tri + list(J.T @ r) + [0.5 * r @ r], dtype=torch.float64)

    def _unpack(self, sums, nx):
        A = np.zeros((nx, nx))
        k = 0
        for i in range(nx):
            for j in range(i + 1):
                A[i, j] = A[j, i] = sums[k]
                k += 1
        return A, sums[k:k + nx].numpy().copy(), float(sums[k + nx])

    def trial(self, sums, theta, state):
        nx = theta.numel()
        A, g, _ = self._unpack(sums, nx)
        D = np.maximum(np.diag(A), 1e-12)
        lam = float(state[0])
        try:
            Lc = np.linalg.cholesky(A + lam * np.diag(D))
            dl = -np.linalg.solve(Lc.T, np.linalg.solve(Lc, g))
            state[2], state[3] = 1.0, 0.5 * dl @ (lam * D * dl - g)
        except np.linalg.LinAlgError:
            dl = np.zeros(nx)
            state[2], state[3] = 0.0, 0.0
        return theta + torch.as_tensor(dl)

    def cost(self, theta_trial):
        r = O.calib_residual(self.rb, self.U, self.Pm, theta_trial.numpy())
        return torch.tensor([0.5 * r @ r], dtype=torch.float64)

    def accept(self, sums, F_trial, theta_trial, theta, state):
        F = float(sums[-1])
        lam, nu = float(state[0]), float(state[1])
        if state[2] != 0 and float(F_trial[0]) < F:
            t = 2.0 * (F - float(F_trial[0])) / float(state[3]) - 1.0
            lam *= max(1.0 / 3.0, 1.0 - t ** 3)
            nu = 2.0
            theta.copy_(theta_trial)
        else:
            lam *= nu
            nu *= 2.0
        state[0], state[1] = lam, nu


def _calib_worker(rank, world, port, q):
    from paper_2607_11340_gb300 import api

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec, rb, U, Pm, nom = _calib_case()
        K = len(U)
        lo, hi = rank * K // world, (rank + 1) * K // world
        theta = torch.tensor(nom, dtype=torch.float64)
        state = torch.tensor([1e-3, 2.0, 0.0, 0.0], dtype=torch.float64)
        api.calibrate_lm_sharded(_OracleCalibShard(rb, U[lo:hi], Pm[lo:hi]), theta, state, 12,
                                 lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM))
        got = [None] * world
        dist.all_gather_object(got, theta.numpy())
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


def test_sharded_calibration_equals_one_process():
    """Two gloo processes, each with half of the poses, run the sharded LM (partial normal equations
    and partial trial costs all-reduced between the pieces): both end with the same parameters, and
    they equal the oracle's one-process calibration of all the poses (to the rounding of the
    different summation order)."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_calib_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    np.testing.assert_array_equal(got[0], got[1])
    spec, rb, U, Pm, nom = _calib_case()
    ref = O.calibrate(rb, U, Pm, nom, 12)
    np.testing.assert_allclose(got[0], ref["theta"], rtol=1e-10)
    assert np.abs(ref["theta"] - nom).max() > 1e-4  # the calibration moved the parameters
