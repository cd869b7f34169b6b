"""Success-rate parity with the FP64 oracle, on samples large enough to resolve one percentage point.

Every config's GPU solver (the FP32-bulk optimised form, and the FP64 form where the config has one)
and the oracle solve the same problems with the same seed counters and settings; success is
<= 1 mm and <= 1 degree (every waypoint for paths, the goal for trajectories), limits and
clearance, each side judged by its own FP64 acceptance. The assertion is |rate_gpu - rate_oracle|
<= 0.01, with the sample size stated per test; each test prints both rates and the per-problem
flag mismatches. Where a config's full shape is too slow for the oracle (paths of 64 waypoints,
trajectories of 32 states with 64 spheres), the sample uses a shorter horizon of the same robot
and scene recipe, stated in the test. Where rounding-level branch choices make a config's per-problem
outcomes coin flips on a few percent of problems (paths), the sample is large enough that their
unbiased noise stays well inside one point.
"""
import concurrent.futures as cf
import dataclasses
import functools
import os

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import dev_soa, host_aos, orc_robot, orc_weights, targets_dev
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu

ONE_PT = 0.01


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _ik_cfg(ik, p0=0, S=None, n_final=None):
    return O.IkConfig(S=ik.S if S is None else S, n_final=ik.n_final if n_final is None else n_final, k_init=ik.k_init,
                      k_final=ik.k_final, lambda0=ik.lambda0, alpha0=ik.alpha0, dedup_eps=ik.dedup_eps,
                      lim_tol=ik.lim_tol, pos_tol=ik.pos_tol, rot_tol=ik.rot_tol, seed=ik.seed, p0=p0)


def _report(name, g, o):
    """Prints both rates and the mismatches; returns True when the success counts differ by at most
    one percentage point of the sample (compared as integer counts)."""
    g, o = np.asarray(g, bool), np.asarray(o, bool)
    d = g.mean() - o.mean()
    print(f"{name}: {len(g)} problems, success GPU {g.mean():.4f} oracle {o.mean():.4f} (difference "
          f"{100 * d:+.2f} pt), flag mismatches {int((g != o).sum())} (GPU only {int((g & ~o).sum())}, "
          f"oracle only {int((~g & o).sum())})")
    return abs(int(g.sum()) - int(o.sum())) <= int(np.floor(ONE_PT * len(g) + 1e-9))


@pytest.mark.parametrize("prec", [lib.CR_F32, lib.CR_F64])
def test_ik_3seg_success_200(prec):
    """The 3-segment two-stage IK workload (256 seeds, 64 PG steps, top 8, 30 LM), 200 targets."""
    spec, ik, P = synth.ROBOT_3SEG, synth.IK_3SEG, 200
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=13)
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, precision=prec)
    out = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    o = O.solve_ik(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, _ik_cfg(ik))
    assert _report(f"IK 3-segment prec={prec}", out.success.cpu().numpy(), o["success"])


def test_ik_e1_shape_success_200():
    """The arc model on the paper's IK benchmark shape (3 extendable 1 m segments, 128 seeds -> top 8,
    150 PG steps + 50 LM), 200 targets, FP32 bulk."""
    spec, ik, P = synth.ROBOT_E1, synth.IK_E1, 200
    rbo = orc_robot(spec)
    tg, _ = synth.e1_workload(spec, P, lambda x: O.fk(rbo, x)[0], seed=14)
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P)
    out = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    o = O.solve_ik(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, _ik_cfg(ik))
    assert _report("IK E1 shape (arc model)", out.success.cpu().numpy(), o["success"])


PATH_N, PATH_H = 2000, 8


@functools.lru_cache(maxsize=1)
def _path_case():
    """The path workload's robot and scene recipe, PATH_N paths of PATH_H waypoints, with the oracle's
    solve (computed once for both precisions)."""
    spec, ik = synth.ROBOT_4SEG, synth.IK_PATH0
    rbo = orc_robot(spec)
    wp, _, sph = synth.path_workload(spec, PATH_N, PATH_H, synth.NO_PATH, lambda u: O.fk(rbo, u, backbone=True),
                                     seed=15)
    o = O.solve_path(rbo, orc_weights(), sph, wp, _ik_cfg(ik), synth.K_WARM, synth.K_JOINT)
    tol_r = np.deg2rad(1.0)
    so = (o["pos"].max(1) <= 1e-3) & (o["rot"].max(1) <= tol_r) & o["lim_ok"] & o["col_ok"]
    return wp, sph, so


@pytest.mark.parametrize("prec", [lib.CR_F32, lib.CR_F64])
def test_path_success(prec):
    """Path following on the path workload's robot and scene recipe (4 segments, 16 backbone samples
    per segment, 32 spheres per path, first-waypoint IK of 64 seeds, 30 warm LM iterations per
    waypoint, 20 joint LM iterations) on 2000 paths of 8 waypoints (64 in the full workload). About
    one path in twenty takes a different, equally valid branch on the two sides (a warm start that
    converged onto a bound's kink, a cost tie of the redundant degrees of freedom), and those
    outcomes are coin flips without bias: 2000 paths keep the count difference they cause well
    inside one percentage point (20 paths); 200 did not resolve it."""
    spec, ik = synth.ROBOT_4SEG, synth.IK_PATH0
    P, H = PATH_N, PATH_H
    wp, sph, so = _path_case()
    s = api.PathSolver(spec, ik, synth.WEIGHTS, P, H, api.Scene(sph, per_problem=True), prec, synth.K_WARM,
                       synth.K_JOINT)
    s.solve(api.waypoints_soa(wp), 0)
    torch.cuda.synchronize()
    tol_r = np.deg2rad(1.0)
    pos, rot = s.pos.cpu().numpy().reshape(P, H), s.rot.cpu().numpy().reshape(P, H)
    g = (pos.max(1) <= 1e-3) & (rot.max(1) <= tol_r) & (s.lim_ok.cpu().numpy() > 0) & (s.col_ok.cpu().numpy() > 0)
    assert _report(f"path prec={prec}", g, so)


@pytest.mark.parametrize("prec", [lib.CR_F32, lib.CR_F64])
def test_traj_success_128(prec):
    """Trajectory planning on the trajectory workload's robot and scene recipe (3 segments, goal IK
    of 64 seeds -> top 4, linear initialiser, 100 PG steps), 128 problems of 16 states with 32
    spheres each (32 states and 64 spheres in the full workload: the oracle's complex-step gradient
    of the whole trajectory costs ~25 core-seconds per problem there)."""
    spec = synth.ROBOT_3SEG
    P, Tn = 128, 16
    rbo = orc_robot(spec)
    us, goal, sph, _ = synth.traj_workload(spec, P, 32, lambda u: O.fk(rbo, u, backbone=True), seed=16)
    ik = synth.IK_GOAL
    sol = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, api.Scene(sph, per_problem=True), precision=prec)
    sol.solve(dev_soa(us, torch.float64), dev_soa(goal, torch.float64))
    torch.cuda.synchronize()
    tol_r = np.deg2rad(1.0)
    g = ((sol.goal_pos.cpu().numpy() <= 1e-3) & (sol.goal_rot.cpu().numpy() <= tol_r) & (sol.lim_ok.cpu().numpy() > 0)
         & (sol.col_ok.cpu().numpy() > 0))
    r = O.solve_traj(rbo, orc_weights(), sph, us, goal, Tn, _ik_cfg(ik), synth.K_TRAJ, synth.ALPHA_TRAJ)
    so = (r["goal_pos"] <= 1e-3) & (r["goal_rot"] <= tol_r) & r["lim_ok"] & r["col_ok"]
    assert _report(f"trajectory prec={prec}", g, so)


def test_ragged_batch_success_200():
    """The ragged serving batch (persistent kernels, one CUDA graph, the serving settings: 64 PG
    steps, top 8, 30 LM, 30 warm and 20 joint iterations) on 200 items with segment counts 1-6 and
    spheres 0-64 as in the workload; paths shortened to 2-16 waypoints and seeds to 16-128 so the
    oracle solves the 200 items in seconds."""
    fam, ik = synth.ROBOT_FAMILY, synth.IK_RAGGED
    rng = np.random.default_rng(17)
    N = 200
    items = synth.ragged_items(rng, N)
    items[:, 2] = np.where(items[:, 0] == 1, rng.integers(2, 17, N), 1)
    items[:, 3] = rng.integers(16, 129, N)
    items, targets, spheres, _ = synth.ragged_workload(N, api.family_fk_backbone(fam), seed=17, items=items)
    s = api.BatchSolver(fam, items, ik, synth.WEIGHTS, synth.K_WARM, synth.K_JOINT, seeds_per_unit=32)
    s.set_inputs(targets, spheres)
    s.plan()
    s.run()
    torch.cuda.synchronize()
    g = (s.flags.cpu().numpy() & 1).astype(bool)
    w0 = np.concatenate([[0], np.cumsum(items[:, 2])])
    o0 = np.concatenate([[0], np.cumsum(items[:, 4])])

    def one(i):
        kind, n, H, S, no = (int(v) for v in items[i])
        tg = targets[w0[i]:w0[i] + H]
        sp = spheres[o0[i]:o0[i] + no] if no else None
        rbo = orc_robot(dataclasses.replace(fam, L=fam.L[:n]))
        cfg = _ik_cfg(ik, p0=i, S=S, n_final=min(ik.n_final, S))
        tol_r = np.deg2rad(1.0)
        if kind == 1 and H > 1:
            o = O.solve_path(rbo, orc_weights(), None if sp is None else sp[None], tg[None], cfg, synth.K_WARM,
                             synth.K_JOINT, threads=1)
            return bool((o["pos"][0] <= 1e-3).all() and (o["rot"][0] <= tol_r).all() and o["lim_ok"][0]
                        and o["col_ok"][0])
        return bool(O.solve_ik(rbo, orc_weights(), sp, 0, tg, cfg, threads=1)["success"][0])

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        so = np.array(list(ex.map(one, range(N))))
    assert _report("ragged batch", g, so)
