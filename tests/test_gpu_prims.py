"""GPU parity of the obstacle primitives (capsules and boxes, the convex pieces of Sec. IV-C, in the
clearance rows of Eq. ik_coll) against the FP64 oracle: the cost, its gradient and the LM normal
equations of states near and inside the primitives, the two-stage IK solve with a shared and with
per-problem primitive sets, trajectories among shelves and paths among primitives.

Tolerances are those of the sphere tests: FP64 1e-12 and FP32 1e-5 relative to the data the cost
is formed from (gpu_util.cost_errors, grad_errors); solves agree on the success flags of all but
one problem in a small batch and every joint success is collision-free by the oracle's check.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (EPS, TDT, TOL, cost_errors, dev_soa, grad_errors, host_aos, near_ties, orc_robot,
                      orc_weights, pose_operand_scale, targets_dev)
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _prims_on_backbones(rng, bb, n_caps, n_boxes):
    """Capsules through and boxes around random backbone samples (so that some samples lie inside a
    box and some pairs are active), with random sizes and orientations."""
    pts = bb.reshape(-1, 3)
    out = []
    for _ in range(n_caps):
        c = pts[rng.integers(len(pts))] + rng.normal(0, 3e-3, 3)
        v = rng.normal(size=3)
        v *= rng.uniform(0.005, 0.03) / np.linalg.norm(v)
        out.append(synth.capsule_record(c - v, c + v, rng.uniform(0.002, 0.006)))
    q = synth.random_quaternions(rng, n_boxes)
    for k in range(n_boxes):
        c = pts[rng.integers(len(pts))] + rng.normal(0, 3e-3, 3)
        out.append(synth.box_record(c, rng.uniform(0.003, 0.02, 3), q[k], rng.uniform(0.0, 0.004) * (k % 2)))
    return np.array(out)


def _case(spec, rng, P, S, kind=lib.CR_TASK_IK6):
    rbo = orc_robot(spec)
    u_true = synth.hexagon_states(rng, P, spec.n, spec.umax)
    T, bb = O.fk(rbo, u_true, backbone=True)
    tg = synth.pose_targets(T, "pose" if kind == lib.CR_TASK_IK6 else "axis")
    u = np.repeat(u_true, S, axis=0) + rng.normal(0, 3e-4, (P * S, spec.d))
    far = rng.random(P * S) < 0.5
    u[far] = synth.hexagon_states(rng, int(far.sum()), spec.n, spec.umax)
    prims = _prims_on_backbones(rng, bb, 5, 7)
    pick = bb[rng.integers(0, P, 4), rng.integers(0, spec.n * spec.nb, 4)]
    sph = np.concatenate([pick + rng.normal(0, 2e-3, pick.shape), rng.uniform(3e-3, 8e-3, (4, 1))], 1)
    return rbo, tg, u, sph, prims


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
@pytest.mark.parametrize("kind", [lib.CR_TASK_IK6, lib.CR_TASK_IK5])
def test_cost_grad_parity_with_primitives(prec, kind):
    spec = synth.ROBOT_3SEG
    rng = np.random.default_rng(900 + kind)
    P, S = 40, 8  # 320 states: two blocks of 128 and a ragged tail
    rbo, tg, u, sph, prims = _case(spec, rng, P, S, kind)
    ug = dev_soa(u, TDT[prec])
    scene = api.Scene(sph, prims=prims)
    task = api.task_struct(kind, targets_dev(tg), S, synth.WEIGHTS)
    cost, coll, gu, gp = api.cost_grad(api.robot_struct(spec), scene, task, ug, grad=True, param_grad=False, coll=True)
    torch.cuda.synchronize()
    ub = host_aos(ug)
    ref = O.ik_eval(rbo, orc_weights(), (sph, prims), kind, tg, S, ub, want=("F", "coll", "g", "r", "J"))
    _, bb = O.fk(rbo, ub, backbone=True)
    inside = sum(int((O.obstacle_sd(rec, bb.reshape(-1, 3)) < 0).sum()) for rec in prims if rec[0] == synth.PRIM_BOX)
    active = int((ref["coll"] > 0).sum())
    assert inside > 0 and active > 20
    rn = np.linalg.norm(ref["r"], axis=1)
    scale = pose_operand_scale(spec)
    Fp, Fd = cost_errors(cost.double().cpu().numpy(), ref["F"], rn, scale)
    Cp, Cd = cost_errors(coll.double().cpu().numpy(), ref["coll"], rn, scale)
    gp_, gd = grad_errors(host_aos(gu), ref["g"], ref["J"], rn, scale)
    tol = TOL[prec]
    print(f"primitives kind={kind} prec={prec}: {active} states with active clearance rows, {inside} samples inside "
          f"boxes; F data {Fd.max():.2e}, clearance data {Cd.max():.2e}, gradient data {gd.max():.2e} "
          f"(tolerance {tol:.0e})")
    if prec == lib.CR_F64:
        assert Fp.max() <= tol and gp_.max() <= tol
    assert Fd.max() <= tol and Cd.max() <= tol and gd.max() <= tol


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_lm_step_with_primitives(prec):
    """One LM iteration (the normal equations with the primitives' clearance rows) from states near
    the targets, against the oracle's first iterate. Seeds whose step acceptance rounding decides
    (a near-tie of trial and start costs) are left out; bound 1e-10 (FP64), 1e-4 (FP32) of the
    displacement bound."""
    spec = synth.ROBOT_3SEG
    rng = np.random.default_rng(910)
    P, S = 32, 4
    rbo = orc_robot(spec)
    u_true = synth.hexagon_states(rng, P, 3, spec.umax)
    T, bb = O.fk(rbo, u_true, backbone=True)
    tg = synth.pose_targets(T, "pose")
    prims = _prims_on_backbones(rng, bb, 6, 8)
    u0 = np.repeat(u_true, S, 0) + rng.normal(0, 1.5e-3, (P * S, 9))
    ug = dev_soa(u0, TDT[prec])
    u0b = host_aos(ug)
    lam = torch.full((P * S,), 1e-3, dtype=torch.float64, device="cuda")
    nu = torch.full((P * S,), 2.0, dtype=torch.float64, device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    lib.cr_lm_step(api.robot_struct(spec), api.Scene(None, prims=prims).c, task, ug, lam, nu, n_iter=1)
    torch.cuda.synchronize()
    ref = O.ik_lm(rbo, orc_weights(), (None, prims), lib.CR_TASK_IK6, tg, S, u0b, 1, history=True)
    coll = O.ik_eval(rbo, orc_weights(), (None, prims), lib.CR_TASK_IK6, tg, S, u0b, want=("coll",))["coll"]
    err = np.abs(host_aos(ug) - ref["hist"][0]).max(axis=1) / spec.umax
    tie = near_ties(ref["Fstart"], ref["Ftrial"], EPS[prec], pose_operand_scale(spec))[:, 0]
    ok = ~tie
    tol = 1e-10 if prec == lib.CR_F64 else 1e-4
    print(f"LM with primitives prec={prec}: {int((coll > 0).sum())} of {P * S} starts with active clearance rows; "
          f"max error {err[ok].max():.2e} over {int(ok.sum())} seeds ({int(tie.sum())} near-ties)")
    assert (coll > 0).sum() >= 16 and ok.mean() >= 0.9
    assert err[ok].max() <= tol


def _solve(spec, ik, tg, prec, scene, plain=False):
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, len(tg), scene, prec, plain)
    o = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    return s, dict(u=host_aos(o.u), F=o.cost.cpu().numpy(), success=o.success.cpu().numpy().astype(bool))


def _oracle_solve(spec, ik, tg, obs, p0=0):
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, lim_tol=ik.lim_tol, pos_tol=ik.pos_tol,
                     rot_tol=ik.rot_tol, seed=ik.seed, p0=p0)
    return O.solve_ik(orc_robot(spec), orc_weights(), obs, lib.CR_TASK_IK6, tg, cfg)


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_solve_ik_shared_primitives(prec):
    """A shelf of boxes and a few capsules shared by 48 targets: success flags as the oracle's for all
    but one target, and every GPU success collision-free by the oracle's check."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=48, n_final=6, k_init=20, k_final=20)
    P = 48
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=11)
    rng = np.random.default_rng(12)
    prims = np.concatenate([synth.shelf_prims([0.09, 0.0, 0.0], 0.4, 0.16, 0.08, 0.17, 3, 0.008),
                            synth.prims_uniform(rng, 3, 0, [-0.08, -0.08, 0.05], [0.08, 0.08, 0.16], 0.003, 0.006,
                                                0.01, 0.03)])
    s, g = _solve(spec, ik, tg, prec, api.Scene(None, prims=prims))
    assert s.status() == 0
    o = _oracle_solve(spec, ik, tg, (None, prims))
    mism = int(np.sum(g["success"] != o["success"]))
    _, _, _, col = O.accept(rbo, (None, prims), lib.CR_TASK_IK6, tg, g["u"], ik.lim_tol)
    print(f"shared primitives prec={prec}: success GPU {g['success'].mean():.3f} oracle {o['success'].mean():.3f}, "
          f"{mism} flag mismatches; GPU solutions collision-free {col.mean():.3f}")
    assert mism <= 1
    assert np.all(col[g["success"]])
    assert 0.2 < o["success"].mean() < 1.0 or (~col).any()  # the scene constrains the solutions


@pytest.mark.parametrize("K,prec", [(5, lib.CR_F32), (10, lib.CR_F32), (5, lib.CR_F64)])
def test_solve_ik_per_problem_primitives(K, prec):
    """Each target with its own spheres and primitives, 30 targets: FP32 with 5 candidates takes the
    warp-cooperative refine, 10 the packed one; against the oracle target by target."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=40, n_final=K, k_init=12, k_final=15)
    P = 30
    rbo = orc_robot(spec)
    tg, u_true = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=13)
    rng = np.random.default_rng(14)
    sph = np.concatenate([rng.uniform(-0.05, 0.05, (P, 2, 2)), rng.uniform(0.05, 0.15, (P, 2, 1)),
                          rng.uniform(0.005, 0.012, (P, 2, 1))], axis=2)
    prims = np.stack([synth.prims_uniform(rng, 2, 2, [-0.05, -0.05, 0.05], [0.05, 0.05, 0.15], 0.003, 0.008,
                                          0.008, 0.025) for _ in range(P)])
    scene = api.Scene(sph, per_problem=True, prims=prims)
    s, g = _solve(spec, ik, tg, prec, scene)
    assert s.status() == 0
    agree = 0
    for p in range(P):
        r = _oracle_solve(spec, ik, tg[p:p + 1], (sph[p], prims[p]), p0=p)
        agree += int(bool(r["success"][0]) == g["success"][p])
        if g["success"][p]:
            _, _, lim, col = O.accept(rbo, (sph[p], prims[p]), lib.CR_TASK_IK6, tg[p:p + 1], g["u"][p:p + 1],
                                      ik.lim_tol)
            assert lim[0] and col[0]
    print(f"per-problem primitives K={K} prec={prec}: {agree} of {P} success flags agree")
    assert agree >= P - 1


def test_plain_form_with_primitives():
    """The plain FP64 comparator takes the same primitives: same success flags as the optimised FP64
    solve, states within 1e-9 where both succeed."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=32, n_final=4, k_init=10, k_final=12)
    P = 6
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=15)
    prims = synth.prims_uniform(np.random.default_rng(16), 2, 3, [-0.06, -0.06, 0.04], [0.06, 0.06, 0.16], 0.003,
                                0.008, 0.01, 0.03)
    _, a = _solve(spec, ik, tg, lib.CR_F64, api.Scene(None, prims=prims))
    _, b = _solve(spec, ik, tg, lib.CR_F64, api.Scene(None, prims=prims), plain=True)
    assert np.array_equal(a["success"], b["success"])
    both = a["success"] & b["success"]
    assert np.abs(a["u"][both] - b["u"][both]).max(initial=0.0) <= 1e-9


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_traj_among_shelves(prec):
    """Trajectories of 16 states with a shelf and two capsules per problem, placed clear of the start
    and goal backbones: collision and limit flags as the oracle's, costs within the trajectory
    tolerances (FP64 1e-4 relative; FP32 5 %)."""
    spec = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=8)
    rbo = orc_robot(spec)
    P, Tn = 4, 16
    us, goal, _, ug = synth.traj_workload(spec, P, 0, lambda u: O.fk(rbo, u, backbone=True), seed=17)
    rng = np.random.default_rng(18)
    _, bb = O.fk(rbo, np.concatenate([us, ug]), backbone=True)
    clear = spec.rc + synth.WEIGHTS.delta
    far = synth.capsule_record([10.0, 10.0, 10.0], [10.0, 10.0, 10.0], 0.0)  # stands in for a dropped board
    prims = []
    for p in range(P):
        pts = np.concatenate([bb[p], bb[P + p]])
        shelf = synth.shelf_prims(pts.mean(0) + [0.12, 0.0, -0.1], rng.uniform(-0.5, 0.5), 0.2, 0.1, 0.25, 3, 0.008)
        shelf = np.array([r if np.min(O.obstacle_sd(r, pts)) >= r[1] + clear else far for r in shelf])
        caps = synth.prims_clear_of(rng, 2, 0, pts, 0.03, 0.003, 0.008, 0.01, 0.03, clear, O.obstacle_sd)
        prims.append(np.concatenate([shelf, caps]))
    prims = np.stack(prims)
    assert (prims[:, :, 0] == synth.PRIM_BOX).sum() >= P
    ik = synth.IK_GOAL
    sol = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, api.Scene(None, per_problem=True, prims=prims),
                         precision=prec)
    sol.solve(dev_soa(us, torch.float64), dev_soa(goal, torch.float64))
    torch.cuda.synchronize()
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final)
    ref = O.solve_traj(rbo, orc_weights(), (None, prims), us, goal, Tn, cfg, synth.K_TRAJ, synth.ALPHA_TRAJ)
    for k in ("lim_ok", "col_ok"):
        assert np.array_equal(getattr(sol, k).cpu().numpy().astype(bool), ref[k]), k
    rt = 1e-4 if prec == lib.CR_F64 else 0.05
    np.testing.assert_allclose(sol.cost.cpu().numpy(), ref["F"], rtol=rt)


def test_path_among_primitives():
    """Paths of 12 waypoints with per-path capsules and boxes clear of the reference backbones: the
    FP64 solve's flags as the oracle's and its states within 1e-6 of the bound of the oracle's."""
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=8)
    rbo = orc_robot(spec)
    P, H = 6, 12
    wp, states, _ = synth.path_workload(spec, P, H, 0, lambda u: O.fk(rbo, u, backbone=True), seed=19)
    rng = np.random.default_rng(20)
    _, bb = O.fk(rbo, states.reshape(P * H, -1), backbone=True)
    bb = bb.reshape(P, -1, 3)
    prims = np.stack([synth.prims_clear_of(rng, 2, 3, bb[p], 0.02, 0.003, 0.008, 0.01, 0.025,
                                           spec.rc + synth.WEIGHTS.delta, O.obstacle_sd) for p in range(P)])
    ik = synth.IkSpec(S=32, n_final=4, k_init=16, k_final=20)
    s = api.PathSolver(spec, ik, synth.WEIGHTS, P, H, api.Scene(None, per_problem=True, prims=prims), lib.CR_F64,
                       10, 8)
    s.solve(api.waypoints_soa(wp), 0)
    torch.cuda.synchronize()
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0)
    o = O.solve_path(rbo, orc_weights(), (None, prims), wp, cfg, 10, 8)
    gx = s.X.cpu().numpy().T.reshape(P, H, -1)
    for k in ("lim_ok", "col_ok"):
        assert np.array_equal(getattr(s, k).cpu().numpy().astype(bool), o[k]), k
    err = np.abs(gx - o["x"]).max(axis=(1, 2)) / spec.umax
    print(f"paths among primitives: state error per path {np.array2string(err, precision=2)}")
    assert np.median(err) <= 1e-6
