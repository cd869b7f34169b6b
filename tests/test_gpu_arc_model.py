"""GPU parity of the arc model (the paper's own (theta, phi, L) per segment, extendable lengths)
against the FP64 oracle: kinematics, tip Jacobian (with the length columns), cost and gradient with
length, curvature and clearance rows, bit-identical seeds, LM iterates, and Algorithm 1 on the
shapes of the paper's IK benchmarks (1 m segments, 128 seeds -> top 8, 200 iterations; the sphere
lattice). Tolerances as in the tendon-model tests: FP64 1e-12, FP32 1e-5 (norm-wise per state; the
FP32 cost and gradient relative to the size of their data, gpu_util.cost_errors / grad_errors).
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (EPS, TDT, TOL, cost_errors, dev_soa, first_true, grad_errors, host_aos, kink_or_pi, near_ties,
                      orc_robot, orc_weights, pose_operand_scale, rowwise_rel, targets_dev)
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu

PRECS = [lib.CR_F64, lib.CR_F32]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _states(spec, rng, B):
    """Uniform configurations plus the degenerate ones: straight, nearly straight, on the bounds."""
    q = synth.arc_states(rng, B, spec)
    q[0, 0::3] = q[0, 1::3] = 0.0
    q[1, 0::3] *= 1e-9
    q[1, 1::3] *= 1e-9
    q[2, 2::3] = spec.lmax
    q[3, 2::3] = spec.lmin
    return q


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("spec", [synth.ROBOT_E1, synth.ROBOT_E2_EXT, synth.arc_robot(1, True)])
def test_fk_and_jacobian_parity(prec, spec):
    rng = np.random.default_rng(600)
    B = 3 * 128 + 29
    q = _states(spec, rng, B)
    rb = api.robot_struct(spec)
    qg = dev_soa(q, TDT[prec])
    T, bb = api.fk(rb, qg, backbone=True)
    J = api.fk_jac(rb, qg)
    torch.cuda.synchronize()
    qb = host_aos(qg)
    rbo = orc_robot(spec)
    To, bbo = O.fk(rbo, qb, backbone=True)
    tol = TOL[prec]
    reach = spec.n * spec.lmax
    bbg = bb.double().cpu().numpy().transpose(2, 0, 1)
    Jo = O.tip_jacobian(rbo, qb)
    Jg = J.double().cpu().numpy().transpose(2, 0, 1)
    e = dict(R=rowwise_rel(host_aos(T)[:, :9], To[:, :9], 1.0).max(),
             p=rowwise_rel(host_aos(T)[:, 9:], To[:, 9:], reach).max(),
             backbone=rowwise_rel(bbg.reshape(B, -1), bbo.reshape(B, -1), reach).max(),
             J_translation=rowwise_rel(Jg[:, :3].reshape(B, -1), Jo[:, :3].reshape(B, -1)).max(),
             J_rotation=rowwise_rel(Jg[:, 3:].reshape(B, -1), Jo[:, 3:].reshape(B, -1)).max())
    print(f"arc FK/J n={spec.n} prec={prec}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()) + f" (tolerance {tol:.0e})")
    assert max(e.values()) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_cost_grad_parity(prec):
    """Length, curvature and clearance rows active: states near FK-built targets and far from them,
    some lengths outside [lmin, lmax] and bends beyond theta_max, spheres on the backbones."""
    spec = synth.RobotSpec(L=(1.0,) * 3, rc=0.1, umax=0.01, nb=10, thmax=2.0, rbody=0.1, lmin=0.5, lmax=1.5)
    rng = np.random.default_rng(601)
    P, S = 40, 8
    rbo = orc_robot(spec)
    q_true = synth.arc_states(rng, P, spec)
    T, bb = O.fk(rbo, q_true, backbone=True)
    tg = synth.pose_targets(T, "pose")
    q = np.repeat(q_true, S, axis=0) + rng.normal(0, 1e-2, (P * S, spec.d))
    far = rng.random(P * S) < 0.5
    q[far] = synth.arc_states(rng, int(far.sum()), spec)
    q[::5, 2] = rng.uniform(0.3, 1.8, len(q[::5]))   # lengths out of bounds
    q[::7, :2] *= 1.6                                # bends beyond theta_max
    pick = bb[rng.integers(0, P, 12), rng.integers(0, spec.n * spec.nb, 12)]
    spheres = np.concatenate([pick + rng.normal(0, 0.05, pick.shape), rng.uniform(0.05, 0.15, (12, 1))], 1)
    qg = dev_soa(q, TDT[prec])
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    cost, coll, gu, _ = api.cost_grad(api.robot_struct(spec), api.Scene(spheres), task, qg, grad=True, coll=True)
    torch.cuda.synchronize()
    qb = host_aos(qg)
    ref = O.ik_eval(rbo, orc_weights(), spheres, lib.CR_TASK_IK6, tg, S, qb, want=("F", "coll", "g", "r", "J"))
    rn = np.linalg.norm(ref["r"], axis=1)
    scale = pose_operand_scale(spec)
    tol = TOL[prec]
    assert (ref["coll"] > 0).sum() > 10
    Fp, Fd = cost_errors(cost.double().cpu().numpy(), ref["F"], rn, scale)
    _, Cd = cost_errors(coll.double().cpu().numpy(), ref["coll"], rn, scale)
    gp, gd = grad_errors(host_aos(gu), ref["g"], ref["J"], rn, scale)
    print(f"arc cost prec={prec}: F plain {Fp.max():.2e} / data {Fd.max():.2e}; clearance part data {Cd.max():.2e}; "
          f"gradient plain {gp.max():.2e} / data {gd.max():.2e} (tolerance {tol:.0e})")
    if prec == lib.CR_F64:
        assert Fp.max() <= tol and gp.max() <= tol
    assert Fd.max() <= tol and Cd.max() <= tol and gd.max() <= tol


def test_seeds_bitwise():
    spec = synth.ROBOT_E2_EXT
    P, S, p0, key = 23, 70, 5, 777
    ref = O.seeds(orc_robot(spec), orc_weights(), None, key, p0, P, S).reshape(P * S, -1)
    for prec in PRECS:
        out = torch.empty((spec.d, P * S), dtype=TDT[prec], device="cuda")
        lib.cr_seeds(api.robot_struct(spec), api.Scene(None).c, api.weights_struct(synth.WEIGHTS), key, p0, P, S, out)
        want = ref if prec == lib.CR_F64 else ref.astype(np.float32).astype(np.float64)
        assert np.array_equal(host_aos(out), want)


@pytest.mark.parametrize("prec,n", [(lib.CR_F64, 2), (lib.CR_F64, 3), (lib.CR_F32, 2)])
def test_lm_iterates(prec, n):
    """20 LM iterations, one call each, against the oracle's iterate history, every seed compared up
    to the first iteration whose outcome rounding decides (a decision tie, a hinge at its kink, in
    FP32 a rotation error near pi; gpu_util). Bounds in the state's units (rad, m): FP32 bulk (FP64
    Cholesky, two-float normal equations) 1e-4 and FP64 1e-10 on the 2-segment robot, whose pose
    fixes the solution; FP64 1e-9 on the 3-segment robot, which is redundant (9 parameters for a
    6-DoF pose): the damped step's component in the 3-dimensional null space is set by the damping,
    and rounding-level differences there grow over the iterations (measured 1.4e-10)."""
    spec = synth.arc_robot(n, True)
    rbo = orc_robot(spec)
    rng = np.random.default_rng(602)
    P, S, iters = 32, 4, 20
    q_true = synth.arc_states(rng, P, spec)
    tg = synth.pose_targets(O.fk(rbo, q_true)[0], "pose")
    q0 = np.repeat(q_true, S, 0) + rng.normal(0, 0.05, (P * S, spec.d))
    qg = dev_soa(q0, TDT[prec])
    q0b = host_aos(qg)
    lam = torch.full((P * S,), 1e-3, dtype=torch.float64, device="cuda")
    nu = torch.full((P * S,), 2.0, dtype=torch.float64, device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    ref = O.ik_lm(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, S, q0b, iters, history=True)
    errs = []
    for it in range(iters):
        lib.cr_lm_step(api.robot_struct(spec), api.Scene(None).c, task, qg, lam, nu, n_iter=1)
        errs.append(np.abs(host_aos(qg) - ref["hist"][it]).max(axis=1))
    err = np.array(errs).T
    B = P * S
    xstart = np.concatenate([q0b[:, None, :], ref["hist"][:-1].transpose(1, 0, 2)], axis=1)
    rs = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tg, S, 0).repeat(iters, 0), 1,
                   xstart.reshape(B * iters, -1), want=("r",))["r"].reshape(B, iters, -1)
    tie = near_ties(ref["Fstart"], ref["Ftrial"], EPS[prec], pose_operand_scale(spec))
    first = first_true(tie | kink_or_pi(xstart, spec, rs[:, :, 3:6], prec))
    checked = np.arange(iters)[None, :] < first[:, None]
    tol = 1e-4 if prec == lib.CR_F32 else (1e-10 if n == 2 else 1e-9)
    print(f"arc LM n={n} prec={prec}: max error {err[checked].max():.2e} over {int(checked.sum())} compared "
          f"iterations; {int((first < iters).sum())} of {len(first)} seeds reach a rounding-decided iteration")
    assert err[checked].max() <= tol, np.sort(err[checked])[-5:]
    assert checked[:, 0].mean() >= 0.9  # the first iteration is compared for (almost) every seed
    assert np.mean(ref["F"] < 1e-12) > 0.5


def _oracle_solve(spec, ik, tg, spheres=None, p0=0):
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, lim_tol=ik.lim_tol, pos_tol=ik.pos_tol,
                     rot_tol=ik.rot_tol, seed=ik.seed, p0=p0)
    return O.solve_ik(orc_robot(spec), orc_weights(), spheres, lib.CR_TASK_IK6, tg, cfg)


@pytest.mark.parametrize("prec", PRECS)
def test_solve_e1_shape(prec):
    """Algorithm 1 with the benchmark's settings on 48 targets of the 3-segment extendable robot:
    success within 1 pt (+1 target) of the oracle, every GPU solution valid under the oracle."""
    spec, ik, P = synth.ROBOT_E1, synth.IK_E1, 48
    rbo = orc_robot(spec)
    tg, _ = synth.e1_workload(spec, P, lambda x: O.fk(rbo, x)[0], seed=11)
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, precision=prec)
    o = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    gs = o.success.cpu().numpy().astype(bool)
    ref = _oracle_solve(spec, ik, tg)
    assert s.status() == 0
    assert abs(gs.mean() - ref["success"].mean()) <= 0.01 + 1.0 / P
    pos, rot, lim, col = O.accept(rbo, None, lib.CR_TASK_IK6, tg, host_aos(o.u), ik.lim_tol)
    np.testing.assert_allclose(o.pos_err.cpu().numpy(), pos, rtol=1e-6, atol=1e-12)
    assert np.array_equal(gs, (pos <= ik.pos_tol) & (rot <= ik.rot_tol) & lim & col)


def test_solve_e2_shape_lattice():
    """The sphere lattice with the 4-segment extendable robot (FP32 bulk, FP64 refine) on 16
    collision-free targets, and the 3-segment fixed-length robot (lengths pinned by equal bounds)."""
    ik = synth.IK_E1
    for spec, P in ((synth.ROBOT_E2_EXT, 16), (synth.ROBOT_E2_FIXED, 12)):
        rbo = orc_robot(spec)
        tg, _, sph = synth.e2_workload(spec, P, lambda x: O.fk(rbo, x, backbone=True), seed=12)
        s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, api.Scene(sph))
        o = s.solve(targets_dev(tg))
        torch.cuda.synchronize()
        gs = o.success.cpu().numpy().astype(bool)
        ref = _oracle_solve(spec, ik, tg, spheres=sph)
        assert np.sum(gs != ref["success"].astype(bool)) <= 1
        u = host_aos(o.u)
        pos, rot, lim, col = O.accept(rbo, sph, lib.CR_TASK_IK6, tg, u, ik.lim_tol)
        assert np.array_equal(gs, (pos <= ik.pos_tol) & (rot <= ik.rot_tol) & lim & col)
        if spec.lmin == spec.lmax:
            assert np.all(np.abs(u[gs][:, 2::3] - spec.lmin) <= 1e-5)


def test_tendon_only_entry_points_refuse_the_arc_model():
    spec = synth.ROBOT_E1
    U = torch.zeros((spec.d, 4), dtype=torch.float64, device="cuda")
    Pm = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    th = torch.ones(2 * spec.n, dtype=torch.float64, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.CrError) as e:
        lib.cr_calibrate(api.robot_struct(spec), U, Pm, th, 2, 1e-3, F, None, ws)
    assert e.value.status == lib.CR_EINVAL
