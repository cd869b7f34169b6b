"""GPU parity of the coupled tendon routing (model B, Eq. l_eq read literally: the state holds the
actuator displacements q_sj = sum_{i <= s} u_ij) against the FP64 oracle: kinematics and Jacobian
(J_q = J_u D) for 1, 3 and 6 segments, cost and gradient with active bound and curvature rows, LM
iterates, and Algorithm 1's success rate. Tolerances as for the per-segment model."""
import dataclasses

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


def _spec(n, thmax=np.pi):
    return synth.RobotSpec(L=tuple([0.12, 0.10, 0.08, 0.1, 0.1, 0.1][:n]), rc=0.005, umax=0.01, nb=6, thmax=thmax,
                           coupled=True)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [1, 3, 6])
def test_fk_and_jacobian(prec, n):
    spec = _spec(n)
    rng = np.random.default_rng(1000 + n)
    B = 2 * 128 + 19
    q = synth.hexagon_states(rng, B, n, spec.umax)
    q[0] = 0.0
    qg = dev_soa(q, TDT[prec])
    rb = api.robot_struct(spec)
    T, bb = api.fk(rb, qg, backbone=True)
    J = api.fk_jac(rb, qg)
    torch.cuda.synchronize()
    qb = host_aos(qg)
    rbo = orc_robot(spec)
    To, bbo = O.fk(rbo, qb, backbone=True)
    Jo = O.tip_jacobian(rbo, qb)
    Jg = J.double().cpu().numpy().transpose(2, 0, 1)
    bbg = bb.double().cpu().numpy().transpose(2, 0, 1)
    e = dict(R=rowwise_rel(host_aos(T)[:, :9], To[:, :9], 1.0).max(),
             p=rowwise_rel(host_aos(T)[:, 9:], To[:, 9:], sum(spec.L)).max(),
             backbone=rowwise_rel(bbg.reshape(B, -1), bbo.reshape(B, -1), sum(spec.L)).max(),
             J_translation=rowwise_rel(Jg[:, :3].reshape(B, -1), Jo[:, :3].reshape(B, -1)).max(),
             J_rotation=rowwise_rel(Jg[:, 3:].reshape(B, -1), Jo[:, 3:].reshape(B, -1)).max())
    tol = TOL[prec]
    print(f"coupled FK/J n={n} prec={prec}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()) + f" (tolerance {tol:.0e})")
    assert max(e.values()) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_cost_grad(prec):
    """States near FK-built targets and far from them, some actuators beyond their bounds, bends past
    a lowered theta_max (the curvature row reaches two segments' actuators through u = D q)."""
    spec = _spec(3, thmax=1.3)
    rng = np.random.default_rng(1010)
    P, S = 32, 8
    rbo = orc_robot(spec)
    q_true = synth.hexagon_states(rng, P, 3, spec.umax)
    tg = synth.pose_targets(O.fk(rbo, q_true)[0], "pose")
    q = np.repeat(q_true, S, 0) + rng.normal(0, 3e-4, (P * S, 9))
    far = rng.random(P * S) < 0.5
    q[far] = synth.hexagon_states(rng, int(far.sum()), 3, spec.umax)
    q[::7] *= 1.3
    qg = dev_soa(q, TDT[prec])
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    cost, _, gu, gp = api.cost_grad(api.robot_struct(spec), api.Scene(None), task, qg, grad=True, param_grad=True)
    gsum = api.reduce_rows(gp)
    torch.cuda.synchronize()
    qb = host_aos(qg)
    W = orc_weights()
    ref = O.ik_eval(rbo, W, None, lib.CR_TASK_IK6, tg, S, qb, want=("F", "g", "r", "J"))
    rn = np.linalg.norm(ref["r"], axis=1)
    scale = pose_operand_scale(spec)
    Fp, Fd = cost_errors(cost.double().cpu().numpy(), ref["F"], rn, scale)
    gp_, gd = grad_errors(host_aos(gu), ref["g"], ref["J"], rn, scale)
    pg = O.ik_param_grad(rbo, W, None, lib.CR_TASK_IK6, tg, S, qb)
    ep = np.abs(gsum.cpu().numpy() - pg).max() / np.abs(pg).max()
    curv = ref["r"][:, 6 + 18 + 3:6 + 18 + 6]
    tol = TOL[prec]
    print(f"coupled cost prec={prec}: F plain {Fp.max():.2e} / data {Fd.max():.2e}; gradient plain {gp_.max():.2e} / "
          f"data {gd.max():.2e}; parameter gradient {ep:.2e}; states with active curvature rows "
          f"{int((np.abs(curv) > 0).any(1).sum())} (tolerance {tol:.0e})")
    assert (np.abs(curv) > 0).any(1).sum() >= 5
    if prec == lib.CR_F64:
        assert Fp.max() <= tol and gp_.max() <= tol
    assert Fd.max() <= tol and gd.max() <= tol and ep <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_lm_iterates(prec):
    spec = _spec(3)
    rbo = orc_robot(spec)
    rng = np.random.default_rng(1011)
    P, S, iters = 32, 4, 20
    q_true = synth.hexagon_states(rng, P, 3, spec.umax)
    tg = synth.pose_targets(O.fk(rbo, q_true)[0], "pose")
    q0 = np.repeat(q_true, S, 0) + rng.normal(0, 1.5e-3, (P * S, 9))
    qg = dev_soa(q0, TDT[prec])
    q0b = host_aos(qg)
    lam = torch.full((P * S,), 1e-3, dtype=torch.float64, device="cuda")
    nu = torch.full((P * S,), 2.0, dtype=torch.float64, device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    ref = O.ik_lm(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, S, q0b, iters, history=True)
    errs = []
    for it in range(iters):
        lib.cr_lm_step(api.robot_struct(spec), api.Scene(None).c, task, qg, lam, nu, n_iter=1)
        errs.append(np.abs(host_aos(qg) - ref["hist"][it]).max(axis=1) / spec.umax)
    err = np.array(errs).T
    B = P * S
    xstart = np.concatenate([q0b[:, None, :], ref["hist"][:-1].transpose(1, 0, 2)], axis=1)
    rs = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tg, S, 0).repeat(iters, 0), 1,
                   xstart.reshape(B * iters, -1), want=("r",))["r"].reshape(B, iters, -1)
    tie = near_ties(ref["Fstart"], ref["Ftrial"], EPS[prec], pose_operand_scale(spec))
    first = first_true(tie | kink_or_pi(xstart, spec, rs[:, :, 3:6], prec))
    checked = np.arange(iters)[None, :] < first[:, None]
    tol = 1e-10 if prec == lib.CR_F64 else 1e-4
    print(f"coupled LM prec={prec}: max error {err[checked].max():.2e} of the bound over {int(checked.sum())} "
          f"compared iterations")
    assert checked[:, 0].mean() >= 0.9
    assert err[checked].max() <= tol, np.sort(err[checked])[-5:]


@pytest.mark.parametrize("prec", PRECS)
def test_solve_ik_success(prec):
    """Algorithm 1 on 200 targets of the 3-segment robot with coupled routing: success within 1 pt
    (counts) of the oracle, every GPU result valid under the oracle's acceptance (bounds on q)."""
    spec, ik, P = _spec(3), synth.IK_3SEG, 200
    rbo = orc_robot(spec)
    rng = np.random.default_rng(1012)
    tg = synth.pose_targets(O.fk(rbo, synth.hexagon_states(rng, P, 3, spec.umax))[0], "pose")
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, precision=prec)
    out = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    gs = out.success.cpu().numpy().astype(bool)
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps)
    o = O.solve_ik(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, cfg)
    pos, rot, lim, col = O.accept(rbo, None, lib.CR_TASK_IK6, tg, host_aos(out.u), ik.lim_tol)
    assert np.array_equal(gs, (pos <= ik.pos_tol) & (rot <= ik.rot_tol) & lim & col)
    print(f"coupled IK prec={prec}: success GPU {gs.mean():.3f} oracle {o['success'].mean():.3f}, mismatches "
          f"{int((gs != o['success']).sum())}")
    assert abs(int(gs.sum()) - int(o["success"].sum())) <= int(0.01 * P)
    assert s.status() == 0
