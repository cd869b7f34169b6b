"""GPU parity of the self-contact rows (Eq. ik_coll's minimum distance over the robot itself,
Sec. IV-A: backbone samples of segments two or more apart, weight rho_s) against the FP64 oracle:
cost, collision penalty and gradient (FP64 1e-12, FP32 1e-5 relative to the size of the data), LM
iterates, Algorithm 1 with the self-contact acceptance, and the trajectory cost; the solvers built
without the rows refuse rho_s > 0."""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (EPS, TDT, TOL, cost_errors, dev_soa, first_true, grad_errors, host_aos, kink_or_pi, near_ties,
                      orc_robot, pose_operand_scale, targets_dev)
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu

RHO_S = 1e4
W_SELF = dataclasses.replace(synth.WEIGHTS, rho_s=RHO_S)
SPEC = synth.RobotSpec(L=(0.1,) * 4, rc=0.005, umax=0.01, nb=8)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _ow(w=W_SELF):
    return O.make_weights(**w.as_dict())


def _curled_states(rng, B, spec=SPEC):
    return synth.curled_states(rng, B, spec)


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_cost_grad_with_self_rows(prec):
    rng = np.random.default_rng(900)
    P, S = 24, 8
    rbo = orc_robot(SPEC)
    u_true = synth.hexagon_states(rng, P, SPEC.n, SPEC.umax)
    tg = synth.pose_targets(O.fk(rbo, u_true)[0], "pose")
    u = _curled_states(rng, P * S)
    ug = dev_soa(u, TDT[prec])
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, W_SELF)
    cost, coll, gu, _ = api.cost_grad(api.robot_struct(SPEC), api.Scene(None), task, ug, grad=True, coll=True)
    torch.cuda.synchronize()
    ub = host_aos(ug)
    ref = O.ik_eval(rbo, _ow(), None, lib.CR_TASK_IK6, tg, S, ub, want=("F", "coll", "g", "r", "J"))
    assert (ref["coll"] > 0).mean() > 0.5  # most states have active self-contact rows
    rn = np.linalg.norm(ref["r"], axis=1)
    scale = pose_operand_scale(SPEC)
    Fp, Fd = cost_errors(cost.double().cpu().numpy(), ref["F"], rn, scale)
    Cp, Cd = cost_errors(coll.double().cpu().numpy(), ref["coll"], rn, scale)
    gp, gd = grad_errors(host_aos(gu), ref["g"], ref["J"], rn, scale)
    tol = TOL[prec]
    print(f"self rows prec={prec}: F plain {Fp.max():.2e} / data {Fd.max():.2e}; collision part data {Cd.max():.2e}; "
          f"gradient plain {gp.max():.2e} / data {gd.max():.2e} (tolerance {tol:.0e})")
    if prec == lib.CR_F64:
        assert Fp.max() <= tol and gp.max() <= tol
    assert Fd.max() <= tol and Cd.max() <= tol and gd.max() <= tol
    # rho_s = 0: the rows are gone (the collision penalty of these sphere-free states is exactly 0)
    task0 = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    _, coll0, _, _ = api.cost_grad(api.robot_struct(SPEC), api.Scene(None), task0, ug, grad=True, coll=True)
    assert float(coll0.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_lm_iterates_with_self_rows(prec):
    """LM iterations (one call each) from curled states towards self-intersecting poses' targets, against
    the oracle's iterate history, compared up to the first rounding-decided iteration (gpu_util);
    bounds as for the tendon model (1e-10 FP64, 1e-4 FP32, of the displacement bound)."""
    rng = np.random.default_rng(901)
    P, S, iters = 16, 4, 12
    rbo = orc_robot(SPEC)
    u_curl = _curled_states(rng, P)
    tg = synth.pose_targets(O.fk(rbo, u_curl)[0], "pose")
    u0 = np.repeat(u_curl, S, 0) + rng.normal(0, 1e-3, (P * S, SPEC.d))
    # strictly inside the bounds: a start clamped onto u_max sits on the bound hinge's kink once rounded
    # to FP32, and the comparison would stop at iteration 0
    u0 = np.clip(u0, -0.995 * SPEC.umax, 0.995 * SPEC.umax)
    ug = dev_soa(u0, TDT[prec])
    u0b = host_aos(ug)
    lam = torch.full((P * S,), 1e-3, dtype=torch.float64, device="cuda")
    nu = torch.full((P * S,), 2.0, dtype=torch.float64, device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, W_SELF)
    ref = O.ik_lm(rbo, _ow(), None, lib.CR_TASK_IK6, tg, S, u0b, iters, history=True)
    errs = []
    for it in range(iters):
        lib.cr_lm_step(api.robot_struct(SPEC), api.Scene(None).c, task, ug, lam, nu, n_iter=1)
        errs.append(np.abs(host_aos(ug) - ref["hist"][it]).max(axis=1) / SPEC.umax)
    err = np.array(errs).T
    B = P * S
    xstart = np.concatenate([u0b[:, None, :], ref["hist"][:-1].transpose(1, 0, 2)], axis=1)
    rs = O.ik_eval(rbo, _ow(), None, lib.CR_TASK_IK6, np.repeat(tg, S, 0).repeat(iters, 0), 1,
                   xstart.reshape(B * iters, -1), want=("r",))["r"].reshape(B, iters, -1)
    tie = near_ties(ref["Fstart"], ref["Ftrial"], EPS[prec], pose_operand_scale(SPEC))
    first = first_true(tie | kink_or_pi(xstart, SPEC, rs[:, :, 3:6], prec))
    checked = np.arange(iters)[None, :] < first[:, None]
    coll0 = O.ik_eval(rbo, _ow(), None, lib.CR_TASK_IK6, tg, S, u0b, want=("coll",))["coll"]
    tol = 1e-10 if prec == lib.CR_F64 else 1e-4
    print(f"self-row LM prec={prec}: {int((coll0 > 0).sum())} of {B} starts in contact; max error "
          f"{err[checked].max():.2e} over {int(checked.sum())} compared iterations")
    assert (coll0 > 0).mean() > 0.25  # a quarter or more of the starts are in self-contact
    assert checked[:, 0].mean() >= 0.9
    assert err[checked].max() <= tol, np.sort(err[checked])[-5:]


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_solve_ik_with_self_contact(prec):
    """Algorithm 1 with the self-contact rows and acceptance on 64 targets, half of them the poses of
    self-intersecting curled states (the solver must find another, contact-free configuration): success
    within 1 pt (counts) of the oracle, every success contact-free under the oracle's acceptance."""
    rng = np.random.default_rng(902)
    P = 64
    rbo = orc_robot(SPEC)
    u_t = np.concatenate([_curled_states(rng, P // 2), synth.hexagon_states(rng, P // 2, SPEC.n, SPEC.umax)])
    tg = synth.pose_targets(O.fk(rbo, u_t)[0], "pose")
    ik = synth.IkSpec(S=64, n_final=8, k_init=32, k_final=30)
    s = api.IkSolver(SPEC, ik, W_SELF, lib.CR_TASK_IK6, P, precision=prec)
    out = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    gs = out.success.cpu().numpy().astype(bool)
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps)
    o = O.solve_ik(rbo, _ow(), None, lib.CR_TASK_IK6, tg, cfg)
    pos, rot, lim, col = O.accept(rbo, None, lib.CR_TASK_IK6, tg, host_aos(out.u), ik.lim_tol, self_contact=True)
    assert np.array_equal(gs, (pos <= ik.pos_tol) & (rot <= ik.rot_tol) & lim & col)
    _, _, _, col_target = O.accept(rbo, None, lib.CR_TASK_IK6, tg, u_t, ik.lim_tol, self_contact=True)
    print(f"self-contact IK prec={prec}: success GPU {gs.mean():.3f} oracle {o['success'].mean():.3f}, mismatches "
          f"{int((gs != o['success']).sum())}; {int((~col_target).sum())} targets come from self-intersecting states")
    assert (~col_target).sum() >= P // 8
    assert abs(int(gs.sum()) - int(o["success"].sum())) <= max(1, int(0.01 * P))
    assert s.status() == 0


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_traj_cost_with_self_rows(prec):
    """Trajectory cost and adjoint with the self-contact rows on every free state, against the oracle."""
    rng = np.random.default_rng(903)
    P, Tn = 3, 6
    rbo = orc_robot(SPEC)
    us = _curled_states(rng, P)
    ug_ = _curled_states(rng, P)
    goal = synth.pose_targets(O.fk(rbo, ug_)[0], "pose")
    s_ = np.linspace(0, 1, Tn)[1:, None]
    x = us[:, None, :] + s_[None] * (ug_ - us)[:, None, :]
    scene = api.Scene(None)
    task = api.traj_task_struct(dev_soa(us, torch.float64), dev_soa(goal, torch.float64), Tn, W_SELF)
    xg = torch.as_tensor(x.reshape(P * (Tn - 1), -1).T.copy(), dtype=TDT[prec]).cuda()
    cost = torch.empty(P, dtype=TDT[prec], device="cuda")
    grad = torch.empty_like(xg)
    lib.cr_traj_cost(api.robot_struct(SPEC), scene.c, task, xg, cost, grad)
    torch.cuda.synchronize()
    xb = xg.double().cpu().numpy().T.reshape(x.shape)
    ref = O.traj_eval(rbo, _ow(), None, us, goal, xb, want=("F", "g"))
    ref0 = O.traj_eval(rbo, O.make_weights(**synth.WEIGHTS.as_dict()), None, us, goal, xb, want=("F",))
    assert np.any(ref["F"] > ref0["F"])  # the self rows are active along (some of) these trajectories
    g = grad.double().cpu().numpy().T.reshape(x.shape)
    eF = (np.abs(cost.double().cpu().numpy() - ref["F"]) / ref["F"]).max()
    eg = (np.abs(g - ref["g"]).reshape(P, -1).max(1) / np.abs(ref["g"]).reshape(P, -1).max(1)).max()
    tol = TOL[prec]
    print(f"self-row trajectory cost prec={prec}: F {eF:.2e}, gradient {eg:.2e} (tolerance {tol:.0e})")
    assert eF <= tol and eg <= tol
