"""GPU parity of the kinematics, Jacobian, cost and adjoint entry points against the FP64 oracle.

Tolerances: FP64 1e-12 and FP32 1e-5, relative, norm-wise per state and per quantity (the largest
component of that quantity sets the scale; lengths scale with the reach). The cost and gradient in
FP32 are measured relative to the size of the data they are formed from (gpu_util.cost_errors,
grad_errors): a least-squares cost near its zero cannot be computed to a relative accuracy better
than the rounding of its operands over the residual. Every test prints the measured maxima.
Batches span several 128-thread blocks plus a ragged tail, and include the straight and
nearly-straight configurations, states on the bounds, and rotations near pi.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (TDT, TOL, cost_errors, dev_soa, edge_states, grad_errors, host_aos, orc_robot, orc_weights,
                      pose_operand_scale, rowwise_rel, targets_dev)
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu

PRECS = [lib.CR_F64, lib.CR_F32]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("spec", [synth.ROBOT_1SEG, synth.ROBOT_3SEG, synth.RobotSpec(L=(0.1,) * 6, rc=0.005, umax=0.01, nb=5)])
def test_fk_parity(prec, spec):
    rng = np.random.default_rng(100)
    B = 3 * 128 + 37
    u = edge_states(spec, rng, B)
    rb = api.robot_struct(spec)
    ug = dev_soa(u, TDT[prec])
    T, bb = api.fk(rb, ug, backbone=True)
    torch.cuda.synchronize()
    ub = host_aos(ug)  # the values the GPU saw (rounded to FP32 where it applies)
    To, bbo = O.fk(orc_robot(spec), ub, backbone=True)
    Tg = host_aos(T)
    tol = TOL[prec]
    bbg = bb.double().cpu().numpy().transpose(2, 0, 1)
    eR = rowwise_rel(Tg[:, :9], To[:, :9], 1.0).max()
    ep = rowwise_rel(Tg[:, 9:], To[:, 9:], sum(spec.L)).max()
    eb = rowwise_rel(bbg.reshape(B, -1), bbo.reshape(B, -1), sum(spec.L)).max()
    print(f"FK n={spec.n} prec={prec}: R {eR:.2e}, p {ep:.2e}, backbone {eb:.2e} (tolerance {tol:.0e})")
    assert max(eR, ep, eb) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_tip_jacobian_parity(prec):
    spec = synth.ROBOT_3SEG
    rng = np.random.default_rng(101)
    B = 2 * 128 + 5
    u = edge_states(spec, rng, B)
    ug = dev_soa(u, TDT[prec])
    J = api.fk_jac(api.robot_struct(spec), ug)
    torch.cuda.synchronize()
    Jo = O.tip_jacobian(orc_robot(spec), host_aos(ug))
    Jg = J.double().cpu().numpy().transpose(2, 0, 1)
    tol = TOL[prec]
    ep = rowwise_rel(Jg[:, :3].reshape(B, -1), Jo[:, :3].reshape(B, -1)).max()
    ew = rowwise_rel(Jg[:, 3:].reshape(B, -1), Jo[:, 3:].reshape(B, -1)).max()
    print(f"J prec={prec}: translation rows {ep:.2e}, rotation rows {ew:.2e} (tolerance {tol:.0e})")
    assert max(ep, ew) <= tol


def _cost_case(spec, kind, rng, P, S, obstacles, thmax=None):
    """Targets from FK of random states, seeds near and far from them, spheres on backbones."""
    rb = orc_robot(spec, thmax)
    u_true = synth.hexagon_states(rng, P, spec.n, spec.umax)
    T, bb = O.fk(rb, u_true, backbone=True)
    tg = synth.pose_targets(T, "pose" if kind == lib.CR_TASK_IK6 else "axis")
    u = np.repeat(u_true, S, axis=0) + rng.normal(0, 3e-4, (P * S, spec.d))
    far = rng.random(P * S) < 0.5
    u[far] = synth.hexagon_states(rng, int(far.sum()), spec.n, spec.umax)
    u[::7] *= 1.3  # some bound violations
    spheres = None
    if obstacles:
        pick = bb[rng.integers(0, P, 12), rng.integers(0, spec.n * spec.nb, 12)]
        spheres = np.concatenate([pick + rng.normal(0, 2e-3, pick.shape), rng.uniform(3e-3, 8e-3, (12, 1))], 1)
    return rb, tg, u, spheres


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kind", [lib.CR_TASK_IK6, lib.CR_TASK_IK5])
@pytest.mark.parametrize("obstacles", [False, True])
def test_cost_grad_parity(prec, kind, obstacles):
    spec = synth.ROBOT_3SEG
    rng = np.random.default_rng(102 + kind + 2 * obstacles)
    P, S = 40, 8
    thmax = 1.3  # low enough that some states activate the curvature rows
    rbo, tg, u, spheres = _cost_case(spec, kind, rng, P, S, obstacles, thmax)
    spec_g = synth.RobotSpec(L=spec.L, rc=spec.rc, umax=spec.umax, nb=spec.nb, thmax=thmax)
    W = orc_weights()
    ug = dev_soa(u, TDT[prec])
    scene = api.Scene(spheres)
    tgd = targets_dev(tg)
    task = api.task_struct(kind, tgd, S, synth.WEIGHTS)
    cost, coll, gu, gp = api.cost_grad(api.robot_struct(spec_g), scene, task, ug, grad=True, param_grad=True, coll=True)
    gsum = api.reduce_rows(gp)
    torch.cuda.synchronize()
    ub = host_aos(ug)
    ref = O.ik_eval(rbo, W, spheres, kind, tg, S, ub, want=("F", "coll", "g", "r", "J"))
    rn = np.linalg.norm(ref["r"], axis=1)
    scale = pose_operand_scale(spec)
    tol = TOL[prec]
    if obstacles:
        assert (ref["coll"] > 0).sum() > 5
    if kind == lib.CR_TASK_IK6:  # the batch includes rotation errors near pi
        assert (np.linalg.norm(ref["r"][:, 3:6], axis=1) / synth.WEIGHTS.wR > math.pi - 0.05).sum() >= 2
    Fp, Fd = cost_errors(cost.double().cpu().numpy(), ref["F"], rn, scale)
    Cp, Cd = cost_errors(coll.double().cpu().numpy(), ref["coll"], rn, scale)
    gp_, gd = grad_errors(host_aos(gu), ref["g"], ref["J"], rn, scale)
    pg = O.ik_param_grad(rbo, W, spheres, kind, tg, S, ub)
    ep = np.abs(gsum.cpu().numpy() - pg).max() / np.abs(pg).max()
    print(f"cost kind={kind} obstacles={obstacles} prec={prec}: F plain {Fp.max():.2e} / data {Fd.max():.2e}; "
          f"clearance part data {Cd.max():.2e}; gradient plain {gp_.max():.2e} / data {gd.max():.2e}; "
          f"parameter gradient {ep:.2e} (tolerance {tol:.0e})")
    if prec == lib.CR_F64:
        assert Fp.max() <= tol and gp_.max() <= tol
    assert Fd.max() <= tol and Cd.max() <= tol and gd.max() <= tol
    assert ep <= tol


def test_cost_edge_cases():
    spec = synth.ROBOT_3SEG
    rb = api.robot_struct(spec)
    tg = np.zeros((2, 7))
    tg[:, 3] = 1.0
    tg[:, 2] = 0.30
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), 1, synth.WEIGHTS)
    u = np.zeros((2, 9))
    u[1, 0] = np.nan
    cost, _, gu, _ = api.cost_grad(rb, api.Scene(None), task, dev_soa(u, torch.float32))
    c = cost.cpu().numpy()
    assert c[0] == pytest.approx(0.0, abs=1e-12)  # straight robot exactly on the target
    assert np.isnan(c[1])
    # empty batch is a no-op
    e = torch.empty((9, 0), dtype=torch.float32, device="cuda")
    api.cost_grad(rb, api.Scene(None), task, e)
