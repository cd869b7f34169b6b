"""GPU parity of the kinematics, Jacobian, cost and adjoint entry points against the FP64 oracle.

Tolerances: FP64 1e-12 and FP32 1e-5, relative, norm-wise per state and per quantity (the largest
component of that quantity sets the scale). Batches span several 128-thread blocks plus a ragged
tail, and include the straight and nearly-straight configurations and states on the bounds.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import TDT, TOL, dev_soa, edge_states, host_aos, orc_robot, orc_weights, rowwise_rel, targets_dev
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
    assert rowwise_rel(Tg[:, :9], To[:, :9], 1.0).max() <= tol * 10
    assert rowwise_rel(Tg[:, 9:], To[:, 9:], sum(spec.L)).max() <= tol * 10
    bbg = bb.double().cpu().numpy().transpose(2, 0, 1)
    assert rowwise_rel(bbg.reshape(B, -1), bbo.reshape(B, -1), sum(spec.L)).max() <= tol * 10


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
    tol = TOL[prec] * 10
    assert rowwise_rel(Jg[:, :3].reshape(B, -1), Jo[:, :3].reshape(B, -1)).max() <= tol
    assert rowwise_rel(Jg[:, 3:].reshape(B, -1), Jo[:, 3:].reshape(B, -1)).max() <= tol


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
    ref = O.ik_eval(rbo, W, spheres, kind, tg, S, ub, want=("F", "coll", "g"))
    # rotation error near pi makes the FP32 log ill-conditioned; those states are compared in FP64 only
    E = O.ik_eval(rbo, W, None, kind, tg, S, ub, want=("r",))["r"][:, 3:6]
    ok = np.linalg.norm(E, axis=1) < math.pi - 0.05 if prec == lib.CR_F32 else np.ones(len(u), bool)
    tol = TOL[prec]
    Fg = cost.double().cpu().numpy()
    assert (np.abs(Fg - ref["F"]) / np.maximum(ref["F"], 1e-30))[ok].max() <= tol * 10
    Cg = coll.double().cpu().numpy()
    if obstacles:
        assert (ref["coll"] > 0).sum() > 5
    assert (np.abs(Cg - ref["coll"]) / np.maximum(ref["F"], 1e-30))[ok].max() <= tol * 10
    assert rowwise_rel(host_aos(gu)[ok], ref["g"][ok]).max() <= tol * 100
    pg = O.ik_param_grad(rbo, W, spheres, kind, tg, S, ub)
    if ok.all():
        np.testing.assert_allclose(gsum.cpu().numpy(), pg, rtol=tol * 100, atol=tol * 100 * np.abs(pg).max())


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
