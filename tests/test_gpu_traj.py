"""GPU parity of trajectory planning (cost, hand-written adjoint, projected-gradient solve),
kinematic calibration and the autograd Functions, against the FP64 oracle and finite differences."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import TDT, TOL, dev_soa, host_aos, orc_robot, orc_weights, rowwise_rel, targets_dev
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


SPEC = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=6)


def _traj_case(P=3, Tn=8, n_spheres=5, seed=60, weights=synth.WEIGHTS):
    rbo = orc_robot(SPEC)
    us, goal, sph, ug = synth.traj_workload(SPEC, P, n_spheres, lambda u: O.fk(rbo, u, backbone=True), seed=seed)
    rng = np.random.default_rng(seed)
    s = np.linspace(0, 1, Tn)[1:, None]
    x = us[:, None, :] + s[None] * (ug - us)[:, None, :] + rng.normal(0, 4e-4, (P, Tn - 1, SPEC.d))
    return rbo, us, goal, sph, x


def _gpu_traj(us, goal, sph, Tn, weights):
    scene = api.Scene(sph, per_problem=True)
    task = api.traj_task_struct(dev_soa(us, torch.float64), dev_soa(goal, torch.float64), Tn, weights)
    return api.robot_struct(SPEC), scene, task


def _x_dev(x, dtype):
    P, Tm1, d = x.shape
    return torch.as_tensor(x.reshape(P * Tm1, d).T.copy(), dtype=dtype).cuda()


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_traj_cost_and_adjoint_parity(prec):
    W = synth.WeightSpec(vmax=0.01, amax=0.05, rho_c=1e3)  # speed / acceleration hinges active
    Tn = 8
    rbo, us, goal, sph, x = _traj_case(Tn=Tn)
    robot, scene, task = _gpu_traj(us, goal, sph, Tn, W)
    xg = _x_dev(x, TDT[prec])
    cost = torch.empty(len(us), dtype=TDT[prec], device="cuda")
    grad = torch.empty_like(xg)
    lib.cr_traj_cost(robot, scene.c, task, xg, cost, grad)
    torch.cuda.synchronize()
    xb = xg.double().cpu().numpy().T.reshape(x.shape)
    ref = O.traj_eval(rbo, O.make_weights(**W.as_dict()), sph, us, goal, xb, want=("F", "g"))
    tol = TOL[prec]
    g = grad.double().cpu().numpy().T.reshape(x.shape)
    eF = (np.abs(cost.double().cpu().numpy() - ref["F"]) / ref["F"]).max()
    eg = rowwise_rel(g.reshape(len(us), -1), ref["g"].reshape(len(us), -1)).max()
    print(f"trajectory cost prec={prec}: F {eF:.2e}, gradient {eg:.2e} (tolerance {tol:.0e})")
    assert eF <= tol and eg <= tol


def test_traj_gradient_vs_central_differences_fp64():
    W = synth.WeightSpec(vmax=0.01, amax=0.05, rho_c=1e3)
    Tn = 6
    rbo, us, goal, sph, x = _traj_case(P=2, Tn=Tn, seed=61)
    robot, scene, task = _gpu_traj(us, goal, sph, Tn, W)
    xg = _x_dev(x, torch.float64)
    cost = torch.empty(2, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(xg)
    lib.cr_traj_cost(robot, scene.c, task, xg, cost, grad)
    h = 1e-6
    fd = torch.empty_like(xg)
    for q in range(xg.shape[0]):
        for c in range(xg.shape[1]):
            xp, xm = xg.clone(), xg.clone()
            xp[q, c] += h
            xm[q, c] -= h
            cp, cm = torch.empty_like(cost), torch.empty_like(cost)
            lib.cr_traj_cost(robot, scene.c, task, xp, cp)
            lib.cr_traj_cost(robot, scene.c, task, xm, cm)
            fd[q, c] = ((cp - cm) / (2 * h)).sum()
    torch.cuda.synchronize()
    g, f = grad.cpu().numpy(), fd.cpu().numpy()
    np.testing.assert_allclose(g, f, rtol=2e-5, atol=1e-6 * np.abs(g).max())


def test_autograd_functions_gradcheck():
    # trajectory cost
    W = synth.WeightSpec(vmax=0.01, amax=0.05, rho_c=1e3)
    Tn = 5
    rbo, us, goal, sph, x = _traj_case(P=2, Tn=Tn, n_spheres=3, seed=62)
    data = _gpu_traj(us, goal, sph, Tn, W)
    xg = _x_dev(x, torch.float64).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda xx: api.TrajCost.apply(xx, data), (xg,), eps=1e-7, atol=1e-6, rtol=1e-5)
    # IK cost w.r.t. states and the kinematic parameters (segment lengths, tendon radii)
    spec = synth.RobotSpec(L=(0.12, 0.10), rc=0.005, umax=0.01, nb=4)
    rb2 = orc_robot(spec)
    rng = np.random.default_rng(63)
    ut = synth.hexagon_states(rng, 3, 2, spec.umax)
    tg = synth.pose_targets(O.fk(rb2, ut)[0], "pose")
    tgd = targets_dev(tg)
    sph2 = np.array([[0.0, 0.02, 0.15, 0.01]])
    scene = api.Scene(sph2)
    task = api.task_struct(lib.CR_TASK_IK6, tgd, 2, synth.WEIGHTS)
    u = torch.as_tensor((np.repeat(ut, 2, 0) + rng.normal(0, 1e-3, (6, 6))).T.copy(), dtype=torch.float64).cuda()
    u.requires_grad_(True)
    L = torch.tensor(spec.L, dtype=torch.float64, requires_grad=True)
    rc = torch.full((2,), spec.rc, dtype=torch.float64, requires_grad=True)
    f = lambda uu, LL, rr: api.IkCost.apply(uu, LL, rr, (spec, scene, task))
    assert torch.autograd.gradcheck(f, (u, L, rc), eps=1e-7, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_solve_traj_parity(prec):
    """Goal IK + linear initialisation + 100 projected-gradient steps on 2 problems of 32 states."""
    spec = synth.ROBOT_3SEG
    rbo = orc_robot(spec)
    P, Tn = 2, synth.T_TRAJ
    us, goal, sph, _ = synth.traj_workload(spec, P, synth.NO_TRAJ, lambda u: O.fk(rbo, u, backbone=True), seed=64)
    ik = synth.IK_GOAL
    scene = api.Scene(sph, per_problem=True)
    sol = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, scene, precision=prec)
    sol.solve(dev_soa(us, torch.float64), dev_soa(goal, torch.float64))
    torch.cuda.synchronize()
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final)
    ref = O.solve_traj(rbo, orc_weights(), sph, us, goal, Tn, cfg, synth.K_TRAJ, synth.ALPHA_TRAJ)
    X = sol.X.cpu().numpy().T.reshape(P, Tn, -1)
    for k in ("lim_ok", "col_ok"):
        assert np.array_equal(getattr(sol, k).cpu().numpy().astype(bool), ref[k])
    if prec == lib.CR_F64:
        # 100 normalised steps: near convergence the step direction g / |g| of a small gradient carries
        # the rounding of g relative to |g|, so FP64 states drift apart by up to alpha times that
        # (measured 6.5e-9 m and 1.1e-8 m, about 1e-6 of the bound, on two builds whose gradients round
        # differently); the bound is 1e-7 m, 1e-5 of the displacement bound
        np.testing.assert_allclose(X, ref["x"], atol=1e-7)
        # with |dF/du| ~ F / 1e-3 m, states within 1e-7 m allow 1e-4 relative in F
        np.testing.assert_allclose(sol.cost.cpu().numpy(), ref["F"], rtol=1e-4)
    else:
        np.testing.assert_allclose(sol.cost.cpu().numpy(), ref["F"], rtol=0.05)
        assert np.all(sol.goal_pos.cpu().numpy() < 1e-3) == np.all(ref["goal_pos"] < 1e-3)


@pytest.mark.parametrize("n_spheres", [1, 5, 9])
def test_solve_traj_fp32_split_edges(n_spheres):
    """FP32 trajectory solve with 20 states (a ragged warp) and an odd number of spheres (two
    threads per state take 3 and 2, or 5 and 4, of them) or a single sphere (no split): the result
    is valid under the oracle's own evaluation of the GPU's states and its cost is close to the
    oracle's."""
    spec = synth.ROBOT_3SEG
    rbo = orc_robot(spec)
    P, Tn = 4, 20
    us, goal, sph, _ = synth.traj_workload(spec, P, n_spheres, lambda u: O.fk(rbo, u, backbone=True), seed=65)
    ik = synth.IK_GOAL
    sol = api.TrajSolver(spec, ik, synth.WEIGHTS, P, Tn, api.Scene(sph, per_problem=True), precision=lib.CR_F32)
    sol.solve(dev_soa(us, torch.float64), dev_soa(goal, torch.float64))
    torch.cuda.synchronize()
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final)
    ref = O.solve_traj(rbo, orc_weights(), sph, us, goal, Tn, cfg, synth.K_TRAJ, synth.ALPHA_TRAJ)
    X = sol.X.cpu().numpy().T.reshape(P, Tn, -1)
    for p in range(P):
        F = O.traj_eval(rbo, orc_weights(), sph[p:p + 1], us[p:p + 1], goal[p:p + 1], X[p:p + 1, 1:])["F"]
        np.testing.assert_allclose(sol.cost.cpu().numpy()[p], F[0], rtol=1e-3)
    np.testing.assert_allclose(sol.cost.cpu().numpy(), ref["F"], rtol=0.05)
    for p in range(P):  # the FP64 flags of the GPU's own states, state by state
        _, _, lim, col = O.accept(rbo, sph[p], lib.CR_TASK_IK6, np.repeat(goal[p:p + 1], Tn, 0), X[p])
        assert bool(sol.col_ok[p].item()) == bool(col.all())


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_calibration_parity_full_size(prec):
    spec = synth.ROBOT_3SEG

    def fkp(U, L, rc):
        return O.fk(O.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    U, Pm, true, nom = synth.calib_workload(spec, synth.K_CALIB, fkp, seed=0)
    ref = O.calibrate(orc_robot(spec), U, Pm, nom, synth.ITERS_CALIB)
    th, F, _ = api.calibrate(spec, dev_soa(U, TDT[prec]), dev_soa(Pm, torch.float64), nom)
    th = th.cpu().numpy()
    if prec == lib.CR_F64:
        np.testing.assert_allclose(th, ref["theta"], rtol=1e-10)
        np.testing.assert_allclose(F.item(), ref["F"], rtol=1e-9)
    else:
        # FP32 residuals (|r| ~ 0.5 mm out of 0.3 m) change the estimate by far less than the noise
        np.testing.assert_allclose(th, ref["theta"], rtol=2e-4)
    assert np.abs(th / true - 1).max() < 5e-3


def test_calibration_iterates_partial_block():
    """K = 300 poses (two full blocks of 128 and a partial one) on a 2-segment robot, FP64: every LM
    iterate against the oracle's, and an undersized workspace is refused."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01)

    def fkp(U, L, rc):
        return O.fk(O.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    U, Pm, true, nom = synth.calib_workload(spec, 300, fkp, seed=5)
    ref = O.calibrate(orc_robot(spec), U, Pm, nom, 12, history=True)
    th, F, hist = api.calibrate(spec, dev_soa(U, torch.float64), dev_soa(Pm, torch.float64), nom, iters=12,
                                history=True)
    np.testing.assert_allclose(hist.cpu().numpy(), ref["hist"], rtol=1e-10)
    np.testing.assert_allclose(th.cpu().numpy(), ref["theta"], rtol=1e-10)
    np.testing.assert_allclose(F.item(), ref["F"], rtol=1e-9)
    robot = api.robot_struct(spec)
    Ud, Pd = dev_soa(U, torch.float64), dev_soa(Pm, torch.float64)
    small = torch.empty(lib.cr_calibrate_workspace_size(robot, 300) - 8, dtype=torch.uint8, device="cuda")
    th2 = torch.as_tensor(nom, dtype=torch.float64, device="cuda").clone()
    F2 = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        lib.cr_calibrate(robot, Ud, Pd, th2, 3, 1e-3, F2, None, small)



@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_sharded_calibration_pieces(prec):
    """The sharded calibration's library pieces on one GPU: without a process group they reproduce
    cr_calibrate bit for bit (same partial sums, order, factorisation and rule); with the 1024 poses
    split into three shards whose partial sums are added in between (what the all-reduce does across
    processes) the estimate equals the one-shard one to the rounding of the summation order."""
    spec = synth.ROBOT_3SEG

    def fkp(U, L, rc):
        return O.fk(O.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    U, Pm, true, nom = synth.calib_workload(spec, synth.K_CALIB, fkp, seed=0)
    Ud, Pd = dev_soa(U, TDT[prec]), dev_soa(Pm, torch.float64)
    th_ref, _, _ = api.calibrate(spec, Ud, Pd, nom)
    th1 = api.calibrate_sharded(spec, Ud, Pd, nom)
    assert torch.equal(th1, th_ref)

    class Shards:  # three shards in one process: their sums added as an all-reduce would
        def __init__(self):
            cuts = [0, 300, 700, U.shape[0]]
            self.parts = [api.CalibShard(spec, Ud[:, a:b].contiguous(), Pd[:, a:b].contiguous())
                          for a, b in zip(cuts, cuts[1:])]

        def sums(self, theta):
            return sum(p.sums(theta) for p in self.parts)

        def trial(self, sums, theta, state):
            return self.parts[0].trial(sums, theta, state)

        def cost(self, theta_trial):
            return sum(p.cost(theta_trial) for p in self.parts)

        def accept(self, sums, F_trial, theta_trial, theta, state):
            self.parts[0].accept(sums, F_trial, theta_trial, theta, state)

    theta = torch.as_tensor(nom, dtype=torch.float64, device="cuda").clone()
    state = torch.tensor([1e-3, 2.0, 0.0, 0.0], dtype=torch.float64, device="cuda")
    api.calibrate_lm_sharded(Shards(), theta, state, synth.ITERS_CALIB, lambda t: None)
    err = (theta / th_ref - 1).abs().max().item()
    print(f"sharded calibration prec={prec}: three shards vs one, max relative parameter difference {err:.2e}")
    assert err <= (1e-10 if prec == lib.CR_F64 else 1e-6)
