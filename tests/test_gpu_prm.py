"""GPU parity of the PRM exploration (Algorithm 2) against the oracle: the roadmap (nodes, validity,
nearest-neighbour lists, the graph in CSR form with its weights) and the queries (path length, hop
count, resampled states) compare exactly, because every decision is taken in FP64 on both sides from
identically rounded operands; the trajectory solve with the PRM initialiser compares like the
linear-initialiser solve."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_11340_gb300 import api, lib, synth

from gpu_util import dev_soa, orc_robot, orc_weights

pytestmark = pytest.mark.gpu

DELTA = synth.WEIGHTS.delta


def _case(P, n_spheres, seed, spec=synth.ROBOT_3SEG):
    rbo = orc_robot(spec)
    us, goal, sph, ug = synth.traj_workload(spec, P, n_spheres, lambda u: O.fk(rbo, u, backbone=True), seed=seed)
    return spec, rbo, us, goal, sph, ug


def _oracle_map(rbo, sph_r, spec, r):
    return O.prm_build(rbo, DELTA, sph_r, spec.seed, r, spec.N, spec.k, spec.n_check, spec.attempts)


def _check_graph(rm, ref):
    np.testing.assert_array_equal(rm["ok"], ref["ok"])
    np.testing.assert_array_equal(rm["nodes"], ref["nodes"])
    np.testing.assert_array_equal(rm["nbr"], ref["nbr"])
    np.testing.assert_array_equal(rm["row"], ref["row"])
    np.testing.assert_array_equal(rm["col"], ref["col"])
    np.testing.assert_array_equal(rm["wt"], ref["wt"])


@pytest.mark.parametrize("N,k,nc,n_spheres", [(96, 6, 4, 24), (200, 7, 5, 40), (37, 1, 1, 0)])
def test_prm_build_matches_oracle(N, k, nc, n_spheres):
    """Per-problem scenes (one roadmap each): N not a multiple of 32 or of the 128-thread blocks,
    k up to N - 1 edge cases, no obstacles."""
    P = 3
    robot, rbo, us, goal, sph, ug = _case(P, n_spheres, seed=70 + N)
    ps = synth.PrmSpec(N=N, k=k, n_check=nc, attempts=8, seed=0x5052_0001)
    scene = api.Scene(sph, per_problem=True)
    rm = api.Roadmap(robot, ps, P).build(scene, synth.WEIGHTS)
    torch.cuda.synchronize()
    for r in range(P):
        _check_graph(rm.graph(r), _oracle_map(rbo, None if sph is None else sph[r], ps, r))
    assert rm.node_ok.cpu().numpy().any()


def test_prm_build_maximum_sizes():
    """N = 1024 nodes and k = 32 neighbours on one shared scene, and two queries on it."""
    robot, rbo, us, goal, sph, ug = _case(2, 16, seed=80)
    ps = synth.PrmSpec(N=1024, k=32, n_check=2, attempts=8, seed=0x5052_0002)
    scene = api.Scene(sph[0])
    rm = api.Roadmap(robot, ps, 1).build(scene, synth.WEIGHTS)
    torch.cuda.synchronize()
    ref = _oracle_map(rbo, sph[0], ps, 0)
    _check_graph(rm.graph(0), ref)
    X, length, hops = rm.query(scene, synth.WEIGHTS, dev_soa(us, torch.float64), dev_soa(ug, torch.float64), 33)
    torch.cuda.synchronize()
    X = X.cpu().numpy().T.reshape(2, 33, -1)
    for p in range(2):
        Xr, Lr, Hr, _ = O.prm_query(rbo, DELTA, sph[0], ref, ps.k, ps.n_check, us[p], ug[p], 33)
        assert hops[p].item() == Hr and length[p].item() == Lr
        np.testing.assert_array_equal(X[p], Xr)


@pytest.mark.parametrize("shared", [False, True])
def test_prm_query_matches_oracle(shared):
    """Queries on per-problem roadmaps (R = P) and on one shared roadmap (R = 1), T = 17 and 2."""
    P = 4
    robot, rbo, us, goal, sph, ug = _case(P, 24, seed=90 + shared)
    ps = synth.PrmSpec(N=128, k=6, n_check=4, attempts=8, seed=0x5052_0003)
    if shared:
        sph = np.repeat(sph[:1], P, axis=0)
        scene = api.Scene(sph[0])
        R = 1
    else:
        scene = api.Scene(sph, per_problem=True)
        R = P
    rm = api.Roadmap(robot, ps, R).build(scene, synth.WEIGHTS)
    refs = [_oracle_map(rbo, sph[r], ps, r) for r in range(R)]
    found = 0
    for T in (17, 2):
        X, length, hops = rm.query(scene, synth.WEIGHTS, dev_soa(us, torch.float64), dev_soa(ug, torch.float64), T)
        torch.cuda.synchronize()
        X = X.cpu().numpy().T.reshape(P, T, -1)
        for p in range(P):
            Xr, Lr, Hr, _ = O.prm_query(rbo, DELTA, sph[p], refs[0 if shared else p], ps.k, ps.n_check, us[p], ug[p],
                                        T)
            assert hops[p].item() == Hr
            assert length[p].item() == Lr
            np.testing.assert_array_equal(X[p], Xr)
            found += Hr > 0
    assert found > 0


def test_prm_query_degenerate_scene():
    """Every draw collides: no valid node, no path, the linear initialiser (hops 0, length inf)."""
    P = 2
    robot, rbo, us, goal, _, ug = _case(P, 0, seed=95)
    sph = np.array([[0.0, 0.0, 0.0, 1.0]])
    ps = synth.PrmSpec(N=40, k=3, n_check=2, attempts=2, seed=0x5052_0004)
    scene = api.Scene(sph)
    rm = api.Roadmap(robot, ps, 1).build(scene, synth.WEIGHTS)
    X, length, hops = rm.query(scene, synth.WEIGHTS, dev_soa(us, torch.float64), dev_soa(ug, torch.float64), 9)
    torch.cuda.synchronize()
    assert not rm.node_ok.cpu().numpy().any()
    assert int(rm.row[0, -1].item()) == 0
    assert np.all(hops.cpu().numpy() == 0) and np.all(np.isinf(length.cpu().numpy()))
    X = X.cpu().numpy().T.reshape(P, 9, -1)
    ref = _oracle_map(rbo, sph, ps, 0)
    for p in range(P):
        Xr, Lr, Hr, _ = O.prm_query(rbo, DELTA, sph, ref, ps.k, ps.n_check, us[p], ug[p], 9)
        assert Hr == 0
        np.testing.assert_array_equal(X[p], Xr)


def test_fp32_backbone_error_far_below_the_filter_margin():
    """The FP32 pass of the collision decision relies on the FP32 backbone error staying far below
    its margin 1e-5 (sum L + reach + |c|_1) >= 1e-5 sum L: measured on hexagon-uniform states."""
    spec = synth.ROBOT_3SEG
    rbo = orc_robot(spec)
    rng = np.random.default_rng(3)
    u = synth.hexagon_states(rng, 4096, spec.n, spec.umax)
    _, bb_ref = O.fk(rbo, u, backbone=True)
    robot = api.robot_struct(spec)
    _, bb = api.fk(robot, torch.as_tensor(u.T.copy(), dtype=torch.float32, device="cuda").contiguous(), backbone=True)
    bb = bb.double().cpu().numpy()
    bb = np.moveaxis(bb, -1, 0).reshape(len(u), -1, 3)
    err = np.abs(bb - bb_ref).max()
    assert err < 0.2 * 1e-5 * sum(spec.L), f"FP32 backbone error {err:.3e} m"


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_solve_traj_prm_parity(prec):
    """Goal IK, PRM query on per-problem roadmaps, 100 projected-gradient steps: FP64 iterates agree
    with the oracle's composition of the same stages; FP32 results are valid under the oracle's own
    evaluation of the GPU's states."""
    P, Tn = 3, synth.T_TRAJ
    robot, rbo, us, goal, sph, _ = _case(P, synth.NO_TRAJ, seed=66)
    ps = synth.PrmSpec(N=128, k=6, n_check=4, attempts=8, seed=0x5052_0005)
    scene = api.Scene(sph, per_problem=True)
    rm = api.Roadmap(robot, ps, P).build(scene, synth.WEIGHTS)
    ik = synth.IK_GOAL
    sol = api.TrajSolver(robot, ik, synth.WEIGHTS, P, Tn, scene, precision=prec, roadmap=rm)
    sol.solve(dev_soa(us, torch.float64), dev_soa(goal, torch.float64))
    torch.cuda.synchronize()
    X = sol.X.cpu().numpy().T.reshape(P, Tn, -1)
    W = orc_weights()
    if prec == lib.CR_F64:
        X0 = np.zeros_like(X)
        hops = []
        for p in range(P):
            cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, p0=p)
            ugp = O.solve_ik(rbo, W, sph[p], O.IK6, goal[p:p + 1], cfg)["u"][0]
            ref_map = _oracle_map(rbo, sph[p], ps, p)
            X0[p], _, h, _ = O.prm_query(rbo, DELTA, sph[p], ref_map, ps.k, ps.n_check, us[p], ugp, Tn)
            hops.append(h)
        assert list(sol.hops.cpu().numpy()) == hops
        ref = O.traj_refine(rbo, W, sph, us, goal, X0, synth.K_TRAJ, synth.ALPHA_TRAJ)
        # iterates within 1e-4 of the state scale (the iterate tolerance of the method's parity
        # bar): roadmap paths run close to obstacles, where a clearance hinge at its kink makes a
        # state sensitive to rounding at the 1e-8 m level over 100 steps
        for p in range(P):
            assert np.abs(X[p] - ref["x"][p]).max() <= 1e-4 * np.abs(ref["x"][p]).max()
        np.testing.assert_allclose(sol.cost.cpu().numpy(), ref["F"], rtol=1e-4)
        for k in ("lim_ok", "col_ok"):
            assert np.array_equal(getattr(sol, k).cpu().numpy().astype(bool), ref[k])
    else:
        for p in range(P):
            F = O.traj_eval(rbo, W, sph[p:p + 1], us[p:p + 1], goal[p:p + 1], X[p:p + 1, 1:])["F"]
            np.testing.assert_allclose(sol.cost.cpu().numpy()[p], F[0], rtol=1e-3)
            _, _, lim, col = O.accept(rbo, sph[p], lib.CR_TASK_IK6, np.repeat(goal[p:p + 1], Tn, 0), X[p])
            assert bool(sol.col_ok[p].item()) == bool(col.all())
        assert np.all(sol.hops.cpu().numpy() >= 0)


@pytest.mark.parametrize("n,N,k,nc,T", [(1, 64, 5, 3, 9), (2, 2, 1, 2, 5), (4, 80, 6, 3, 256), (6, 64, 5, 2, 17)])
def test_prm_other_segment_counts(n, N, k, nc, T):
    """Roadmaps and queries of 1, 2, 4 and 6-segment robots (each a separate kernel instantiation),
    the smallest roadmap (N = 2, k = 1) and the longest horizon (T = 256), against the oracle."""
    spec = synth.RobotSpec(L=(0.1,) * n, rc=0.005, umax=0.01, nb=8)
    P = 2
    robot, rbo, us, goal, sph, ug = _case(P, 16, seed=100 + n, spec=spec)
    ps = synth.PrmSpec(N=N, k=k, n_check=nc, attempts=8, seed=0x5052_0006)
    scene = api.Scene(sph, per_problem=True)
    rm = api.Roadmap(robot, ps, P).build(scene, synth.WEIGHTS)
    X, length, hops = rm.query(scene, synth.WEIGHTS, dev_soa(us, torch.float64), dev_soa(ug, torch.float64), T)
    torch.cuda.synchronize()
    X = X.cpu().numpy().T.reshape(P, T, -1)
    for p in range(P):
        ref = _oracle_map(rbo, sph[p], ps, p)
        _check_graph(rm.graph(p), ref)
        Xr, Lr, Hr, _ = O.prm_query(rbo, DELTA, sph[p], ref, ps.k, ps.n_check, us[p], ug[p], T)
        assert hops[p].item() == Hr and length[p].item() == Lr
        np.testing.assert_array_equal(X[p], Xr)
