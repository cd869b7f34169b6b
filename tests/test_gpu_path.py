"""GPU parity of path following (exploration sweep + joint LM with the FP64 block-tridiagonal
Cholesky) against the FP64 oracle (dense Cholesky of the whole normal matrix)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import EPS, consequential_ties, kink_or_pi, orc_robot, orc_weights, pose_operand_scale
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _case(spec, P, H, n_spheres, seed):
    rbo = orc_robot(spec)
    wp, states, sph = synth.path_workload(spec, P, H, n_spheres, lambda u: O.fk(rbo, u, backbone=True), seed=seed)
    return rbo, wp, states, sph


def _gpu(spec, ik, wp, sph, prec, k_warm, k_joint, p0=0):
    P, H, _ = wp.shape
    s = api.PathSolver(spec, ik, synth.WEIGHTS, P, H, api.Scene(sph, per_problem=True), prec, k_warm, k_joint)
    s.solve(api.waypoints_soa(wp), p0)
    torch.cuda.synchronize()
    d = spec.d
    return dict(x=s.X.cpu().numpy().T.reshape(P, H, d), F=s.cost.cpu().numpy(), pos=s.pos.cpu().numpy().reshape(P, H),
                rot=s.rot.cpu().numpy().reshape(P, H), lim_ok=s.lim_ok.cpu().numpy().astype(bool),
                col_ok=s.col_ok.cpu().numpy().astype(bool))


def _cfg(ik, p0=0):
    return O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                      alpha0=ik.alpha0, p0=p0)


def test_path_fp64_parity():
    """FP64 path following against the oracle (dense Cholesky of the whole normal matrix) on 16 paths
    of 8 waypoints: states, cost, errors and flags within 1e-9 for every path whose warm sweep and
    joint LM take no consequential decision at the rounding level: (a) the oracle's own start / trial
    costs of an iteration within the FP64 band while the step at stake can exceed 1e-9
    (gpu_util.consequential_ties); (b) a warm start, the joint stage's start or its end on a bound or
    curvature hinge's kink to within the FP64 band (gpu_util.kink_or_pi: a waypoint whose target
    needs a tendon past u_max converges onto the bound, where one side may take the bound row as
    active and the other not, and with two redundant degrees of freedom the next waypoint's warm LM
    then settles on a different point of its solution set). After such a decision the two may
    continue on different branches."""
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=6)
    ik = synth.IkSpec(S=32, n_final=4, k_init=16, k_final=20)
    P = 16
    rbo, wp, states, sph = _case(spec, P, 8, 6, seed=70)
    g = _gpu(spec, ik, wp, sph, lib.CR_F64, 10, 8)
    o = O.solve_path(rbo, orc_weights(), sph, wp, _cfg(ik), 10, 8, trace=True)
    tie = consequential_ties(o["trace"][..., 0], o["trace"][..., 1], EPS[lib.CR_F64], pose_operand_scale(spec),
                             1e-9).any(axis=1)
    tie |= kink_or_pi(np.concatenate([o["stage_x"], o["x"]], axis=1), spec, None, lib.CR_F64).any(axis=1)
    ok = ~tie
    dx = np.abs(g["x"] - o["x"]).max(axis=(1, 2))
    print(f"FP64 paths: {int(ok.sum())} of {P} without a rounding-level decision; state error on those "
          f"{dx[ok].max():.2e}, on the others {dx[~ok].max() if tie.any() else 0:.2e}")
    assert ok.sum() >= P // 2
    np.testing.assert_allclose(g["x"][ok], o["x"][ok], atol=1e-9)
    np.testing.assert_allclose(g["F"][ok], o["F"][ok], rtol=1e-6, atol=1e-18)
    np.testing.assert_allclose(g["pos"][ok], o["pos"][ok], atol=1e-9)
    assert np.array_equal(g["lim_ok"][ok], o["lim_ok"][ok]) and np.array_equal(g["col_ok"][ok], o["col_ok"][ok])


def _check_valid(spec, rbo, wp, sph, g):
    """The GPU's reported per-waypoint errors and flags equal the oracle's FP64 evaluation of the
    GPU's own states."""
    P, H, _ = wp.shape
    for p in range(P):
        pos, rot, lim, col = O.accept(rbo, sph[p], 0, wp[p], g["x"][p])
        np.testing.assert_allclose(g["pos"][p], pos, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(g["rot"][p], rot, rtol=1e-9, atol=1e-12)
        assert g["lim_ok"][p] == lim.all() and g["col_ok"][p] == col.all()


def test_path_fp32_parity():
    """FP32 bulk on a ragged warp of paths: every GPU result is valid under the oracle's FP64
    evaluation of the GPU's own states (the success rate against the oracle's own solves is
    compared on 200 paths in tests/test_gpu_success_parity.py)."""
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=64, n_final=8, k_init=32, k_final=30)
    rbo, wp, states, sph = _case(spec, 12, 16, 8, seed=71)
    g = _gpu(spec, ik, wp, sph, lib.CR_F32, synth.K_WARM, synth.K_JOINT)
    _check_valid(spec, rbo, wp, sph, g)


def test_path_full_size_sampled():
    """512 paths of 64 waypoints with 32 spheres each (FP32 bulk, FP64 block Cholesky) in the
    launch configuration of the benchmark: validity of a 16-path sample under the oracle's FP64
    evaluation of the GPU's states (success against the oracle's own solves: 200 paths of 16
    waypoints in tests/test_gpu_success_parity.py)."""
    spec, ik = synth.ROBOT_4SEG, synth.IK_PATH0
    P, H = synth.P_PATH, synth.H_PATH
    rbo, wp, states, sph = _case(spec, P, H, synth.NO_PATH, seed=0)
    g = _gpu(spec, ik, wp, sph, lib.CR_F32, synth.K_WARM, synth.K_JOINT)
    assert np.isfinite(g["F"]).all()
    sel = list(range(16))
    sub = {k: v[sel] for k, v in g.items()}
    _check_valid(spec, rbo, wp[sel], sph[sel], sub)
    rate_g = (g["pos"].max(axis=1) <= 1e-3).mean()
    print(f"full-size paths: {rate_g:.3f} tracked within 1 mm at every waypoint")
    assert rate_g > 0.5
