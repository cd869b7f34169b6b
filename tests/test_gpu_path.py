"""GPU parity of path following (exploration sweep + joint LM with the FP64 block-tridiagonal
Cholesky) against the FP64 oracle (dense Cholesky of the whole normal matrix)."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import orc_robot, orc_weights
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
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=6)
    ik = synth.IkSpec(S=32, n_final=4, k_init=16, k_final=20)
    rbo, wp, states, sph = _case(spec, 3, 8, 6, seed=70)
    g = _gpu(spec, ik, wp, sph, lib.CR_F64, 10, 8)
    o = O.solve_path(rbo, orc_weights(), sph, wp, _cfg(ik), 10, 8)
    np.testing.assert_allclose(g["x"], o["x"], atol=1e-9)
    np.testing.assert_allclose(g["F"], o["F"], rtol=1e-6, atol=1e-18)
    np.testing.assert_allclose(g["pos"], o["pos"], atol=1e-9)
    assert np.array_equal(g["lim_ok"], o["lim_ok"]) and np.array_equal(g["col_ok"], o["col_ok"])


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
    """FP32 bulk: the 4-segment robot is redundant (8 free DoF for a 6-DoF pose), so FP32 and FP64
    may settle on different, equally valid solution branches; what is unique is checked instead:
    the validity of every GPU result under the oracle and the tracking rate on the same paths."""
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=64, n_final=8, k_init=32, k_final=30)
    rbo, wp, states, sph = _case(spec, 12, 16, 8, seed=71)
    g = _gpu(spec, ik, wp, sph, lib.CR_F32, synth.K_WARM, synth.K_JOINT)
    _check_valid(spec, rbo, wp, sph, g)
    o = O.solve_path(rbo, orc_weights(), sph, wp, _cfg(ik), synth.K_WARM, synth.K_JOINT)
    rate_g = (g["pos"].max(axis=1) <= 1e-3).mean()
    rate_o = (o["pos"].max(axis=1) <= 1e-3).mean()
    assert abs(rate_g - rate_o) <= 3 / 12


def test_path_full_size_sampled():
    """512 paths of 64 waypoints with 32 spheres each (FP32 bulk, FP64 block Cholesky); validity of
    a sample under the oracle, and the tracking rate against the oracle on 16 of the same paths."""
    spec, ik = synth.ROBOT_4SEG, synth.IK_PATH0
    P, H = synth.P_PATH, synth.H_PATH
    rbo, wp, states, sph = _case(spec, P, H, synth.NO_PATH, seed=0)
    g = _gpu(spec, ik, wp, sph, lib.CR_F32, synth.K_WARM, synth.K_JOINT)
    assert np.isfinite(g["F"]).all()
    sel = list(range(16))
    sub = {k: v[sel] for k, v in g.items()}
    _check_valid(spec, rbo, wp[sel], sph[sel], sub)
    o = O.solve_path(rbo, orc_weights(), sph[sel], wp[sel], _cfg(ik, 0), synth.K_WARM, synth.K_JOINT)
    rate_o = (o["pos"].max(axis=1) <= 1e-3).mean()
    rate_g16 = (sub["pos"].max(axis=1) <= 1e-3).mean()
    rate_g = (g["pos"].max(axis=1) <= 1e-3).mean()
    assert abs(rate_g16 - rate_o) <= 4 / 16
    assert rate_g > 0.5
