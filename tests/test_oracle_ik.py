"""Pins of the oracle's Algorithm 1 (beam-search IK) against brute force.

For the 1-segment robot the feasible set is a 2-D hexagon, so the global minimum of the penalised
cost can be found by exhaustive grid search (a coarse grid to locate the basin, then a 1e-6 m grid
around it). The oracle's multi-start LM must reach that minimum, including for targets that are
not reachable (minimum > 0).
"""
import numpy as np
import pytest

from paper_2607_11340_gb300 import synth


def _setup(orc):
    spec = synth.ROBOT_1SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    return spec, rb, W


def _grid_min(orc, rb, W, tg, b, center=None, half=None, step=None):
    if center is None:
        xs = np.arange(-b, b + 1e-12, step)
        g0, g1 = np.meshgrid(xs, xs, indexing="ij")
    else:
        xs = np.arange(-half, half + 1e-15, step)
        g0, g1 = np.meshgrid(center[0] + xs, center[1] + xs, indexing="ij")
    g0, g1 = g0.ravel(), g1.ravel()
    g2 = -g0 - g1
    ok = (np.abs(g0) <= b) & (np.abs(g1) <= b) & (np.abs(g2) <= b)
    U = np.stack([g0[ok], g1[ok], g2[ok]], 1)
    F = orc.ik_eval(rb, W, None, 1, np.repeat(tg, len(U), 0), 1, U)["F"]
    i = int(np.argmin(F))
    return F[i], U[i]


@pytest.mark.parametrize("offset", [0.0, 4e-3, 1.5e-2])
def test_ik_reaches_brute_force_minimum(orc, offset):
    spec, rb, W = _setup(orc)
    rng = np.random.default_rng(30)
    u_true = synth.hexagon_states(rng, 3, 1, spec.umax)
    T, _ = orc.fk(rb, u_true)
    tg = synth.pose_targets(T, "axis")
    # push the target off the reachable surface along a random direction
    dirs = rng.normal(size=(3, 3))
    tg[:, :3] += offset * dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    cfg = orc.IkConfig(S=32, n_final=32, k_init=0, k_final=50)
    sol = orc.solve_ik(rb, W, None, 1, tg, cfg)
    for q in range(3):
        Fc, uc = _grid_min(orc, rb, W, tg[q:q + 1], spec.umax, step=2e-4)
        Ff, uf = _grid_min(orc, rb, W, tg[q:q + 1], spec.umax, center=uc, half=4e-4, step=1e-6)
        assert sol["F"][q] <= Ff * (1 + 1e-6) + 1e-14, (q, sol["F"][q], Ff)
        if offset == 0.0:
            assert sol["success"][q]
            np.testing.assert_allclose(sol["u"][q], u_true[q], atol=1e-9)


def test_two_stage_ik_success_on_small_sample(orc):
    """Three-segment full-pose IK with the two-stage schedule reaches <= 1 mm / <= 1 deg, and the
    final cost never exceeds the best stage-one cost it started from."""
    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    tg, _ = synth.ik_workload(spec, 6, "pose", lambda u: orc.fk(rb, u)[0], seed=1)
    cfg = orc.IkConfig(S=64, n_final=8, k_init=32, k_final=30)
    sol = orc.solve_ik(rb, W, None, 0, tg, cfg, extra=True)
    assert sol["success"].all()
    assert np.all(sol["F"] <= sol["stage1_F"].min(axis=1))


def test_opcount_is_plausible(orc):
    """Op counts of one 3-segment full-pose evaluation: a few hundred forward flops, a handful
    of special-function calls per segment, and a tangent map of the same order."""
    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    u = synth.hexagon_states(np.random.default_rng(31), 2, 3, spec.umax)
    tg = synth.pose_targets(orc.fk(rb, u[:1])[0], "pose")[0]
    ff, fs, tf, ts = orc.opcount_ik(rb, W, None, 0, tg, u[1])
    assert 200 < ff < 1200 and 9 <= fs <= 30 and 0.5 * ff < tf < 4 * ff
