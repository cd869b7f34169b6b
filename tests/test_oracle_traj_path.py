"""Pins of the oracle's trajectory cost (Eq. mp_length_only and the tendon speed / acceleration
finite differences), path-following normal equations (Eq. constrained_mp with smoothness) and
kinematic calibration, against finite differences, hand-built trajectories, numpy least squares
and the statistics of the estimator."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2607_11340_gb300 import synth


def _rb(orc, spec):
    return orc.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius)


def _W(orc, **kw):
    d = synth.WEIGHTS.as_dict()
    d.update(kw)
    return orc.make_weights(**d)


def _traj_case(orc, Tn=6, P=2, n_spheres=4, seed=40):
    spec = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=4)
    rb = _rb(orc, spec)
    us, goal, sph, ug = synth.traj_workload(spec, P, n_spheres, lambda u: orc.fk(rb, u, backbone=True), seed=seed)
    rng = np.random.default_rng(seed)
    s = np.linspace(0, 1, Tn)[1:, None]
    x = us[:, None, :] + s[None] * (ug - us)[:, None, :] + rng.normal(0, 4e-4, (P, Tn - 1, spec.d))
    return spec, rb, us, goal, sph, x


def test_traj_gradient_vs_central_differences(orc):
    spec, rb, us, goal, sph, x = _traj_case(orc)
    # tight limits so that speed and acceleration hinges are active
    W = _W(orc, vmax=0.01, amax=0.05, rho_c=1e3)
    out = orc.traj_eval(rb, W, sph, us, goal, x, want=("F", "g", "r"))
    assert np.count_nonzero(out["r"]) > 50
    h = 1e-6
    g = out["g"].reshape(len(x), -1)
    for c in range(g.shape[1]):
        e = np.zeros(g.shape[1])
        e[c] = h
        Fp = orc.traj_eval(rb, W, sph, us, goal, x + e.reshape(x.shape[1:]))["F"]
        Fm = orc.traj_eval(rb, W, sph, us, goal, x - e.reshape(x.shape[1:]))["F"]
        np.testing.assert_allclose(g[:, c], (Fp - Fm) / (2 * h), rtol=2e-5, atol=1e-6 * np.abs(g).max())


def test_traj_rows_on_constructed_trajectory(orc):
    """Constant tendon velocity v per state: speed rows sqrt(rho_v) max(0, |v|/dt - v_max) on every
    component that moves, acceleration rows zero, length rows sqrt(w_len)(p_t - p_{t-1}) from FK, goal
    rows zero when the last state is the goal state."""
    spec = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=4)
    rb = _rb(orc, spec)
    W = _W(orc)
    Tn, d = 5, spec.d
    u0 = np.zeros(d)
    step = np.zeros(d)
    step[0:3] = [2e-3, -1e-3, -1e-3]  # 0.04 m/s on tendon 0 (inside), 0.02 m/s on 1, 2
    step[3:6] = [-4e-3, 2e-3, 2e-3]   # 0.08 m/s: above v_max = 0.05 m/s
    X = u0 + np.arange(Tn)[:, None] * step
    T, _ = orc.fk(rb, X)
    goal = synth.pose_targets(T[-1:], "pose")
    r = orc.traj_eval(rb, W, None, u0[None], goal, X[None, 1:], want=("r",))["r"][0]
    nsc = 2 * d + 2 * spec.n  # state rows without spheres
    per_t = 3 + 2 * d + nsc
    sv = math.sqrt(W.rho_v)
    for t in range(1, Tn):
        base = (t - 1) * per_t + (2 * d if t > 2 else 0) * 0
        # rows of step t start after the previous steps' rows (t >= 2 adds 2d acceleration rows)
        base = sum(per_t + (2 * d if tt >= 2 else 0) for tt in range(1, t))
        np.testing.assert_allclose(r[base:base + 3], math.sqrt(W.w_len) * (T[t, 9:] - T[t - 1, 9:]), atol=1e-15)
        vel = r[base + 3:base + 3 + 2 * d].reshape(d, 2)
        v = step / W.dt
        np.testing.assert_allclose(vel[:, 0], sv * np.maximum(0, v - W.vmax), atol=1e-12)
        np.testing.assert_allclose(vel[:, 1], sv * np.maximum(0, -W.vmax - v), atol=1e-12)
        if t >= 2:
            acc = r[base + per_t:base + per_t + 2 * d]
            assert np.abs(acc).max() < 1e-9
    assert np.abs(r[-6:]).max() < 1e-12


def test_calibration_recovers_noise_free_parameters(orc):
    spec = synth.ROBOT_3SEG

    def fkp(U, L, rc):
        return orc.fk(orc.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    U, Pm, true, nom = synth.calib_workload(spec, 256, fkp, seed=3, sigma=0.0)
    out = orc.calibrate(_rb(orc, spec), U, Pm, nom, 20)
    np.testing.assert_allclose(out["theta"], true, rtol=1e-10)
    assert out["F"] < 1e-24


def test_calibration_error_matches_covariance(orc):
    """With N(0, sigma^2) noise the estimate's error e satisfies e^T (J^T J / sigma^2) e ~ chi^2(2n)."""
    spec = synth.ROBOT_3SEG

    def fkp(U, L, rc):
        return orc.fk(orc.make_robot(list(L), list(rc), spec.umax, nb=spec.nb), U)[0]

    rb = _rb(orc, spec)
    d2 = []
    for seed in range(12):
        U, Pm, true, nom = synth.calib_workload(spec, 512, fkp, seed=100 + seed)
        est = orc.calibrate(rb, U, Pm, nom, 20)["theta"]
        J = orc.calib_jacobian(rb, U, Pm, est)
        e = est - true
        d2.append(e @ (J.T @ J / synth.SIGMA_CALIB ** 2) @ e)
    d2 = np.array(d2)
    assert np.all(d2 < stats.chi2.ppf(0.999, 6))
    assert 2.0 < d2.mean() < 12.0


def _path_case(orc, H=4, n_spheres=6, seed=50):
    spec = synth.RobotSpec(L=(0.1, 0.1, 0.1, 0.1), rc=0.005, umax=0.01, nb=4)
    rb = _rb(orc, spec)
    wp, states, sph = synth.path_workload(spec, 1, H, n_spheres, lambda u: orc.fk(rb, u, backbone=True), seed=seed)
    return spec, rb, wp[0], states[0], sph[0]


def test_path_rows_at_ground_truth(orc):
    """The reference poses are FK of the ground-truth states and the spheres keep clear of their
    backbones, so only the smoothness rows sqrt(w_s)(u_t - u_{t-1}) are non-zero there."""
    spec, rb, wp, X, sph = _path_case(orc)
    W = _W(orc)
    r = orc.path_residual(rb, W, sph, wp, X)
    H, d = X.shape
    nw = orc.ik_rows(rb, len(sph))
    assert np.abs(r[:H * nw]).max() < 1e-12
    np.testing.assert_allclose(r[H * nw:], math.sqrt(W.w_s) * np.diff(X, axis=0).ravel(), atol=1e-16)


def test_path_lm_step_is_damped_least_squares(orc):
    """One joint LM iteration from a perturbed path moves by the augmented least-squares step built
    from the full complex-step Jacobian of the stacked path residual (the oracle assembles its
    normal equations blockwise per waypoint)."""
    spec, rb, wp, X, sph = _path_case(orc, H=3)
    W = _W(orc, rho_c=1e3)
    rng = np.random.default_rng(51)
    x0 = X + rng.normal(0, 3e-4, X.shape)
    r, J = orc.path_residual(rb, W, sph, wp, x0, jacobian=True)
    lam = 1e-3
    D = np.maximum(np.diag(J.T @ J), 1e-12)
    aug = np.vstack([J, np.diag(np.sqrt(lam * D))])
    step = np.linalg.lstsq(aug, np.concatenate([-r, np.zeros(J.shape[1])]), rcond=None)[0]
    out = orc.path_lm(rb, W, sph, wp, x0, 1, lambda0=lam)
    assert out["acc"][0] == 1
    np.testing.assert_allclose(out["x"].ravel(), x0.ravel() + step, atol=1e-12)
    many = orc.path_lm(rb, W, sph, wp, x0, 15, lambda0=lam, history=True)
    Fs = [0.5 * np.sum(orc.path_residual(rb, W, sph, wp, h) ** 2) for h in many["hist"]]
    assert np.all(np.diff(Fs) <= 0)
