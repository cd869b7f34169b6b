"""Pins of the oracle's pose error (Eq. ik_opt / error_eq) and penalty rows (Eq. penalized_form).

The SO(3) logarithm is checked against scipy's rotation-vector conversion, the quaternion map
against scipy, and every penalty row against its value at hand-built violations.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2607_11340_gb300 import synth


def test_so3_log_inverts_exp(orc):
    rng = np.random.default_rng(10)
    w = rng.normal(size=(400, 3))
    w *= (rng.uniform(0, np.pi - 1e-3, 400) / np.linalg.norm(w, axis=1))[:, None]
    w[:5] *= 1e-9          # near identity
    w[5:10] *= 1e-4
    R = Rotation.from_rotvec(w).as_matrix()
    np.testing.assert_allclose(orc.so3_log(R), w, atol=2e-13)


def test_so3_log_near_pi(orc):
    rng = np.random.default_rng(11)
    for eps in [1e-2, 1e-4, 1e-7]:
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        w = (np.pi - eps) * ax
        R = Rotation.from_rotvec(w).as_matrix()
        np.testing.assert_allclose(orc.so3_log(R)[0], w, atol=1e-8)
    # known axes
    for k in range(3):
        w = np.zeros(3)
        w[k] = 2.5
        R = Rotation.from_rotvec(w).as_matrix()
        np.testing.assert_allclose(orc.so3_log(R)[0], w, atol=1e-14)


def test_quaternion_map_vs_scipy(orc):
    q = np.random.default_rng(12).normal(size=(50, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    Rs = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy is scalar-last
    np.testing.assert_allclose(orc.quat_to_R(q), Rs, atol=1e-15)


def _setup(orc, thmax=np.pi):
    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, thmax=thmax, nb=4)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    return spec, rb, W


def test_pose_rows_at_known_offsets(orc):
    """A target offset by dp and rotated by Rz(a) about the tip gives
    cost = 1/2 (w_p^2 |dp|^2 + w_R^2 a^2) exactly, for an in-bound state."""
    spec, rb, W = _setup(orc)
    u = synth.hexagon_states(np.random.default_rng(13), 1, 3, spec.umax) * 0.5
    T, _ = orc.fk(rb, u)
    R = T[0, :9].reshape(3, 3)
    dp = np.array([1e-3, -2e-3, 0.5e-3])
    a = 0.3
    Rt = R @ Rotation.from_rotvec([0, 0, a]).as_matrix()
    tg = np.zeros((1, 7))
    tg[0, :3] = T[0, 9:] + dp
    tg[0, 3:] = synth.rotation_to_quaternion(Rt[None])[0]
    F = orc.ik_eval(rb, W, None, 0, tg, 1, u)["F"][0]
    expect = 0.5 * (W.wp ** 2 * dp @ dp + W.wR ** 2 * a * a)
    assert abs(F - expect) < 1e-12 * expect
    r = orc.ik_eval(rb, W, None, 0, tg, 1, u, want=("r",))["r"][0]
    np.testing.assert_allclose(r[:3], -W.wp * dp, atol=1e-15)
    # Log(R_t^T R) = Log(Rz(-a)) in the tip frame
    np.testing.assert_allclose(r[3:6], [0, 0, -a], atol=1e-13)
    # 5-DoF: tilt the target axis by b about x: axis chord |z - z_t| = 2 sin(b / 2)
    b = 0.2
    Rt5 = R @ Rotation.from_rotvec([b, 0, 0]).as_matrix()
    tg5 = np.zeros((1, 7))
    tg5[0, :3] = T[0, 9:]
    tg5[0, 3:6] = Rt5[:, 2]
    r5 = orc.ik_eval(rb, W, None, 1, tg5, 1, u, want=("r",))["r"][0]
    assert abs(np.linalg.norm(r5[3:6]) - 2 * math.sin(b / 2)) < 1e-14


def test_penalty_rows(orc):
    spec, rb, W = _setup(orc, thmax=1.2)
    u = np.zeros((1, 9))
    tg = synth.pose_targets(orc.fk(rb, u)[0], "pose")
    r = orc.ik_eval(rb, W, None, 0, tg, 1, u, want=("r",))["r"][0]
    assert np.abs(r).max() < 1e-15  # feasible and on target
    # bound violation (upper on u_0, lower on u_4), sum-zero residual on segments 1 and 2
    u = np.zeros((1, 9))
    u[0, 0] = spec.umax + 2e-3
    u[0, 4] = -spec.umax - 1e-3
    r = orc.ik_eval(rb, W, None, 0, tg, 1, u, want=("r",))["r"][0]
    lim = r[6:24].reshape(9, 2)
    sb = math.sqrt(W.rho_b)
    assert abs(lim[0, 0] - sb * 2e-3) < 1e-15 and lim[0, 1] == 0
    assert abs(lim[4, 1] - sb * 1e-3) < 1e-15 and lim[4, 0] == 0
    assert np.count_nonzero(lim) == 2
    se = math.sqrt(W.rho_eq)
    np.testing.assert_allclose(r[24:27], [se * u[0, 0], se * u[0, 4], 0], atol=1e-15)
    # curvature row: theta above thmax = 1.2 rad
    th = 1.5
    a = 2 * np.pi * np.arange(3) / 3
    u = np.zeros((1, 9))
    u[0, 3:6] = -spec.rc * th * np.cos(a - 0.3)
    r = orc.ik_eval(rb, W, None, 0, tg, 1, u, want=("r",))["r"][0]
    sk = math.sqrt(W.rho_k)
    np.testing.assert_allclose(r[27:30], [0, sk * (th - 1.2), 0], atol=1e-12)


def test_clearance_rows(orc):
    """A sphere at distance D from one backbone sample: row = sqrt(rho_c)(r_s + r_body + delta - D)
    when positive, zero beyond reach."""
    spec, rb, W = _setup(orc)
    u = np.zeros((1, 9))
    T, bb = orc.fk(rb, u, backbone=True)  # straight: samples on the z axis
    tg = synth.pose_targets(T, "pose")
    p = bb[0, 5]
    rs = 0.004
    reach = rs + spec.rc + W.delta
    for D in [0.5 * reach, 0.99 * reach, 1.01 * reach]:
        sph = np.array([[p[0] + D, p[1], p[2], rs]])
        r = orc.ik_eval(rb, W, sph, 0, tg, 1, u, want=("r", "coll"))
        rows = r["r"][0, 30:]
        assert rows.shape[0] == 12
        want = math.sqrt(W.rho_c) * max(0.0, reach - D)
        # the sample 5 row; neighbours (spacing 0.025 m) are out of reach
        assert abs(rows[5] - want) < 1e-13
        assert np.count_nonzero(rows) == (1 if want > 0 else 0)
        assert abs(r["coll"][0] - 0.5 * want * want) < 1e-15
