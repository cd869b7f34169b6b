"""Pins of the oracle's arc model: the paper's own segment configuration q_i = (theta, phi, L) of
Sec. IV-A with extendable length L in [lmin, lmax], written as (theta cos phi, theta sin phi, L).

Each check rests on something outside the arc model's code: the textbook constant-curvature arc,
the tendon model's kinematics (pinned in test_oracle_kinematics.py) at the same bend, the geometry
of two arcs of equal curvature, the closest point of a disk and of an interval, the uniform law of
the seeds, central differences, and exact solvability of targets built by forward kinematics.
"""
import math

import numpy as np
import pytest

from paper_2607_11340_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")

LMIN, LMAX, THMAX = 0.5, 1.5, 0.5 * np.pi


def arc_robot(orc, n, nb=10, L=1.0, thmax=THMAX, lmin=LMIN, lmax=LMAX):
    return orc.make_robot([L] * n, 0.01, 0.01, thmax=thmax, nb=nb, rbody=0.05, lmin=lmin, lmax=lmax)


def arc_tip(theta, phi, L):
    """Textbook constant-curvature arc (kappa = theta / L), with 1 - cos x = 2 sin^2(x/2)."""
    if theta == 0:
        return np.array([0.0, 0.0, L])
    k = theta / L
    omc = 2 * math.sin(theta / 2) ** 2
    return np.array([omc / k * math.cos(phi), omc / k * math.sin(phi), math.sin(theta) / k])


def test_single_arc_closed_form(orc):
    rng = np.random.default_rng(1)
    rb = arc_robot(orc, 1)
    for _ in range(20):
        th, ph, L = rng.uniform(0, THMAX), rng.uniform(-np.pi, np.pi), rng.uniform(LMIN, LMAX)
        T, _ = orc.fk(rb, np.array([[th * np.cos(ph), th * np.sin(ph), L]]))
        np.testing.assert_allclose(T[0, 9:], arc_tip(th, ph, L), atol=1e-13)
        z = T[0, [2, 5, 8]]
        np.testing.assert_allclose(z, [math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)],
                                   atol=1e-14)
    # straight, any length
    T, _ = orc.fk(rb, np.array([[0.0, 0.0, 1.3]]))
    np.testing.assert_allclose(T[0, 9:], [0, 0, 1.3], atol=0)


def test_same_bend_as_tendon_model(orc):
    """At the bend (theta, phi) the tendon model gives (inverse of Eq. 4) and the robot's lengths,
    both models place every frame and backbone sample identically."""
    spec = synth.ROBOT_3SEG
    rt = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=8)
    ra = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=8, lmin=0.05, lmax=0.2)
    u = synth.hexagon_states(np.random.default_rng(2), 50, 3, spec.umax)
    tp = orc.bend(rt, u)
    q = np.zeros_like(u)
    for i in range(3):
        q[:, 3 * i] = tp[:, i, 0] * np.cos(tp[:, i, 1])
        q[:, 3 * i + 1] = tp[:, i, 0] * np.sin(tp[:, i, 1])
        q[:, 3 * i + 2] = spec.L[i]
    Tt, bt = orc.fk(rt, u, backbone=True)
    Ta, ba = orc.fk(ra, q, backbone=True)
    np.testing.assert_allclose(Ta, Tt, atol=1e-14)
    np.testing.assert_allclose(ba, bt, atol=1e-14)


def test_two_equal_curvature_segments_are_one_arc(orc):
    """Extendable segments of equal curvature and plane: one arc of the summed angle and length."""
    rng = np.random.default_rng(3)
    rb = arc_robot(orc, 2)
    for _ in range(10):
        kappa, ph = rng.uniform(0.1, 0.9), rng.uniform(-np.pi, np.pi)
        L1, L2 = rng.uniform(LMIN, LMAX, 2)
        q = [kappa * L1 * np.cos(ph), kappa * L1 * np.sin(ph), L1, kappa * L2 * np.cos(ph), kappa * L2 * np.sin(ph), L2]
        T, _ = orc.fk(rb, np.array([q]))
        np.testing.assert_allclose(T[0, 9:], arc_tip(kappa * (L1 + L2), ph, L1 + L2), atol=1e-13)


def test_constraint_rows(orc):
    """Eq. ik_limits on q: two length hinges and the bend-angle hinge per segment, no sum-zero row."""
    w = synth.WEIGHTS
    rb = arc_robot(orc, 2, thmax=1.0)
    W = orc.make_weights(**w.as_dict())
    assert orc.ik_rows(rb, 0) == 6 + 3 * 2
    th = 1.3
    q = np.array([[th, 0.0, 1.7, 0.0, 0.2, 0.3]])  # L1 above lmax, L2 below lmin, theta1 > thmax
    tg = np.array([[0, 0, 2.0, 1, 0, 0, 0]])
    r = orc.ik_eval(rb, W, None, orc.IK6, tg, 1, q, want=("r",))["r"][0]
    sb, sk = math.sqrt(w.rho_b), math.sqrt(w.rho_k)
    np.testing.assert_allclose(r[6:10], [sb * 0.2, 0.0, 0.0, sb * 0.2], rtol=1e-12)
    np.testing.assert_allclose(r[10:12], [sk * (th - 1.0), 0.0], rtol=1e-12)


def test_gradient_central_differences(orc):
    """dF/dq (complex step, including the length column) against central differences."""
    rb = arc_robot(orc, 3, thmax=1.0)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(4)
    q = np.array([[0.4, -0.3, 1.6, 1.1, 0.2, 0.9, -0.2, 0.1, 0.45]])  # L1, L3 and theta2 violated
    tg = np.array([[0.3, -0.2, 2.1, 0.9, 0.1, -0.3, 0.2]])
    tg[0, 3:] /= np.linalg.norm(tg[0, 3:])
    sph = np.array([[0.2, 0.0, 1.0, 0.3]])
    g = orc.ik_eval(rb, W, sph, orc.IK6, tg, 1, q, want=("g",))["g"][0]
    h = 1e-6
    for c in range(9):
        e = np.zeros((1, 9))
        e[0, c] = h
        Fp = orc.ik_eval(rb, W, sph, orc.IK6, tg, 1, q + e, want=("F",))["F"][0]
        Fm = orc.ik_eval(rb, W, sph, orc.IK6, tg, 1, q - e, want=("F",))["F"][0]
        np.testing.assert_allclose(g[c], (Fp - Fm) / (2 * h), rtol=1e-5, atol=1e-6 * max(1.0, abs(g).max()))
    del rng


def test_projection_is_the_closest_point(orc):
    """Against the closest point found by brute force over a polar grid of the disk times the
    interval (the grid's spacing bounds the distance gap)."""
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(-3, 3, (40, 2)), rng.uniform(0, 2, (40, 1))], axis=1)
    u = orc.project_arc(v, THMAX, LMIN, LMAX)
    r = np.linspace(0, THMAX, 301)
    a = np.linspace(-np.pi, np.pi, 1441)
    R, A = np.meshgrid(r, a)
    X, Y = (R * np.cos(A)).ravel(), (R * np.sin(A)).ravel()
    for k in range(len(v)):
        d_disk = np.min((X - v[k, 0]) ** 2 + (Y - v[k, 1]) ** 2)
        d_len = (np.clip(v[k, 2], LMIN, LMAX) - v[k, 2]) ** 2
        got = (u[k, 0] - v[k, 0]) ** 2 + (u[k, 1] - v[k, 1]) ** 2 + (u[k, 2] - v[k, 2]) ** 2
        assert got <= d_disk + d_len + 1e-12
        assert d_disk - ((u[k, 0] - v[k, 0]) ** 2 + (u[k, 1] - v[k, 1]) ** 2) <= 1e-4 * (1 + d_disk)
        assert math.hypot(u[k, 0], u[k, 1]) <= THMAX * (1 + 1e-15) and LMIN <= u[k, 2] <= LMAX
    inside = np.array([[0.1, -0.2, 0.9]])
    np.testing.assert_array_equal(orc.project_arc(inside, THMAX, LMIN, LMAX), inside)


def test_seeds_uniform_on_disk_and_interval(orc):
    """Seeds lie in the set; the squared radius / thmax^2, the azimuth / 2 pi + 1/2 and the length
    fraction are uniform on [0, 1) (chi-square with 20 bins, 99.9 % quantile)."""
    rb = arc_robot(orc, 2)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    x = orc.seeds(rb, W, None, 99, 0, 40, 250, ).reshape(-1, 3)
    r2 = (x[:, 0] ** 2 + x[:, 1] ** 2) / THMAX ** 2
    assert r2.max() <= 1.0 and x[:, 2].min() >= LMIN and x[:, 2].max() <= LMAX
    crit = 45.3  # chi-square, 19 degrees of freedom, 0.999
    for s in (r2, np.arctan2(x[:, 1], x[:, 0]) / (2 * np.pi) + 0.5, (x[:, 2] - LMIN) / (LMAX - LMIN)):
        cnt, _ = np.histogram(s, bins=20, range=(0, 1))
        e = len(s) / 20
        assert np.sum((cnt - e) ** 2 / e) < crit
    # counter-based: the seeds of problem 7 do not depend on the batch they are drawn in
    a = orc.seeds(rb, W, None, 99, 7, 1, 250)
    np.testing.assert_array_equal(a[0], orc.seeds(rb, W, None, 99, 0, 40, 250)[7])


def test_ik_solves_reachable_targets(orc):
    """Targets built by FK of in-bound arc states are exactly reachable: Algorithm 1 on a 2-segment
    extendable robot finds zero-residual solutions within the bounds."""
    rb = arc_robot(orc, 2, nb=8)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(6)
    n = 24
    r, a = THMAX * np.sqrt(rng.uniform(0, 1, (n, 2))), rng.uniform(-np.pi, np.pi, (n, 2))
    q = np.stack([r[:, 0] * np.cos(a[:, 0]), r[:, 0] * np.sin(a[:, 0]), rng.uniform(LMIN, LMAX, n),
                  r[:, 1] * np.cos(a[:, 1]), r[:, 1] * np.sin(a[:, 1]), rng.uniform(LMIN, LMAX, n)], axis=1)
    tg = synth.pose_targets(orc.fk(rb, q)[0], "pose")
    cfg = orc.IkConfig(S=64, n_final=4, k_init=32, k_final=40, alpha0=0.05, pos_tol=1e-3, rot_tol=np.pi / 180)
    out = orc.solve_ik(rb, W, None, orc.IK6, tg, cfg)
    assert out["success"].mean() >= 0.9
    ok = out["success"].astype(bool)
    assert np.all(out["F"][ok] < 1e-10)
    pos, rot, lim, col = orc.accept(rb, None, orc.IK6, tg, out["u"])
    assert np.all(lim[ok])
