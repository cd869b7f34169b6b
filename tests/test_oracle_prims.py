"""Pins of the oracle's obstacle primitives (the convex pieces of Sec. IV-C in the clearance rows of
Eq. ik_coll): the signed distance to a capsule's segment and to a solid box, and the clearance rows
and acceptance they feed.

The references here are independent of the oracle's arithmetic: a bounded scalar minimisation over
the capsule's segment, a quadratic programme over the box written as six world-frame half-spaces
(built from scipy's rotation of the quaternion, scalar-last), the distance to the nearest face plane
inside the box, reductions to a sphere, and finite differences.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar
from scipy.spatial.transform import Rotation

from paper_2607_11340_gb300 import synth


def _halfspaces(rec):
    """Box record -> (A [6][3], b [6]) with the solid box = {y : A y <= b}."""
    c, h, q = rec[2:5], rec[5:8], rec[8:12]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    A, b = [], []
    for a in range(3):
        n = R[:, a]
        A += [n, -n]
        b += [n @ c + h[a], -(n @ c) + h[a]]
    return np.array(A), np.array(b)


def _box_sd_reference(rec, x):
    A, b = _halfspaces(rec)
    slack = b - A @ x
    if np.all(slack >= 0):
        return -slack.min()  # inside: minus the distance to the nearest face plane
    res = minimize(lambda y: 0.5 * np.sum((y - x) ** 2), x, jac=lambda y: y - x, method="SLSQP",
                   constraints=[{"type": "ineq", "fun": lambda y: b - A @ y, "jac": lambda y: -A}],
                   options={"ftol": 1e-16, "maxiter": 500})
    return float(np.linalg.norm(res.x - x))


def _capsule_sd_reference(rec, x):
    a, bb = rec[2:5], rec[5:8]
    f = lambda t: np.linalg.norm(a + t * (bb - a) - x)
    res = minimize_scalar(f, bounds=(0.0, 1.0), method="bounded", options={"xatol": 1e-13})
    return min(res.fun, f(0.0), f(1.0))


def _boxes(rng, count):
    q = synth.random_quaternions(rng, count)
    return [synth.box_record(rng.uniform(-0.1, 0.1, 3), rng.uniform(0.005, 0.05, 3), q[k]) for k in range(count)]


def test_capsule_distance_vs_scalar_minimisation(orc):
    rng = np.random.default_rng(1)
    recs = synth.prims_uniform(rng, 8, 0, [-0.1] * 3, [0.1] * 3, 0.005, 0.02, 0.01, 0.08)
    for rec in recs:
        x = rng.uniform(-0.2, 0.2, (64, 3))
        sd = orc.obstacle_sd(rec, x)
        ref = np.array([_capsule_sd_reference(rec, xi) for xi in x])
        np.testing.assert_allclose(sd, ref, rtol=0, atol=1e-9)


def test_capsule_end_caps_and_middle(orc):
    """Beyond an end the distance is to that end point; beside the segment it is the perpendicular
    distance."""
    rec = synth.capsule_record([0.0, 0.0, 0.0], [0.0, 0.0, 0.2], 0.01)
    x = np.array([[0.0, 0.0, -0.05], [0.03, 0.04, 0.25], [0.03, 0.04, 0.1]])
    np.testing.assert_allclose(orc.obstacle_sd(rec, x), [0.05, math.hypot(0.05, 0.05), 0.05], atol=1e-15)


def test_box_distance_outside_vs_qp(orc):
    rng = np.random.default_rng(2)
    for rec in _boxes(rng, 6):
        A, b = _halfspaces(rec)
        x = rng.uniform(-0.2, 0.2, (200, 3))
        x = x[np.any(A @ x.T > b[:, None] + 1e-3, axis=0)][:40]
        sd = orc.obstacle_sd(rec, x)
        ref = np.array([_box_sd_reference(rec, xi) for xi in x])
        assert np.all(sd > 0)
        np.testing.assert_allclose(sd, ref, rtol=0, atol=1e-7)


def test_box_distance_inside_is_minus_nearest_face(orc):
    rng = np.random.default_rng(3)
    for rec in _boxes(rng, 6):
        A, b = _halfspaces(rec)
        R = Rotation.from_quat([rec[9], rec[10], rec[11], rec[8]]).as_matrix()
        p = rng.uniform(-1, 1, (40, 3)) * rec[5:8]  # box coordinates inside
        x = rec[2:5] + p @ R.T
        sd = orc.obstacle_sd(rec, x)
        ref = -(b[None, :] - x @ A.T).min(axis=1)
        assert np.all(sd <= 0)
        np.testing.assert_allclose(sd, ref, rtol=0, atol=1e-13)


def test_sign_matches_half_space_membership(orc):
    rng = np.random.default_rng(4)
    for rec in _boxes(rng, 4):
        A, b = _halfspaces(rec)
        x = rng.uniform(-0.12, 0.12, (500, 3))
        inside = np.all(A @ x.T <= b[:, None], axis=0)
        sd = orc.obstacle_sd(rec, x)
        assert inside.any() and (~inside).any()
        np.testing.assert_array_equal(sd <= 0, inside)


def test_degenerate_primitives_are_spheres(orc):
    """A capsule with a = b and a box with zero extents are a sphere about that point; a point
    record (kind 0) and any unknown kind read as a sphere."""
    rng = np.random.default_rng(5)
    c = np.array([0.02, -0.01, 0.05])
    x = rng.uniform(-0.2, 0.2, (50, 3))
    want = np.linalg.norm(x - c, axis=1)
    cap = synth.capsule_record(c, c, 0.01)
    box = synth.box_record(c, [0, 0, 0], synth.random_quaternions(rng, 1)[0], 0.01)
    pt = np.zeros(16)
    pt[2:5] = c
    odd = pt.copy()
    odd[0] = 7
    for rec in (cap, box, pt, odd):
        np.testing.assert_allclose(orc.obstacle_sd(rec, x), want, rtol=0, atol=1e-15)


def test_distance_gradient_is_unit_and_matches_differences(orc):
    rng = np.random.default_rng(6)
    recs = list(synth.prims_uniform(rng, 3, 3, [-0.05] * 3, [0.05] * 3, 0.005, 0.02, 0.01, 0.05))
    h = 1e-7
    for rec in recs:
        x = rng.uniform(-0.15, 0.15, (60, 3))
        sd, g = orc.obstacle_sd(rec, x, gradient=True)
        np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-12)
        fd = np.stack([(orc.obstacle_sd(rec, x + h * e) - orc.obstacle_sd(rec, x - h * e)) / (2 * h)
                       for e in np.eye(3)], axis=1)
        # away from the kinks (the medial planes inside a box) the difference quotient agrees
        ok = np.all(np.abs(fd - g) < 1e-5, axis=1)
        assert ok.mean() > 0.9
        np.testing.assert_allclose(fd[ok], g[ok], atol=1e-5)


def _setup(orc, nb=8):
    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    return spec, rb, W


def _scene(rng):
    prims = synth.prims_uniform(rng, 4, 6, [-0.12, -0.12, 0.05], [0.12, 0.12, 0.3], 0.004, 0.012, 0.01, 0.05)
    sph = synth.spheres_uniform(rng, 5, [-0.12, -0.12, 0.05], [0.12, 0.12, 0.3], 0.01, 0.03)
    return sph, prims


def _sd_ref(rec, x):
    return _capsule_sd_reference(rec, x) if rec[0] == synth.PRIM_CAPSULE else _box_sd_reference(rec, x)


def test_clearance_cost_with_primitives(orc):
    """coll = 1/2 rho_c sum over samples and obstacles of max(0, r + r_body + delta - sd)^2, with the
    distances from the independent references."""
    spec, rb, W = _setup(orc)
    rng = np.random.default_rng(7)
    sph, prims = _scene(rng)
    u = synth.hexagon_states(rng, 24, 3, spec.umax)
    T, bb = orc.fk(rb, u, backbone=True)
    tg = synth.pose_targets(T, "pose")
    out = orc.ik_eval(rb, W, (sph, prims), 0, tg, 1, u, want=("coll",))["coll"]
    reach_add = spec.rc + synth.WEIGHTS.delta
    hits = 0
    for b in range(u.shape[0]):
        tot = 0.0
        for x in bb[b]:
            for s in sph:
                v = s[3] + reach_add - np.linalg.norm(x - s[:3])
                tot += max(0.0, v) ** 2
            for rec in prims:
                v = rec[1] + reach_add - _sd_ref(rec, x)
                tot += max(0.0, v) ** 2
                hits += v > 0
        assert abs(out[b] - 0.5 * synth.WEIGHTS.rho_c * tot) <= 1e-6 * max(1.0, 0.5 * synth.WEIGHTS.rho_c * tot)
    assert hits > 20


def test_gradient_with_primitives_vs_differences(orc):
    spec, rb, W = _setup(orc)
    rng = np.random.default_rng(8)
    sph, prims = _scene(rng)
    u = synth.hexagon_states(rng, 32, 3, spec.umax)
    tg = synth.pose_targets(orc.fk(rb, synth.hexagon_states(rng, 32, 3, spec.umax))[0], "pose")
    r = orc.ik_eval(rb, W, (sph, prims), 0, tg, 1, u, want=("F", "g", "coll"))
    assert (r["coll"] > 0).sum() >= 4
    h = 1e-8
    fd = np.zeros_like(u)
    for q in range(u.shape[1]):
        up, um = u.copy(), u.copy()
        up[:, q] += h
        um[:, q] -= h
        fd[:, q] = (orc.ik_eval(rb, W, (sph, prims), 0, tg, 1, up)["F"] -
                    orc.ik_eval(rb, W, (sph, prims), 0, tg, 1, um)["F"]) / (2 * h)
    scale = np.abs(r["g"]).max(axis=1, keepdims=True) + 1.0
    assert np.all(np.abs(fd - r["g"]) / scale < 1e-4)


def test_acceptance_against_primitives(orc):
    """A straight robot through a box is rejected; the same box moved so that every sample clears
    it by r + r_body is accepted; a capsule along the backbone is rejected."""
    spec, rb, W = _setup(orc)
    u = np.zeros((1, 9))
    T, bb = orc.fk(rb, u, backbone=True)
    tg = synth.pose_targets(T, "pose")
    q = np.array([1.0, 0.0, 0.0, 0.0])
    through = synth.box_record([0.0, 0.0, 0.15], [0.02, 0.02, 0.01], q, 0.002)
    clear = synth.box_record([0.02 + 0.002 + spec.rc + 1e-4, 0.0, 0.15], [0.02, 0.02, 0.01], q, 0.002)
    along = synth.capsule_record([0.0, 0.0, 0.05], [0.0, 0.0, 0.25], 0.001)
    flags = []
    for rec in (through, clear, along):
        flags.append(bool(orc.accept(rb, (None, rec[None, :]), 0, tg, u)[3][0]))
    assert flags == [False, True, False]


def test_trajectory_and_path_obstacles_per_problem(orc):
    """Per-problem obstacle sets in the trajectory and path residuals: the cost with problem p's
    spheres and primitives, less the cost without obstacles, is the clearance part of the IK cost of
    the states that carry rows (trajectory states 1..T-1; every waypoint of a path) with that same
    set, so each problem reads its own records."""
    spec, rb, W = _setup(orc)
    rng = np.random.default_rng(9)
    P, Tn = 3, 5
    us = synth.hexagon_states(rng, P, 3, spec.umax)
    x = synth.hexagon_states(rng, P * (Tn - 1), 3, spec.umax).reshape(P, Tn - 1, 9)
    goal = synth.pose_targets(orc.fk(rb, synth.hexagon_states(rng, P, 3, spec.umax))[0], "pose")
    _, bb = orc.fk(rb, x.reshape(-1, 9), backbone=True)
    sph = np.stack([synth.spheres_uniform(rng, 2, [-0.1, -0.1, 0.05], [0.1, 0.1, 0.3], 0.01, 0.03)
                    for _ in range(P)])
    prims = np.stack([_prims_near(rng, bb.reshape(P, -1, 3)[p]) for p in range(P)])
    with_obs = orc.traj_eval(rb, W, (sph, prims), us, goal, x)["F"]
    without = orc.traj_eval(rb, W, None, us, goal, x)["F"]
    tg = np.zeros((1, 7))
    tg[0, 3] = 1.0
    for p in range(P):
        coll = orc.ik_eval(rb, W, (sph[p], prims[p]), 0, tg, Tn - 1, x[p], want=("coll",))["coll"]
        assert coll.sum() > 0
        assert abs((with_obs[p] - without[p]) - coll.sum()) <= 1e-9 * max(1.0, coll.sum())
    # paths: the residual rows of waypoint t's IK block with the path's own set
    wp = np.stack([synth.pose_targets(orc.fk(rb, x[p])[0], "pose") for p in range(P)])
    for p in range(P):
        r_obs = orc.path_residual(rb, W, (sph[p], prims[p]), wp[p], x[p])
        r_none = orc.path_residual(rb, W, None, wp[p], x[p])
        coll = orc.ik_eval(rb, W, (sph[p], prims[p]), 0, wp[p], 1, x[p], want=("coll",))["coll"]
        assert abs(0.5 * (r_obs @ r_obs - r_none @ r_none) - coll.sum()) <= 1e-9 * max(1.0, coll.sum())


def _prims_near(rng, pts):
    """A capsule and a box around points of the given backbones (some samples inside the box)."""
    c = pts[rng.integers(len(pts))]
    d = pts[rng.integers(len(pts))]
    q = synth.random_quaternions(rng, 1)[0]
    return np.stack([synth.capsule_record(c + [0.006, 0.0, 0.0], c + [0.006, 0.02, 0.0], 0.003),
                     synth.box_record(d, [0.012, 0.008, 0.006], q, 0.002)])
