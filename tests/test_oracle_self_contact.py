"""Pins of the oracle's self-contact rows (the robot itself in Eq. ik_coll's minimum distance):
a 4-segment robot bent into one full circle, whose backbone samples lie on a circle of known radius
so that every row has a closed form; the straight robot, whose only close pairs are adjacent
segments (excluded); the gradient against central differences."""
import ctypes as C
import math

import numpy as np


RHO, DELTA = 1e4, 1e-3
L, RC, NB, RBODY = 0.1, 0.005, 8, 0.015


def _rb(orc, n=4):
    return orc.make_robot([L] * n, RC, 0.01, thmax=math.pi, nb=NB, rbody=RBODY)


def _bend(theta, n=4):
    """u of n segments each bent by theta in one plane: u_i = (c, -c/2, -c/2), c = theta r_c."""
    c = theta * RC
    return np.tile([c, -c / 2, -c / 2], n)


def test_full_circle_rows_have_the_closed_form(orc):
    rb = _rb(orc)
    u = _bend(math.pi / 2)
    r, F, _ = orc.self_rows(rb, RHO, DELTA, u[None])
    R = 4 * L / (2 * math.pi)
    gap = 2 * RBODY + DELTA
    want = []
    for i in range(4):
        for ka in range(NB):
            for j in range(i + 2, 4):
                for kb in range(NB):
                    pa = (i + (ka + 1) / NB) * math.pi / 2
                    pb = (j + (kb + 1) / NB) * math.pi / 2
                    dist = 2 * R * abs(math.sin((pb - pa) / 2))
                    want.append(math.sqrt(RHO) * max(0.0, gap - dist))
    want = np.array(want)
    assert np.count_nonzero(want) >= 3, "the circle should close within the gap"
    np.testing.assert_allclose(r[0], want, rtol=0, atol=1e-11)
    assert F[0] == np.float64(0.5 * np.sum(r[0] ** 2))


def test_straight_robot_has_no_self_contact(orc):
    """Straight: segments two apart are at least L + L / n_b > gap apart; adjacent samples
    (L / n_b = 12.5 mm < gap = 31 mm) would be active, but adjacent segments are not paired."""
    rb = _rb(orc)
    r, F, _ = orc.self_rows(rb, RHO, DELTA, np.zeros((1, 12)))
    assert r.shape == (1, 3 * NB * NB) and np.all(r == 0) and F[0] == 0.0
    assert L / NB < 2 * RBODY + DELTA


def test_self_contact_gradient_matches_central_differences(orc):
    rb = _rb(orc)
    rng = np.random.default_rng(2)
    u = _bend(math.pi / 2) + rng.uniform(-2e-4, 2e-4, 12)
    _, F, g = orc.self_rows(rb, RHO, DELTA, u[None], gradient=True)
    assert F[0] > 0
    h = 1e-8
    fd = np.array([(orc.self_rows(rb, RHO, DELTA, (u + h * e)[None])[1][0] -
                    orc.self_rows(rb, RHO, DELTA, (u - h * e)[None])[1][0]) / (2 * h) for e in np.eye(12)])
    np.testing.assert_allclose(g[0], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_self_contact_rows_count_pairs_of_non_adjacent_segments(orc):
    for n, pairs in ((1, 0), (2, 0), (3, 1), (4, 3), (6, 10)):
        rb = orc.make_robot([L] * n, RC, 0.01, nb=NB)
        assert orc.lib().orc_self_row_count(C.byref(rb)) == pairs * NB * NB


def _weights(orc, rho_s):
    from paper_2607_11340_gb300 import synth

    return orc.make_weights(**{**synth.WEIGHTS.as_dict(), "rho_s": rho_s})


def test_ik_residual_carries_the_self_rows_when_weighted(orc):
    """With rho_s > 0 the IK residual ends with exactly the standalone self-contact rows (same values,
    same order), their squares are part of the collision penalty, and rho_s = 0 leaves them out."""
    rb = _rb(orc)
    u = _bend(math.pi / 2)[None]
    tg = np.array([[0.0, 0.0, 0.1, 1.0, 0.0, 0.0, 0.0]])
    W0, W1 = _weights(orc, 0.0), _weights(orc, RHO)
    r0 = orc.ik_eval(rb, W0, None, 0, tg, 1, u, want=("r", "F", "coll"))
    r1 = orc.ik_eval(rb, W1, None, 0, tg, 1, u, want=("r", "F", "coll"))
    rs, Fs, _ = orc.self_rows(rb, RHO, W1.delta, u)
    ns = rs.shape[1]
    assert r1["r"].shape[1] == r0["r"].shape[1] + ns
    np.testing.assert_array_equal(r1["r"][0, :-ns], r0["r"][0])
    np.testing.assert_array_equal(r1["r"][0, -ns:], rs[0])
    assert Fs[0] > 0 and abs(r1["F"][0] - r0["F"][0] - Fs[0]) <= 1e-12 * r1["F"][0]
    assert abs(r1["coll"][0] - r0["coll"][0] - Fs[0]) <= 1e-12 * r1["F"][0]


def test_ik_gradient_with_self_rows_matches_central_differences(orc):
    rb = _rb(orc)
    W = _weights(orc, RHO)
    rng = np.random.default_rng(3)
    u = _bend(math.pi / 2 * 0.97) + rng.normal(0, 2e-5, 12)
    tg = np.array([[0.02, 0.01, 0.05, 0.9, 0.1, 0.3, 0.3]])
    tg[0, 3:] /= np.linalg.norm(tg[0, 3:])
    g = orc.ik_eval(rb, W, None, 0, tg, 1, u[None], want=("g",))["g"][0]
    h = 1e-7
    fd = np.zeros(12)
    for q in range(12):
        up, um = u.copy(), u.copy()
        up[q] += h
        um[q] -= h
        fd[q] = (orc.ik_eval(rb, W, None, 0, tg, 1, up[None])["F"][0] - orc.ik_eval(rb, W, None, 0, tg, 1, um[None])["F"][0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_acceptance_checks_self_contact_only_when_asked(orc):
    """The curled robot (one full circle of 4 segments: segments 0 and 3 meet at the base) is
    collision-free without the self check and collides with it; the straight robot passes both."""
    rb = _rb(orc)
    tg = np.zeros((1, 7))
    tg[0, 3] = 1.0
    curled, straight = _bend(math.pi / 2)[None], np.zeros((1, 12))
    assert orc.accept(rb, None, 0, tg, curled)[3][0]
    assert not orc.accept(rb, None, 0, tg, curled, self_contact=True)[3][0]
    assert orc.accept(rb, None, 0, tg, straight, self_contact=True)[3][0]


def test_lm_with_self_rows_leaves_contact(orc):
    """LM on the IK cost with self-contact rows, from the curled robot towards its own tip pose: the
    pose rows hold the robot curled while the self rows push segments 0 and 3 apart; the solution
    trades a little pose error for clearance (strictly lower self-contact penalty than at the
    start), and the cost never rises."""
    rb = _rb(orc)
    W = _weights(orc, RHO)
    u0 = _bend(math.pi / 2)[None]
    T = orc.fk(rb, u0)[0]
    from paper_2607_11340_gb300 import synth

    tg = synth.pose_targets(T, "pose")
    e0 = orc.ik_eval(rb, W, None, 0, tg, 1, u0, want=("F", "coll"))
    out = orc.ik_lm(rb, W, None, 0, tg, 1, u0, 15, history=True)
    e1 = orc.ik_eval(rb, W, None, 0, tg, 1, out["u"], want=("F", "coll"))
    assert e1["coll"][0] < 0.5 * e0["coll"][0] and e1["F"][0] < e0["F"][0]
    assert np.all(np.diff(out["Fstart"][0]) <= 0)
