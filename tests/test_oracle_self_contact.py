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
