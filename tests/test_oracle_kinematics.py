"""Pins of the oracle's kinematics (Sec. III, Eq. 1-4) against closed forms and invariants.

Each check uses something the oracle does not: a textbook constant-curvature arc formula, the
forward tendon map of Eq. 4 (the oracle implements its inverse), a group property of rotations,
or an exact geometric fact about circular arcs.
"""
import math

import numpy as np
import pytest

from paper_2607_11340_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def robot(orc, L, rc=0.005, umax=0.01, nb=16):
    return orc.make_robot(list(L), rc, umax, nb=nb)


def u_from_bend(rc, theta, phi, m=3):
    """Forward Eq. 4 per segment: u_j = -r_c theta cos(alpha_j - phi), alpha_j = 2 pi j / m."""
    a = 2 * np.pi * np.arange(m) / m
    return -rc * theta * np.cos(a - phi)


def arc_tip(theta, phi, L):
    """Textbook constant-curvature arc (kappa = theta / L), written with 1 - cos x = 2 sin^2(x/2)."""
    if theta == 0:
        return np.array([0.0, 0.0, L])
    k = theta / L
    omc = 2 * math.sin(theta / 2) ** 2
    return np.array([omc / k * math.cos(phi), omc / k * math.sin(phi), math.sin(theta) / k])


def test_straight_configuration(orc):
    """u = 0: every segment straight, tip at (0, 0, sum L), R = I (Eq. 3, theta = 0 case)."""
    rb = robot(orc, [0.12, 0.10, 0.08])
    T, bb = orc.fk(rb, np.zeros((1, 9)), backbone=True)
    np.testing.assert_allclose(T[0, :9], np.eye(3).ravel(), atol=0)
    np.testing.assert_allclose(T[0, 9:], [0, 0, 0.30], atol=1e-15)
    z = bb[0, :, 2]
    assert np.all(np.diff(z) > 0) and abs(z[-1] - 0.30) < 1e-15


@pytest.mark.parametrize("theta,phi", [(0.3, 0.2), (1.2, 2.5), (2.0, -1.0), (1e-6, 0.7), (2.9, 4.0)])
def test_single_arc_closed_form(orc, theta, phi):
    """Tendon displacements from Eq. 4 -> tip equals the constant-curvature arc end point."""
    L, rc = 0.1, 0.005
    rb = robot(orc, [L], rc=rc)
    u = u_from_bend(rc, theta, phi)[None]
    T, _ = orc.fk(rb, u)
    np.testing.assert_allclose(T[0, 9:], arc_tip(theta, phi, L), rtol=0, atol=1e-15)
    # tip axis = (sin theta cos phi, sin theta sin phi, cos theta)
    R = T[0, :9].reshape(3, 3)
    axis = [math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)]
    np.testing.assert_allclose(R[:, 2], axis, atol=1e-14)


def test_small_angle_branch_matches_arc(orc):
    """Below the theta^2 switch the series branch still gives the arc end point."""
    L, rc = 0.1, 0.005
    rb = robot(orc, [L], rc=rc)
    for theta in [0.0, 1e-9, 5e-5, 9.9e-5, 1.01e-4, 3e-4]:
        u = u_from_bend(rc, theta, 0.4)[None]
        T, _ = orc.fk(rb, u)
        np.testing.assert_allclose(T[0, 9:], arc_tip(theta, 0.4, L), rtol=0, atol=5e-17)


def test_two_coplanar_segments_equal_one_arc(orc):
    """Two segments with the same phi and equal curvature form one arc of L1+L2, theta1+theta2."""
    rc = 0.005
    L1, L2 = 0.12, 0.08
    kappa, phi = 9.0, 1.1
    th1, th2 = kappa * L1, kappa * L2
    rb = robot(orc, [L1, L2], rc=rc)
    u = np.concatenate([u_from_bend(rc, th1, phi), u_from_bend(rc, th2, phi)])[None]
    T, _ = orc.fk(rb, u)
    np.testing.assert_allclose(T[0, 9:], arc_tip(th1 + th2, phi, L1 + L2), atol=1e-15)
    R = T[0, :9].reshape(3, 3)
    th = th1 + th2
    axis = [math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)]
    np.testing.assert_allclose(R[:, 2], axis, atol=1e-14)


def test_rotations_orthonormal(orc):
    rb = robot(orc, [0.12, 0.10, 0.08])
    u = synth.hexagon_states(np.random.default_rng(1), 500, 3, 0.01)
    T, _ = orc.fk(rb, u)
    R = T[:, :9].reshape(-1, 3, 3)
    err = np.einsum("bij,bik->bjk", R, R) - np.eye(3)
    assert np.abs(err).max() < 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-12


def test_rodrigues_form_equals_zyz_product(orc):
    """Eq. 2 as Z(phi) Y(theta) Z(-phi) equals the Rodrigues form the op counter uses."""
    rb = robot(orc, [0.12, 0.10, 0.08])
    u = synth.hexagon_states(np.random.default_rng(2), 300, 3, 0.01)
    T1, _ = orc.fk(rb, u)
    T2 = orc.fk_rodrigues(rb, u)
    assert np.abs(T1 - T2).max() < 4e-15


def test_cyclic_tendon_permutation_rotates_robot(orc):
    """Shifting every segment's tendons by one slot adds 120 deg to every phi_i (Eq. 4), which
    rotates the whole robot about the base z axis: p' = Rz p, R' = Rz R Rz^T."""
    rb = robot(orc, [0.12, 0.10, 0.08])
    u = synth.hexagon_states(np.random.default_rng(3), 50, 3, 0.01)
    up = u.reshape(-1, 3, 3)[:, :, [2, 0, 1]].reshape(-1, 9)
    T, _ = orc.fk(rb, u)
    Tp, _ = orc.fk(rb, up)
    a = 2 * np.pi / 3
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    np.testing.assert_allclose(Tp[:, 9:], T[:, 9:] @ Rz.T, atol=1e-15)
    R = T[:, :9].reshape(-1, 3, 3)
    Rp = Tp[:, :9].reshape(-1, 3, 3)
    np.testing.assert_allclose(Rp, Rz @ R @ Rz.T, atol=1e-14)


def test_tendon_map_round_trip(orc):
    """Eq. 4 forward (the oracle's tendon_lengths) then the oracle's inverse returns (theta, phi),
    and the displacements sum to zero (the sum-zero plane)."""
    rc, L = 0.005, 0.1
    rb = robot(orc, [L], rc=rc)
    rng = np.random.default_rng(4)
    for _ in range(50):
        th, ph = rng.uniform(0.01, 3.0), rng.uniform(-np.pi, np.pi)
        l = orc.tendon_lengths(rc, L, th, ph)
        u = l - L
        assert abs(u.sum()) < 1e-16
        np.testing.assert_allclose(u, u_from_bend(rc, th, ph), atol=1e-16)
        tp = orc.bend(rb, u[None])[0, 0]
        assert abs(tp[0] - th) < 1e-13
        assert abs(math.remainder(tp[1] - ph, 2 * np.pi)) < 1e-13


def test_backbone_lies_on_the_arc(orc):
    """Single segment: every sample is at distance r = L / theta from the arc centre
    r (cos phi, sin phi, 0); consecutive samples are chords 2 r sin(theta / (2 nb)); the last
    sample is the tip."""
    L, rc, nb = 0.1, 0.005, 16
    rb = robot(orc, [L], rc=rc, nb=nb)
    for th, ph in [(0.8, 0.3), (2.2, -2.0), (1e-3, 1.0)]:
        u = u_from_bend(rc, th, ph)[None]
        T, bb = orc.fk(rb, u, backbone=True)
        pts = bb[0]
        r = L / th
        ctr = np.array([r * math.cos(ph), r * math.sin(ph), 0.0])
        np.testing.assert_allclose(np.linalg.norm(pts - ctr, axis=1), r, rtol=1e-12)
        pts0 = np.vstack([np.zeros(3), pts])
        chords = np.linalg.norm(np.diff(pts0, axis=0), axis=1)
        np.testing.assert_allclose(chords, 2 * r * math.sin(th / (2 * nb)), rtol=1e-10)
        np.testing.assert_allclose(pts[-1], T[0, 9:], atol=1e-16)


def test_backbone_arc_length_converges(orc):
    """Sum of chords -> L as the number of samples grows (arc length is preserved)."""
    L, rc = 0.1, 0.005
    u = u_from_bend(rc, 2.0, 0.5)[None]
    errs = []
    for nb in (4, 16, 64, 256):
        rb = robot(orc, [L], rc=rc, nb=nb)
        _, bb = orc.fk(rb, u, backbone=True)
        pts = np.vstack([np.zeros(3), bb[0]])
        errs.append(L - np.linalg.norm(np.diff(pts, axis=0), axis=1).sum())
    assert all(e > 0 for e in errs)
    # chord deficit is O(1/nb^2)
    for a, b in zip(errs, errs[1:]):
        assert 14 < a / b < 18
