"""Pins of the oracle's coupled tendon routing (model B): the actuator displacement of the tendons
that end at segment s equals Eq. l_eq's sum over segments 1..s of the per-segment tendon lengths
of Eq. 4 minus the segment lengths (for s = n, the paper's total tendon length l_j(q)); the map
back to per-segment displacements inverts it; a single segment is model A."""
import numpy as np

from paper_2607_11340_gb300 import synth


def _case(orc, n=4, B=16, seed=3):
    spec = synth.RobotSpec(L=(0.12, 0.10, 0.08, 0.11)[:n], rc=0.005, umax=0.01)
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax)
    u = synth.hexagon_states(np.random.default_rng(seed), B, n, spec.umax)
    return spec, rb, u


def test_actuator_displacements_are_eq_leq_sums(orc):
    spec, rb, u = _case(orc)
    q = orc.routing_b_from_a(rb, u).reshape(len(u), spec.n, 3)
    tp = orc.bend(rb, u)  # (theta_i, phi_i) by the inverse of Eq. 4
    for b in range(len(u)):
        seg = np.array([orc.tendon_lengths(spec.rc, spec.L[i], tp[b, i, 0], tp[b, i, 1]) for i in range(spec.n)])
        for s in range(spec.n):
            total = seg[:s + 1].sum(axis=0)  # Eq. l_eq over the segments the tendons run through
            np.testing.assert_allclose(q[b, s], total - sum(spec.L[:s + 1]), rtol=0, atol=1e-15)


def test_routing_round_trip_and_single_segment(orc):
    spec, rb, u = _case(orc)
    back = orc.routing_a_from_b(rb, orc.routing_b_from_a(rb, u))
    np.testing.assert_allclose(back, u, rtol=0, atol=4 * np.finfo(float).eps * spec.umax * spec.n)
    q = np.random.default_rng(4).uniform(-0.02, 0.02, (8, 12))
    np.testing.assert_allclose(orc.routing_b_from_a(rb, orc.routing_a_from_b(rb, q)), q, rtol=0,
                               atol=8 * np.finfo(float).eps * 0.02)
    spec1, rb1, u1 = _case(orc, n=1)
    np.testing.assert_array_equal(orc.routing_b_from_a(rb1, u1), u1)
    np.testing.assert_array_equal(orc.routing_a_from_b(rb1, u1), u1)


def test_model_b_fk_is_model_a_fk_of_the_differences(orc):
    """FK in actuator coordinates: the segment bends follow from the differences of consecutive
    actuator displacements, so a displacement common to all segments' tendon j (q_sj = c for every
    s) bends only the first segment."""
    spec, rb, _ = _case(orc)
    q = np.zeros((1, 12))
    q[0, 0::3] = 0.006
    q[0, 1::3] = -0.003
    q[0, 2::3] = -0.003
    u = orc.routing_a_from_b(rb, q)
    assert np.all(u[0, 3:] == 0) and np.allclose(u[0, :3], [0.006, -0.003, -0.003])
    tp = orc.bend(rb, u)
    assert tp[0, 0, 0] > 0 and np.all(tp[0, 1:, 0] == 0)


def test_actuator_gradient_is_the_transposed_difference_map(orc):
    """F_B(q) = F_A(D q) with the IK cost F_A: the gradient from routing_b_grad (D^T of the model A
    gradient) matches central differences in q; the actuator feasible set is again per-segment
    hexagons (sum_j q_sj = 0 for every s when every segment's displacements sum to zero)."""
    spec, rb, u = _case(orc, B=3)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    tgt = synth.pose_targets(orc.fk(rb, synth.hexagon_states(np.random.default_rng(8), 1, spec.n, spec.umax))[0],
                             "pose")
    q = orc.routing_b_from_a(rb, u)
    assert np.abs(q.reshape(len(q), spec.n, 3).sum(axis=2)).max() < 1e-17

    def F_B(qq):
        return orc.ik_eval(rb, W, None, orc.IK6, tgt, len(qq), orc.routing_a_from_b(rb, qq), want=("F",))["F"]

    g_u = orc.ik_eval(rb, W, None, orc.IK6, tgt, len(u), u, want=("g",))["g"]
    g_q = orc.routing_b_grad(rb, g_u)
    h = 1e-7
    fd = np.stack([(F_B(q + h * e) - F_B(q - h * e)) / (2 * h) for e in np.eye(q.shape[1])], axis=1)
    np.testing.assert_allclose(g_q, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_coupled_model_state_is_the_actuator_displacement(orc):
    """The coupled model (model B) takes the actuator displacements q as its state: its kinematics,
    cost and gradient equal the per-segment model's at u = the inverse prefix sum of q; its gradient is
    D^T of the per-segment gradient (g_q,s = g_u,s - g_u,s+1), its Jacobian J_u D; bounds act on q."""
    from paper_2607_11340_gb300 import synth

    spec = synth.ROBOT_3SEG
    rbA = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    rbB = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb, coupled=True)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(41)
    q = synth.hexagon_states(rng, 12, 3, spec.umax)  # in the actuator bounds (and so sum-zero)
    u = orc.routing_a_from_b(rbA, q)
    TA, bbA = orc.fk(rbA, u, backbone=True)
    TB, bbB = orc.fk(rbB, q, backbone=True)
    np.testing.assert_array_equal(TA, TB)
    np.testing.assert_array_equal(bbA, bbB)
    tg = synth.pose_targets(orc.fk(rbA, synth.hexagon_states(rng, 12, 3, spec.umax))[0], "pose")
    eA = orc.ik_eval(rbA, W, None, 0, tg, 1, u, want=("g", "J"))
    eB = orc.ik_eval(rbB, W, None, 0, tg, 1, q, want=("F", "g", "J"))
    # pose rows: J_q = J_u D with D the prefix-sum inverse: column s of J_q = col s - col s+1 of J_u
    JA = eA["J"][:, :6, :]
    Jq = JA.copy()
    Jq[:, :, :6] -= JA[:, :, 3:]
    np.testing.assert_allclose(eB["J"][:, :6, :], Jq, rtol=1e-12, atol=1e-12 * np.abs(JA).max())
    # q inside its bounds and sum-zero: model B's bound and sum-zero rows vanish (u = D q itself may
    # leave the per-segment bounds, whose rows model A would add), so g_q = D^T (J_u^T r) over the rows
    # that are functions of the kinematics: the pose rows and the curvature rows (theta of u = D q may
    # pass theta_max). Model A's rows: 6 pose, 2d bound, n sum-zero, n curvature.
    rA = orc.ik_eval(rbA, W, None, 0, tg, 1, u, want=("r",))["r"]
    JAall = eA["J"]
    kin = np.r_[0:6, 6 + 18 + 3:6 + 18 + 3 + 3]
    gu_kin = np.einsum("bkq,bk->bq", JAall[:, kin, :], rA[:, kin])
    gq = gu_kin.copy()
    gq[:, :6] -= gu_kin[:, 3:]
    np.testing.assert_allclose(eB["g"], gq, rtol=1e-10, atol=1e-12 * np.abs(gq).max())
    # the bound rows act on q: a q beyond the bound is penalised even where u is inside
    q2 = q[:1].copy()
    q2[0, 3:6] = [spec.umax * 1.2, -spec.umax * 0.6, -spec.umax * 0.6]
    r2 = orc.ik_eval(rbB, W, None, 0, tg[:1], 1, q2, want=("r",))["r"][0]
    assert np.any(r2[6:6 + 18] > 0)
