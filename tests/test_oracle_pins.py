"""Worked-example pins of the oracle's step rules and of its op counter.

Each expected value below is derived by hand in the comments, from the rule as the readings of the
paper state it (stage one of Algorithm 1: normalised projected-gradient steps with an adaptive
length; Sec. IV-C: Levenberg-Marquardt with Marquardt scaling and the Madsen-Nielsen-Tingleff
damping update), not by re-running oracle code. `tests/test_oracle_mutants.py` plants plausible
mistakes in a copy of the oracle and checks that these pins catch them.
"""
import math

import numpy as np


# ------------------------------------------------------------------------------------------------
# Stage-one step rule: trial x' = Pi(x - alpha g/|g|); accept iff F(x') < F(x), then alpha *= 1.25
# and g is refreshed at x'; otherwise x stays and alpha /= 2.
# ------------------------------------------------------------------------------------------------
def pin_pg_interior(orc):
    """F = 1/2 |u|^2 on the hexagon b = 0.01, from u0 = (8, -4, -4) mm, alpha0 = 4 mm.

    The minimiser c = 0 is inside the hexagon and u0 lies on the ray from it along
    e = (2, -1, -1)/sqrt(6), so every trial stays on that line: x = s e with the signed distance s,
    g = x, and the step moves s towards 0 by alpha (crossing it if alpha > |s|). d0 = |u0| = sqrt(96) mm.
      step 1: s = d0 - 4 = 5.798 mm, |s| < d0: accept, alpha = 5
      step 2: s = d0 - 9 = 0.798 mm: accept, alpha = 6.25
      step 3: trial s = d0 - 15.25 = -5.45 mm, |.| > 0.798: reject, alpha = 3.125
      step 4: trial s = d0 - 12.125 = -2.33 mm: reject, alpha = 1.5625
      step 5: trial s = d0 - 10.5625 = -0.765 mm, |.| < 0.798: accept (crossed), alpha = 1.953125
      step 6: g now points the other way: trial s = -0.765 + 1.953 = 1.189 mm > 0.765: reject, alpha = 0.9765625
      step 7: trial s = -0.765 + 0.977 = 0.212 mm: accept, alpha = 1.220703125
    """
    b = 0.01
    u0 = np.array([0.008, -0.004, -0.004])
    e = u0 / np.linalg.norm(u0)
    d0 = math.sqrt(96.0) * 1e-3
    s_after = [d0 - 0.004, d0 - 0.009, d0 - 0.009, d0 - 0.009, d0 - 0.0105625, d0 - 0.0105625,
               d0 - 0.0105625 + 0.0009765625]
    alpha_after = [0.005, 0.00625, 0.003125, 0.0015625, 0.001953125, 0.0009765625, 0.001220703125]
    u, F, hist = orc.pg_quadratic(np.zeros(3), b, u0, 7, 0.004)
    for k in range(7):
        np.testing.assert_allclose(hist[k, :3], s_after[k] * e, rtol=0, atol=1e-15, err_msg=f"step {k + 1}")
        assert hist[k, 3] == alpha_after[k], (k, hist[k, 3])
        assert abs(hist[k, 4] - 0.5 * s_after[k] ** 2) <= 1e-18, k
    assert F == hist[-1, 4]


def _project_first_clamped(v, b):
    """Euclidean projection onto {|u_j| <= b, sum u = 0} when only u_0 sits on its upper bound:
    the KKT conditions give u = (b, v1 - tau, v2 - tau) with tau = (b + v1 + v2) / 2 (the sum is
    zero); the caller checks that the active set is the assumed one."""
    tau = (b + v[1] + v[2]) / 2
    u = np.array([b, v[1] - tau, v[2] - tau])
    assert v[0] - tau >= b and abs(u[1]) <= b and abs(u[2]) <= b
    return u


def pin_pg_projected(orc):
    """F = 1/2 |u - c|^2 with c = (30, -10, -20) mm outside the hexagon b = 10 mm, u0 = 0, alpha0 = 10 mm.

      step 1: trial 10 c/|c| = (8.02, -2.67, -5.35) mm is inside: accept, alpha = 12.5
      step 2: x1 is on the ray to c, so the trial is 22.5 c/|c| = (18.0, -6.0, -12.0) mm, outside;
              its projection (u_0 on its bound, KKT) is closer to c: accept, alpha = 15.625
      step 3: g = x2 - c is no longer along c; the trial x2 - 15.625 g/|g| projects the same way and
              is closer: accept, alpha = 19.53125
    The constrained minimiser is (10, 0, -10) mm (F* = 3e-4); the iterates approach it.
    """
    b = 0.01
    c = np.array([0.03, -0.01, -0.02])
    ch = c / np.linalg.norm(c)
    x1 = 0.01 * ch
    x2 = _project_first_clamped(0.0225 * ch, b)
    g2 = x2 - c
    x3 = _project_first_clamped(x2 - 0.015625 * g2 / np.linalg.norm(g2), b)
    F = [0.5 * np.dot(x - c, x - c) for x in (x1, x2, x3)]
    assert F[0] > F[1] > F[2] > 3e-4
    u, _, hist = orc.pg_quadratic(c, b, np.zeros(3), 3, 0.01)
    for k, (x, a) in enumerate(zip((x1, x2, x3), (0.0125, 0.015625, 0.01953125))):
        np.testing.assert_allclose(hist[k, :3], x, rtol=0, atol=1e-15, err_msg=f"step {k + 1}")
        assert hist[k, 3] == a and abs(hist[k, 4] - F[k]) <= 1e-18, k


def pin_pg_stall_at_vertex(orc):
    """c = (20, -20, 0) mm: the closest point of the hexagon is its vertex (10, -10, 0) mm, on the
    ray from u0 = 0. Step 1 (alpha 10 mm) lands inside and is accepted; step 2's trial projects
    onto the vertex, closer, accepted; from the vertex every trial projects back onto it, so F does
    not strictly decrease and steps 3-5 are rejected with alpha halving each time."""
    b = 0.01
    c = np.array([0.02, -0.02, 0.0])
    u, F, hist = orc.pg_quadratic(c, b, np.zeros(3), 5, 0.01)
    ch = c / np.linalg.norm(c)
    np.testing.assert_allclose(hist[0, :3], 0.01 * ch, atol=1e-15)
    vertex = np.array([b, -b, 0.0])
    for k in range(1, 5):
        np.testing.assert_allclose(hist[k, :3], vertex, atol=1e-15)
    np.testing.assert_array_equal(hist[:, 3], [0.0125, 0.015625, 0.0078125, 0.00390625, 0.001953125])
    assert F == 0.5 * 2e-4 or abs(F - 1e-4) < 1e-19


def test_pg_interior(orc):
    pin_pg_interior(orc)


def test_pg_projected(orc):
    pin_pg_projected(orc)


def test_pg_stall_at_vertex(orc):
    pin_pg_stall_at_vertex(orc)


def pin_pg_ik_is_the_rule(orc):
    """Stage one of the IK (orc.ik_pg) and the trajectory refinement take their steps with the same
    rule: one IK PG step from a seed equals, by the rule above, either the projected normalised
    step (if its cost is lower) or no move. Checked on 32 seeds against the oracle's own cost,
    gradient and projection (the rule's composition, not its arithmetic)."""
    from paper_2607_11340_gb300 import synth

    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(31)
    tg = synth.pose_targets(orc.fk(rb, synth.hexagon_states(rng, 4, 3, spec.umax))[0], "pose")
    u0 = orc.seeds(rb, W, None, 0, 0, 4, 8).reshape(32, 9)
    ev = orc.ik_eval(rb, W, None, 0, tg, 8, u0, want=("F", "g"))
    a0 = 2e-2  # long enough that 7 of the 32 trials raise the cost
    v = u0 - a0 * ev["g"] / np.linalg.norm(ev["g"], axis=1, keepdims=True)
    x1 = orc.project(v.reshape(-1, 3), spec.umax).reshape(32, 9)
    F1 = orc.ik_eval(rb, W, None, 0, tg, 8, x1)["F"]
    acc = F1 < ev["F"]
    assert 0 < acc.sum() < 32
    u, F = orc.ik_pg(rb, W, None, 0, tg, 8, u0, 1, a0)
    # same decisions; the iterates agree to rounding (the test forms alpha g / |g| in another order)
    np.testing.assert_allclose(u[acc], x1[acc], rtol=0, atol=1e-17)
    np.testing.assert_array_equal(u[~acc], u0[~acc])
    np.testing.assert_allclose(F, np.where(acc, F1, ev["F"]), rtol=1e-13, atol=0)


def test_pg_ik_is_the_rule(orc):
    pin_pg_ik_is_the_rule(orc)


# ------------------------------------------------------------------------------------------------
# LM (Sec. IV-C): the rejection branch, then an accept after rejections
# ------------------------------------------------------------------------------------------------
def pin_lm_rejections(orc):
    """r(x) = x^2 - 4 from x0 = 0.5, lambda0 = 1e-3. At x0: r = -3.75, J = 2 x0 = 1, so
    J^T J = 1 = D and the step is delta = 3.75 / (1 + lambda). F0 = 3.75^2 / 2 = 7.03125.
      it 1: delta = 3.7463, x = 4.246, r = 14.03: F rises -> reject: lambda = 1e-3 * 2 = 2e-3, nu = 4
      it 2: delta = 3.75 / 1.002 -> x = 4.2425, F rises -> reject: lambda = 2e-3 * 4 = 8e-3, nu = 8
      it 3: delta = 3.75 / 1.008 -> reject: lambda = 8e-3 * 8 = 0.064, nu = 16
      it 4: delta = 3.75 / 1.064, x = 4.024, r = 12.2 -> reject: lambda = 0.064 * 16 = 1.024, nu = 32
      it 5: delta = 3.75 / 2.024 = 1.8528, x = 2.3528, r = 1.5355, F = 1.1789 < F0: accept.
            Predicted decrease 1/2 delta (lambda D delta - g) = 1/2 * 1.8528 * (1.024 * 1.8528 + 3.75)
            = 5.2315, gain ratio (7.03125 - 1.1789) / 5.2315 = 1.119, 2 rho - 1 = 1.237,
            1 - 1.237^3 < 1/3: lambda = 1.024 / 3, nu = 2.
    x stays at 0.5 through every rejected iteration."""
    r = orc.lm_scalar(4.0, 0.5, 5)
    np.testing.assert_array_equal(r["acc"], [0, 0, 0, 0, 1])
    np.testing.assert_array_equal(r["x"][:4], [0.5] * 4)
    np.testing.assert_allclose(r["lam"], [2e-3, 8e-3, 0.064, 1.024, 1.024 / 3], rtol=1e-15)
    np.testing.assert_array_equal(r["nu"], [4.0, 8.0, 16.0, 32.0, 2.0])
    np.testing.assert_array_equal(r["F"][:5], [7.03125] * 5)
    assert abs(r["x"][4] - (0.5 + 3.75 / 2.024)) <= 1e-15


def pin_lm_gain_ratio_branch(orc):
    """The two accept branches of the damping update lambda *= max(1/3, 1 - (2 rho - 1)^3):
      r(x) = x^2 - 4 from x0 = 1, lambda0 = 0.05: r = -3, J = 2, J^T J = D = 4, g = -6;
        delta = 6 / (4 * 1.05) = 1.428571, x1 = 2.428571, F0 = 4.5, F1 = (x1^2 - 4)^2 / 2 = 1.801124;
        predicted decrease 1/2 delta (0.05 * 4 * delta + 6) = 4.489796, rho = 0.601113:
        1 - (2 rho - 1)^3 = 0.991730 > 1/3, lambda = 0.0495865, nu = 2;
      from x0 = 1.9, lambda0 = 1: J = 3.8, D = 14.44, r = -0.39, delta = 1.482 / 28.88 = 0.051316;
        rho = 1.0089, 1 - (2 rho - 1)^3 = -0.0545 < 1/3: lambda = 1/3."""
    r = orc.lm_scalar(4.0, 1.0, 1, lambda0=0.05)
    delta = 6.0 / 4.2
    x1 = 1.0 + delta
    rho = (4.5 - 0.5 * (x1 * x1 - 4.0) ** 2) / (0.5 * delta * (0.05 * 4.0 * delta + 6.0))
    assert abs(rho - 0.601113) < 1e-6
    assert r["acc"][0] == 1 and r["nu"][0] == 2.0 and abs(r["x"][0] - x1) < 1e-15
    assert abs(r["lam"][0] - 0.0495865) < 1e-7
    r = orc.lm_scalar(4.0, 1.9, 1, lambda0=1.0)
    assert r["acc"][0] == 1 and abs(r["lam"][0] - 1.0 / 3.0) < 1e-15 and r["nu"][0] == 2.0
    assert abs(r["x"][0] - (1.9 + 1.482 / 28.88)) < 1e-15


def test_lm_rejections(orc):
    pin_lm_rejections(orc)


def test_lm_gain_ratio_branch(orc):
    pin_lm_gain_ratio_branch(orc)


# ------------------------------------------------------------------------------------------------
# Op counter: forward flops / special calls and the tangent (linearised program) counts
# ------------------------------------------------------------------------------------------------
def pin_opcounts(orc):
    """Counting rules: +, -, *, / are one forward flop each (a negation is free); in the tangent a
    sum of two input-dependent values costs 1, a product 3 (x dy + y dx) or 1 if one factor is a
    constant, a quotient 3 (2 if only the denominator depends on the input), sqrt 2, sin / cos one
    special call and one multiply.
      0: 3x3 product, both dependent: 27 multiplies + 18 adds = 45; tangent 27 * 3 + 18 = 99
      1: 3x3 product, B constant: 45; tangent 27 * 1 + 18 = 45
      2: y = sum of 5 constant-weighted inputs: 5 multiplies + 4 adds = 9; tangent 9
      3: one segment, minimal form (x = tx^2 + ty^2, theta = sqrt x, h = theta / 2, sin h, cos h,
         sc = sin h / h, s = sc cos h, c = sc^2 / 2, R = I + s[w]x + c[w]x^2, d = L (c tx, c ty, s)):
         forward: x 3, h 1, sc 1, s 1, c 2 = 8; R: c tx ty 2, R00 3, R02 1, R11 3, R12 1, R20 1,
         R21 1, R22 5 (tx^2, ty^2, +, c *, 1 -); d: 2 + 2 + 1 = 22 -> 30 flops; sqrt, sin, cos = 3.
         tangent: x 7, sqrt 2, h 1, sin 1, cos 1, sc 3, s 3, c 1 + 3 = 4 -> 22; R: 6 + 6 + 3 + 6 +
         3 + 3 + 3 + 10 = 40; d: 4 + 4 + 1 = 9 -> 71 flops; 2 special calls (the cos of sin', the
         sin of cos').
      4: sin x cos x / sqrt x: forward 2 flops + 3 special; tangent 1 + 1 + 3 + 2 + 3 = 10, 2 special.
    """
    assert orc.opcount_probe(0) == (45, 0, 99, 0)
    assert orc.opcount_probe(1) == (45, 0, 45, 0)
    assert orc.opcount_probe(2) == (9, 0, 9, 0)
    assert orc.opcount_probe(3) == (30, 3, 71, 2)
    assert orc.opcount_probe(4) == (2, 3, 10, 2)


def test_opcounts(orc):
    pin_opcounts(orc)


def pin_opcount_ik_one_segment(orc):
    """The whole 5-DoF IK cost of a 1-segment robot (no spheres, state inside every bound, theta
    below theta_max), counted by hand from the counting rules of pin_opcounts:
      tendon map: sx = sum_j u_j cos a_j from 0 (3 mult + 3 add; tangent 3 + 2), sy alike,
        k = (-2/m) / r_c (1, constant), tx = k sx, ty = k sy (2; tangent 2): 15 flops, tangent 12;
      theta^2 for the output: 3, tangent 7;
      segment transform (probe 3): 30 + 3 special, tangent 71 + 2;
      the tip frame is the segment's own (T_0 is not composed with the identity base frame): 0;
      pose rows: 6 x (difference with a constant target, times a weight) = 12, tangent 6;
      bound rows: 6 x (difference, weight times an exact 0) = 12, tangent 0;
      sum-zero row: 3 adds + weight = 4, tangent 3; curvature row inactive: 0;
      F = 1/2 sum of 14 squared rows: 14 mult + 14 add + 1 = 29; tangent: 7 dependent rows x 3
        + 6 dependent adds + 1 = 28.
    Forward 15 + 3 + 30 + 12 + 12 + 4 + 29 = 105 flops and 3 special calls; tangent
    12 + 7 + 71 + 6 + 0 + 3 + 28 = 127 flops and 2 special calls. The benchmark's
    1-segment denominator (tests/golden/opcounts.json, ik_1seg_axis) is this count."""
    from paper_2607_11340_gb300 import synth

    rb = orc.make_robot([0.1], 0.005, 0.008, nb=4)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    u = np.array([0.003, -0.001, -0.002])
    tg = np.array([0.01, 0.0, 0.09, 0.1, 0.0, 0.99, 0.0])
    assert tuple(orc.opcount_ik(rb, W, None, 1, tg, u)) == (105, 3, 127, 2)
    # without the bound and sum-zero rows (a projected trial point): the 6 bound rows (12 flops) and
    # the sum-zero row (4, tangent 3) go, and F sums 7 squared rows: 14 + 1 = 15 flops, tangent
    # 6 x 3 + 5 + 1 = 24: forward 105 - 12 - 4 - 29 + 15 = 75, tangent 127 - 3 - 28 + 24 = 120
    assert tuple(orc.opcount_ik(rb, W, None, 1, tg, u, box=False)) == (75, 3, 120, 2)


def test_opcount_ik_one_segment(orc):
    pin_opcount_ik_one_segment(orc)


def test_opcount_rodrigues_matches_forward_kinematics_part(orc):
    """Every added segment adds the same counted work (its tendon map, its transform, one more
    chain product and its penalty rows), and that increment contains one probe-3 segment and the
    chain product of the 1-segment count's tip frame with it: R Ri (R dependent, 45 / 99) and
    p + R d (9 mult + 9 add = 18; tangent 9 x 3 + 9 = 36)."""
    from paper_2607_11340_gb300 import synth

    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    c = []
    for n in (1, 2, 3):
        rb = orc.make_robot([0.1] * n, 0.005, 0.01, nb=4)
        u = np.tile([0.003, -0.001, -0.002], n)
        tg = np.array([0.0, 0.0, 0.1 * n, 1.0, 0.0, 0.0, 0.0])
        c.append(np.array(orc.opcount_ik(rb, W, None, 0, tg, u)))
    d1, d2 = c[1] - c[0], c[2] - c[1]
    np.testing.assert_array_equal(d1, d2)
    seg = np.array(orc.opcount_probe(3))
    assert np.all(d1 >= seg)
    # the increment holds one chain product (45 + 18 forward flops), which the 1-segment count lacks
    assert d1[0] >= seg[0] + 63


def test_lm_trace_and_pg_history_are_consistent(orc):
    """The recorded costs the GPU tests classify near-ties with: an LM iteration is accepted exactly
    when its trial cost is below its starting cost, the next iteration starts from the accepted
    cost; a PG step likewise, and its alpha follows the rule."""
    from paper_2607_11340_gb300 import synth

    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(33)
    u_true = synth.hexagon_states(rng, 4, 3, spec.umax)
    tg = synth.pose_targets(orc.fk(rb, u_true)[0], "pose")
    u0 = np.repeat(u_true, 4, 0) + rng.normal(0, 1.5e-3, (16, 9))
    r = orc.ik_lm(rb, W, None, 0, tg, 4, u0, 10, history=True)
    np.testing.assert_array_equal(r["acc"].astype(bool), r["Ftrial"] < r["Fstart"])
    nxt = np.where(r["acc"][:, :-1].astype(bool), r["Ftrial"][:, :-1], r["Fstart"][:, :-1])
    np.testing.assert_array_equal(r["Fstart"][:, 1:], nxt)
    u, F, h = orc.ik_pg(rb, W, None, 0, tg, 4, u0, 12, 1e-3, history=True)
    Fprev = np.concatenate([orc.ik_eval(rb, W, None, 0, tg, 4, u0)["F"][:, None], h[:, :-1, 10]], axis=1)
    acc = h[:, :, 11] < Fprev
    assert 0 < acc.mean() < 1
    np.testing.assert_array_equal(h[:, :, 10], np.where(acc, h[:, :, 11], Fprev))
    aprev = np.concatenate([np.full((16, 1), 1e-3), h[:, :-1, 9]], axis=1)
    np.testing.assert_array_equal(h[:, :, 9], np.where(acc, aprev * 1.25, aprev * 0.5))


def test_argmin_keeps_first_rounding_level_solution(orc):
    """Algorithm 1's argmin: among the refined candidates, costs at or below 1e-8 (solutions whose
    cost differences are rounding) tie, and the first of them in SelectTop order is kept; above that
    the lowest cost wins. On a redundant robot (4 segments: 8 free displacements for a 6-DoF pose)
    several candidates reach exact solutions; the pipeline is recomposed here from the oracle's own
    steps (seeds, projected gradient, SelectTop, LM) to check which one solve_ik returns."""
    from paper_2607_11340_gb300 import synth

    spec = synth.ROBOT_4SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    ik = synth.IkSpec(S=32, n_final=6, k_init=16, k_final=20)
    cfg = orc.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                       alpha0=ik.alpha0, dedup_eps=ik.dedup_eps)
    tg, _ = synth.ik_workload(spec, 6, "pose", lambda x: orc.fk(rb, x)[0], seed=34)
    res = orc.solve_ik(rb, W, None, 0, tg, cfg, extra=True)
    n_tied = 0
    for p in range(len(tg)):
        U = orc.seeds(rb, W, None, cfg.seed, p, 1, ik.S).reshape(ik.S, -1)
        U, _ = orc.ik_pg(rb, W, None, 0, tg[p:p + 1], ik.S, U, ik.k_init, ik.alpha0)
        X = U[res["cand"][p]]
        r = orc.ik_lm(rb, W, None, 0, tg[p:p + 1], len(X), X, ik.k_final)
        F = orc.ik_eval(rb, W, None, 0, tg[p:p + 1], len(X), r["u"])["F"]
        tied = np.nonzero(F <= 1e-8)[0]
        n_tied += len(tied) > 1
        want = tied[0] if len(tied) else int(np.argmin(F))
        np.testing.assert_array_equal(res["u"][p], r["u"][want])
        assert res["F"][p] == F[want]
    assert n_tied >= 3  # the rule decided between several exact solutions on most targets


def test_opcount_lm_update(orc):
    """Steps 2-5 of one LM iteration on n unknowns, counted by hand: damping of the diagonal 2n;
    Cholesky sum_j [2j (pivot) + (n-1-j)(2j+1) (column)] flops and n square roots; forward and
    back substitution sum_i (2i+1) each, n^2 + n^2; predicted decrease 5n + 1; gain ratio 2; the
    damping update 2 + 4 (t = 2 rho - 1, lambda (1 - t^3)).
      n = 1: 2 + 0 + 2 + 6 + 2 + 2 + 4 = 18 flops, 1 square root;
      n = 9: 18 + (72 + 204) + 162 + 46 + 8 = 510 flops, 9 square roots."""
    assert orc.opcount_lm_update(1) == (18, 1)
    assert orc.opcount_lm_update(9) == (510, 9)


def test_opcount_pg_step(orc):
    """The step of one projected-gradient iteration on n unknowns, counted by hand: |g|^2 as a sum
    from zero, n products and n additions; one square root; the step length alpha / |g|, one
    division; the move x - (alpha / |g|) g, n products and n subtractions: 4n + 1 flops, 1 square
    root (n = 9: 37)."""
    assert orc.opcount_pg_step(1) == (5, 1)
    assert orc.opcount_pg_step(9) == (37, 1)
