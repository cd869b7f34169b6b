"""Pins of the oracle's complex-step derivatives: symbolic differentiation (sympy) of the
closed-form single arc, and central finite differences of the multi-segment kinematics, cost and
kinematic-parameter gradient."""
import math

import numpy as np
import pytest

from paper_2607_11340_gb300 import synth


def _robot(orc, spec):
    return orc.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb,
                          rbody=spec.body_radius)


def _weights(orc, **over):
    kw = synth.WEIGHTS.as_dict()
    kw.update(over)
    return orc.make_weights(**kw)


def test_single_segment_jacobian_vs_symbolic(orc):
    sp = pytest.importorskip("sympy")
    L, rc = 0.1, 0.005
    u0, u1, u2 = sp.symbols("u0 u1 u2", real=True)
    alpha = [0, 2 * sp.pi / 3, 4 * sp.pi / 3]
    us = [u0, u1, u2]
    tx = -sp.Rational(2, 3) / rc * sum(u * sp.cos(a) for u, a in zip(us, alpha))
    ty = -sp.Rational(2, 3) / rc * sum(u * sp.sin(a) for u, a in zip(us, alpha))
    th = sp.sqrt(tx ** 2 + ty ** 2)
    ph = sp.atan2(ty, tx)
    r = L / th
    tip = sp.Matrix([r * sp.cos(ph) * (1 - sp.cos(th)), r * sp.sin(ph) * (1 - sp.cos(th)), r * sp.sin(th)])
    axis = sp.Matrix([sp.sin(th) * sp.cos(ph), sp.sin(th) * sp.sin(ph), sp.cos(th)])
    Jp = sp.lambdify(us, tip.jacobian(us), "mpmath")
    Jz = sp.lambdify(us, axis.jacobian(us), "mpmath")
    import mpmath

    mpmath.mp.dps = 40
    rb = orc.make_robot([L], rc, 0.008)
    for u in synth.hexagon_states(np.random.default_rng(5), 8, 1, 0.008):
        J = orc.tip_jacobian(rb, u[None])[0]
        ref = np.array(Jp(*[mpmath.mpf(x) for x in u]).tolist(), dtype=float)
        np.testing.assert_allclose(J[:3], ref, rtol=1e-11, atol=1e-13)
        # world angular velocity w moves the axis as dz = w x z
        T, _ = orc.fk(rb, u[None])
        z = T[0, :9].reshape(3, 3)[:, 2]
        dz = np.cross(J[3:].T, z).T
        refz = np.array(Jz(*[mpmath.mpf(x) for x in u]).tolist(), dtype=float)
        np.testing.assert_allclose(dz, refz, rtol=1e-11, atol=1e-12)


def test_tip_jacobian_vs_central_differences(orc):
    spec = synth.ROBOT_3SEG
    rb = _robot(orc, spec)
    u = synth.hexagon_states(np.random.default_rng(6), 6, 3, spec.umax)
    J = orc.tip_jacobian(rb, u)
    h = 1e-7
    for c in range(9):
        e = np.zeros(9)
        e[c] = h
        Tp, _ = orc.fk(rb, u + e)
        Tm, _ = orc.fk(rb, u - e)
        dp = (Tp[:, 9:] - Tm[:, 9:]) / (2 * h)
        np.testing.assert_allclose(J[:, :3, c], dp, rtol=1e-6, atol=1e-7)
        Rp, Rm = Tp[:, :9].reshape(-1, 3, 3), Tm[:, :9].reshape(-1, 3, 3)
        T0, _ = orc.fk(rb, u)
        R0 = T0[:, :9].reshape(-1, 3, 3)
        W = np.einsum("bij,bkj->bik", (Rp - Rm) / (2 * h), R0)
        w = np.stack([W[:, 2, 1] - W[:, 1, 2], W[:, 0, 2] - W[:, 2, 0], W[:, 1, 0] - W[:, 0, 1]], 1) / 2
        np.testing.assert_allclose(J[:, 3:, c], w, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("kind", [0, 1])
def test_cost_gradient_vs_central_differences(orc, kind):
    """grad F (complex step, J^T r) against central differences of F (h = 1e-6, FP64), at
    states with every hinge row clearly active or inactive, including clearance rows."""
    spec = synth.ROBOT_3SEG
    rb = _robot(orc, spec)
    W = _weights(orc, rho_c=1e3)
    rng = np.random.default_rng(7)
    u_true = synth.hexagon_states(rng, 4, 3, spec.umax)
    T, bb = orc.fk(rb, u_true, backbone=True)
    tg = synth.pose_targets(T, "pose" if kind == 0 else "axis")
    # spheres sitting on backbone samples, so that clearance rows are active
    spheres = np.concatenate([bb[0, [10, 30, 40]], np.full((3, 1), 0.004)], 1)
    u = u_true + rng.normal(0, 3e-4, u_true.shape)
    u[1, 0] = 0.013  # violates the bound (seed 0 stays near its spheres)
    out = orc.ik_eval(rb, W, spheres, kind, tg, 1, u, want=("F", "g", "r"))
    h = 1e-6
    for c in range(9):
        e = np.zeros(9)
        e[c] = h
        Fp = orc.ik_eval(rb, W, spheres, kind, tg, 1, u + e)["F"]
        Fm = orc.ik_eval(rb, W, spheres, kind, tg, 1, u - e)["F"]
        fd = (Fp - Fm) / (2 * h)
        np.testing.assert_allclose(out["g"][:, c], fd, rtol=2e-5, atol=1e-6 * np.abs(out["g"]).max())
    nr = out["r"].shape[1]
    assert np.count_nonzero(out["r"][:, 6 + 18 + 6:]) > 0  # some clearance rows active


def test_param_gradient_vs_central_differences(orc):
    spec = synth.ROBOT_3SEG
    rb = _robot(orc, spec)
    W = _weights(orc)
    rng = np.random.default_rng(8)
    u = synth.hexagon_states(rng, 5, 3, spec.umax)
    T, _ = orc.fk(rb, synth.hexagon_states(rng, 5, 3, spec.umax))
    tg = synth.pose_targets(T, "pose")
    g = orc.ik_param_grad(rb, W, None, 0, tg, 1, u)
    h = 1e-7
    for q in range(6):
        def F_at(sign):
            L = list(spec.L)
            rc = [spec.rc] * 3
            if q < 3:
                L[q] += sign * h
            else:
                rc[q - 3] += sign * h
            r2 = orc.make_robot(L, rc, spec.umax, nb=spec.nb)
            return orc.ik_eval(r2, W, None, 0, tg, 1, u)["F"].sum()
        fd = (F_at(1) - F_at(-1)) / (2 * h)
        assert abs(g[q] - fd) <= 1e-5 * max(abs(fd), 1e-3)
