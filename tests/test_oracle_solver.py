"""Pins of the oracle's solver pieces: Cholesky, the LM iteration (Sec. IV-C), the stage-one
projection and step rule, the seed generator (SampleSeeds) and SelectTop (Algorithm 1)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from paper_2607_11340_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_cholesky_vs_numpy(orc):
    rng = np.random.default_rng(20)
    for n in (1, 3, 9, 12, 18):
        M = rng.normal(size=(n + 3, n))
        A = M.T @ M + 1e-3 * np.eye(n)
        np.testing.assert_allclose(orc.cholesky(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)
    A = -np.eye(3)
    assert orc.cholesky(A) is None


def test_lm_linear_first_step_is_damped_least_squares(orc):
    """On r(x) = A x - y one LM iteration from x0 moves by the solution of the augmented least-
    squares problem [A; sqrt(lam D)] delta = [-(A x0 - y); 0] (numpy lstsq), and the iterations
    converge to the least-squares solution."""
    rng = np.random.default_rng(21)
    A = rng.normal(size=(15, 6))
    y = rng.normal(size=15)
    x0 = rng.normal(size=6)
    lam = 1e-1
    x1, lam1, nu1, F1 = orc.lm_linear(A, y, x0, 1, lambda0=lam)
    D = np.maximum(np.diag(A.T @ A), 1e-12)
    aug = np.vstack([A, np.diag(np.sqrt(lam * D))])
    rhs = np.concatenate([-(A @ x0 - y), np.zeros(6)])
    delta = np.linalg.lstsq(aug, rhs, rcond=None)[0]
    np.testing.assert_allclose(x1, x0 + delta, rtol=1e-10, atol=1e-12)
    # a linear model is predicted exactly: gain ratio 1 -> lambda *= max(1/3, 1 - 1) = 1/3
    assert abs(lam1 - lam / 3) < 1e-15 and nu1 == 2.0
    xs = orc.lm_linear(A, y, x0, 40, lambda0=lam)[0]
    np.testing.assert_allclose(xs, np.linalg.lstsq(A, y, rcond=None)[0], rtol=1e-9, atol=1e-10)


def _ik_setup(orc):
    spec = synth.ROBOT_3SEG
    rb = orc.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    return spec, rb, W


def test_lm_monotone_and_converges_on_reachable_targets(orc):
    spec, rb, W = _ik_setup(orc)
    rng = np.random.default_rng(22)
    u_true = synth.hexagon_states(rng, 16, 3, spec.umax)
    tg = synth.pose_targets(orc.fk(rb, u_true)[0], "pose")
    u0 = orc.project(u_true.reshape(-1, 3) + rng.normal(0, 5e-4, (48, 3)), spec.umax).reshape(16, 9)
    out = orc.ik_lm(rb, W, None, 0, tg, 1, u0, 20, history=True)
    F = [orc.ik_eval(rb, W, None, 0, tg, 1, u0)["F"]]
    for it in range(20):
        F.append(orc.ik_eval(rb, W, None, 0, tg, 1, out["hist"][it])["F"])
    F = np.array(F)
    assert np.all(np.diff(F, axis=0) <= 0)
    assert np.all(F[-1] < 1e-20)


def _hexagon_closest(v, b):
    """Brute force: closest point of the hexagon {|u|<=b, sum u = 0} to v, by checking the
    plane projection (if inside) and the closest point of each of the six edges."""
    V = b * np.array([[1, 0, -1], [1, -1, 0], [0, -1, 1], [-1, 0, 1], [-1, 1, 0], [0, 1, -1]], float)
    w = v - v.mean()
    if np.all(np.abs(w) <= b + 1e-15):
        return w
    best, bd = None, np.inf
    for k in range(6):
        a, c = V[k], V[(k + 1) % 6]
        t = np.clip(np.dot(w - a, c - a) / np.dot(c - a, c - a), 0, 1)
        q = a + t * (c - a)
        dd = np.linalg.norm(w - q)
        if dd < bd:
            best, bd = q, dd
    return best


def test_projection_vs_brute_force(orc):
    rng = np.random.default_rng(23)
    b = 0.01
    v = rng.normal(0, 0.012, size=(2000, 3))
    v[:10] *= 1e-3
    u = orc.project(v, b)
    ref = np.array([_hexagon_closest(x, b) for x in v])
    np.testing.assert_allclose(u, ref, atol=1e-15)
    assert np.abs(u.sum(axis=1)).max() < 1e-17 and np.abs(u).max() <= b


def test_pg_cost_non_increasing(orc):
    spec, rb, W = _ik_setup(orc)
    rng = np.random.default_rng(24)
    tg = synth.pose_targets(orc.fk(rb, synth.hexagon_states(rng, 4, 3, spec.umax))[0], "pose")
    u = orc.seeds(rb, W, None, 0, 0, 4, 8, ).reshape(32, 9)
    F_prev = orc.ik_eval(rb, W, None, 0, tg, 8, u)["F"]
    for steps in (1, 2, 5, 10, 30):
        _, F = orc.ik_pg(rb, W, None, 0, tg, 8, u, steps, 1e-3)
        assert np.all(F <= F_prev + 0.0)
        F_prev = F
    assert np.median(F) < 0.5 * np.median(orc.ik_eval(rb, W, None, 0, tg, 8, u)["F"])


def test_splitmix64_published_outputs(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l[0] != "#"]
    for k, hx in rows:
        assert orc.splitmix64_at(0, int(k)) == int(hx, 16)


def test_seeds_uniform_on_hexagon(orc):
    """SampleSeeds: every draw is in bounds with zero sum; a chi-square test over a 2-D histogram
    of (u_1, u_2) restricted to the hexagon accepts uniformity."""
    b = 0.01
    rb = orc.make_robot([0.1], 0.005, b, nb=4)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    u = orc.seeds(rb, W, None, 7, 0, 60, 1000).reshape(-1, 3)
    assert np.abs(u).max() <= b and np.abs(u.sum(1)).max() < 1e-17
    nb = 12
    H, xe, ye = np.histogram2d(u[:, 0], u[:, 1], bins=nb, range=[[-b, b], [-b, b]])
    # exact hexagon area fraction of every cell by fine sub-sampling of the cell
    g = (np.arange(40) + 0.5) / 40
    frac = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            x = xe[i] + g[:, None] * (xe[i + 1] - xe[i])
            y = ye[j] + g[None, :] * (ye[j + 1] - ye[j])
            frac[i, j] = np.mean(np.abs(x + y) <= b)
    expect = frac / frac.sum() * len(u)
    m = expect > 20
    chi2 = ((H[m] - expect[m]) ** 2 / expect[m]).sum()
    p = stats.chi2.sf(chi2, m.sum() - 1)
    assert p > 1e-3, (chi2, m.sum(), p)


def test_seeds_are_counter_based(orc):
    """The same (seed, problem) gives the same draws whatever the batch it is drawn in."""
    spec, rb, W = _ik_setup(orc)
    a = orc.seeds(rb, W, None, 3, 0, 6, 16)
    b = orc.seeds(rb, W, None, 3, 4, 2, 16)
    assert np.array_equal(a[4:], b)
    assert not np.array_equal(a[0], a[1])


def test_seeds_avoid_spheres(orc):
    spec, rb, W = _ik_setup(orc)
    sph = np.array([[0.0, 0.0, 0.1, 0.02], [0.05, 0.0, 0.2, 0.02]])
    u = orc.seeds(rb, W, sph, 3, 0, 4, 64).reshape(-1, 9)
    _, bb = orc.fk(rb, u, backbone=True)
    reach = sph[:, 3] + spec.rc + W.delta
    d = np.linalg.norm(bb[:, :, None, :] - sph[None, None, :, :3], axis=-1)
    clear = np.all(d >= reach, axis=(1, 2))
    assert clear.mean() > 0.95


def test_topk_matches_library_sort(orc):
    """Without de-duplication SelectTop is the first k of a lexicographic sort by
    (cost, collision penalty, index) (numpy lexsort); non-finite costs rank last."""
    rng = np.random.default_rng(25)
    S, d, k = 256, 9, 8
    for trial in range(20):
        cost = rng.choice(np.linspace(0, 1, 40), S).astype(np.float32)
        coll = rng.choice([0.0, 0.5], S).astype(np.float32)
        cost[rng.integers(0, S, 3)] = np.nan
        u = rng.normal(size=(S, d))
        got = orc.topk(cost, coll, u, k, 0.0)
        key = np.where(np.isfinite(cost), cost, np.inf)
        ref = np.lexsort((np.arange(S), coll, key))[:k]
        assert np.array_equal(got, ref)


def test_topk_dedup_properties(orc):
    rng = np.random.default_rng(26)
    S, d, k, eps = 64, 9, 8, 1e-4
    base = rng.normal(size=(6, d))
    u = base[rng.integers(0, 6, S)] + rng.uniform(-3e-5, 3e-5, (S, d))
    cost = rng.uniform(size=S).astype(np.float32)
    coll = np.zeros(S, np.float32)
    got = orc.topk(cost, coll, u, k, eps)
    # six clusters: the first six picks are the best member of each cluster, in cost order
    cl = [np.argmin(np.abs(u[:, None, :] - base[None]).max(-1), axis=1)][0]
    best = sorted([min(np.nonzero(cl == c)[0], key=lambda i: cost[i]) for c in range(6)],
                  key=lambda i: cost[i])
    assert list(got[:6]) == best
    # the remaining two are the best of the rest (duplicates) in rank order
    rest = [i for i in np.argsort(cost, kind="stable") if i not in best]
    assert list(got[6:]) == rest[:2]
