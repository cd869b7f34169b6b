"""GPU parity of the solver pieces against the FP64 oracle: counter-based seeds (bitwise),
SelectTop (bitwise on float32 keys), projected-gradient and LM iterates, and Algorithm 1 end to
end (success rate within 1 percentage point; FP64 mode reaches the oracle's solutions)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (EPS, TDT, TOL, dev_soa, first_true, host_aos, near_ties, orc_robot, orc_weights,
                      kink_or_pi, pose_operand_scale, rowwise_rel, targets_dev)
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


@pytest.mark.parametrize("spec", [synth.ROBOT_1SEG, synth.ROBOT_3SEG])
def test_seeds_bitwise(spec):
    P, S, p0, key = 37, 70, 11, 12345
    rb = api.robot_struct(spec)
    ref = O.seeds(orc_robot(spec), orc_weights(), None, key, p0, P, S).reshape(P * S, -1)
    for prec in (lib.CR_F64, lib.CR_F32):
        out = torch.empty((spec.d, P * S), dtype=TDT[prec], device="cuda")
        lib.cr_seeds(rb, api.Scene(None).c, api.weights_struct(synth.WEIGHTS), key, p0, P, S, out)
        got = host_aos(out)
        want = ref if prec == lib.CR_F64 else ref.astype(np.float32).astype(np.float64)
        assert np.array_equal(got, want)


def test_seeds_with_spheres():
    spec = synth.ROBOT_3SEG
    P, S = 8, 64
    sph = np.array([[0.0, 0.0, 0.1, 0.02], [0.05, 0.0, 0.2, 0.02], [-0.03, 0.04, 0.15, 0.015]])
    ref = O.seeds(orc_robot(spec), orc_weights(), sph, 5, 0, P, S).reshape(P * S, -1)
    out = torch.empty((spec.d, P * S), dtype=torch.float64, device="cuda")
    lib.cr_seeds(api.robot_struct(spec), api.Scene(sph).c, api.weights_struct(synth.WEIGHTS), 5, 0, P, S, out)
    same = np.all(host_aos(out) == ref, axis=1)
    assert same.mean() >= 0.995  # a redraw decision may flip only for a sample on a sphere boundary


def test_topk_bitwise():
    rng = np.random.default_rng(200)
    P, S, d, K = 19, 100, 9, 8
    base = rng.normal(size=(6, d)) * 0.01
    u = base[rng.integers(0, 6, P * S)] + rng.uniform(-3e-5, 3e-5, (P * S, d))
    cost = rng.choice(np.linspace(0, 1, 30), P * S).astype(np.float32)
    coll = rng.choice([0.0, 0.25], P * S).astype(np.float32)
    cost[rng.integers(0, P * S, 10)] = np.nan
    for eps in (0.0, 1e-4):
        for prec in (lib.CR_F64, lib.CR_F32):
            ug = dev_soa(u, TDT[prec])
            idx = torch.empty((P, K), dtype=torch.int32, device="cuda")
            lib.cr_topk(torch.tensor(cost).cuda(), torch.tensor(coll).cuda(), ug, P, S, K, eps, idx)
            ub = host_aos(ug)
            for p in range(P):
                ref = O.topk(cost[p * S:(p + 1) * S], coll[p * S:(p + 1) * S], ub[p * S:(p + 1) * S], K, eps)
                assert np.array_equal(idx[p].cpu().numpy(), ref), (eps, prec, p)


def _ik_case(spec, kind, P, S, seed=300, spheres=None):
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose" if kind == lib.CR_TASK_IK6 else "axis", lambda x: O.fk(rbo, x)[0], seed)
    u0 = O.seeds(rbo, orc_weights(), spheres, 7, 0, P, S).reshape(P * S, -1)
    return rbo, tg, u0


@pytest.mark.parametrize("prec,steps", [(lib.CR_F64, 64), (lib.CR_F32, 64)])
def test_pg_iterates(prec, steps):
    """Stage one's projected-gradient steps (one call per step, 64 steps, 512 seeds) against the
    oracle, in two views.

    Step by step (the bound that is asserted everywhere): every GPU step k is compared with one
    oracle step from the GPU's own iterate k-1 and step length, so a difference cannot come from an
    earlier step. Steps whose outcome rounding decides are left out (computed from the oracle's own
    one-step quantities, gpu_util): (a) the accept decision within the rounding band of the deciding
    precision (near_ties), (b) a bound or curvature hinge at its kink in the starting state, (c) in
    FP32 a rotation error within 0.05 rad of pi (kink_or_pi). Bound: 1e-4 of the displacement bound
    in FP32, 1e-10 in FP64.

    Whole trajectories: each seed against the oracle's own 64-step history from the same seed, up to
    its first rounding-decided step. The normalised step x - alpha g / |g| can magnify a difference
    by several times per step (by up to 1 + alpha |H| / |g|), so rounding differences of a few steps
    can grow past the bound without any decision changing; 99 % of the seeds must stay within it."""
    spec = synth.ROBOT_3SEG
    P, S = 32, 16
    rbo, tg, u0 = _ik_case(spec, lib.CR_TASK_IK6, P, S, seed=301)
    ug = dev_soa(u0, TDT[prec])
    u0b = host_aos(ug)
    alpha = torch.full((P * S,), 1e-3, dtype=TDT[prec], device="cuda")
    F = torch.empty(P * S, dtype=TDT[prec], device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    got, alph = [], []
    for it in range(steps):
        lib.cr_pg_steps(api.robot_struct(spec), api.Scene(None).c, task, ug, alpha, F, 1)
        got.append(host_aos(ug))
        alph.append(alpha.double().cpu().numpy())
    got = np.stack(got, axis=1)  # [B][steps][d]
    alph = np.stack(alph, axis=1)  # [B][steps]: step length after each step
    d, B = spec.d, P * S
    tol = 1e-10 if prec == lib.CR_F64 else 1e-4
    scale = pose_operand_scale(spec)
    tgB = np.repeat(tg, S, 0)

    # ---- step by step: oracle steps from the GPU's iterates
    xs = np.concatenate([u0b[:, None, :], got[:, :-1]], axis=1)  # GPU state before step k
    a_s = np.concatenate([np.full((B, 1), 1e-3), alph[:, :-1]], axis=1)
    one = np.zeros((B, steps, d))
    Fs1 = np.zeros((B, steps))
    Ft1 = np.zeros((B, steps))
    for k in range(steps):
        _, _, hk = O.ik_pg(rbo, orc_weights(), None, lib.CR_TASK_IK6, tgB, 1, xs[:, k], 1, a_s[:, k], history=True)
        one[:, k] = hk[:, 0, :d]
        Ft1[:, k] = hk[:, 0, d + 2]
    Fs1 = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tgB, steps, 0), 1, xs.reshape(B * steps, d),
                    want=("F",))["F"].reshape(B, steps)
    rs1 = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tgB, steps, 0), 1, xs.reshape(B * steps, d),
                    want=("r",))["r"].reshape(B, steps, -1)
    dec1 = near_ties(Fs1, Ft1, EPS[prec], scale) | kink_or_pi(xs, spec, rs1[:, :, 3:6], prec)
    err1 = np.abs(got - one).max(axis=2) / spec.umax
    ok1 = ~dec1
    print(f"PG {'f64' if prec == lib.CR_F64 else 'f32'} step by step: {int(ok1.sum())} of {B * steps} steps compared "
          f"({int(dec1.sum())} rounding-decided left out); max error {err1[ok1].max():.2e} of the bound")
    assert ok1.mean() >= 0.7  # late steps of converged seeds are mostly ties (about 80 % compared)
    assert err1[ok1].max() <= tol, np.sort(err1[ok1])[-5:]

    # ---- whole trajectories against the oracle's own history
    _, _, h = O.ik_pg(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, S, u0b, steps, 1e-3, history=True)
    F0 = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, S, u0b)["F"]
    Fstart = np.concatenate([F0[:, None], h[:, :-1, d + 1]], axis=1)
    xstart = np.concatenate([u0b[:, None, :], h[:, :-1, :d]], axis=1)
    rs = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tg, S, 0).repeat(steps, 0), 1,
                   xstart.reshape(B * steps, d), want=("r",))["r"].reshape(B, steps, -1)
    tie = near_ties(Fstart, h[:, :, d + 2], EPS[prec], scale)
    ill = kink_or_pi(xstart, spec, rs[:, :, 3:6], prec)
    first = first_true(tie | ill)
    checked = np.arange(steps)[None, :] < first[:, None]
    err = np.abs(got - h[:, :, :d]).max(axis=2) / spec.umax
    seed_ok = np.all(~checked | (err <= tol), axis=1)
    print(f"PG {'f64' if prec == lib.CR_F64 else 'f32'} trajectories: {int(checked.sum())} steps compared up to the first "
          f"rounding-decided one; {int(seed_ok.sum())} of {B} seeds within the bound throughout (max error "
          f"{err[checked].max():.2e}); seeds stopped by a decision tie {int((first_true(tie) < steps).sum())}, by a "
          f"kink / near-pi start {int((first_true(ill) < steps).sum())}")
    assert checked.sum() >= 0.5 * checked.size
    assert seed_ok.mean() >= 0.99


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_lm_iterates(prec):
    """20 LM iterations, one call per iteration, against the oracle's iterate history. A seed is
    compared at every iteration up to the first one whose outcome rounding decides (as in
    test_pg_iterates: a decision within the rounding band of the precision that takes it, FP64 or
    the bulk form's FP32; a hinge at its kink; in FP32 a rotation error near pi). Bound at every
    compared iteration of every seed: 1e-4 of the displacement bound (FP32 bulk, FP64 Cholesky),
    1e-10 (FP64)."""
    spec = synth.ROBOT_3SEG
    P, S, iters = 32, 4, 20
    rbo = orc_robot(spec)
    rng = np.random.default_rng(302)
    u_true = synth.hexagon_states(rng, P, 3, spec.umax)
    tg = synth.pose_targets(O.fk(rbo, u_true)[0], "pose")
    u0 = np.repeat(u_true, S, 0) + rng.normal(0, 1.5e-3, (P * S, 9))
    ug = dev_soa(u0, TDT[prec])
    u0b = host_aos(ug)
    lam = torch.full((P * S,), 1e-3, dtype=torch.float64, device="cuda")
    nu = torch.full((P * S,), 2.0, dtype=torch.float64, device="cuda")
    task = api.task_struct(lib.CR_TASK_IK6, targets_dev(tg), S, synth.WEIGHTS)
    ref = O.ik_lm(rbo, orc_weights(), None, lib.CR_TASK_IK6, tg, S, u0b, iters, history=True)
    errs = []
    for it in range(iters):
        lib.cr_lm_step(api.robot_struct(spec), api.Scene(None).c, task, ug, lam, nu, n_iter=1)
        errs.append(np.abs(host_aos(ug) - ref["hist"][it]).max(axis=1) / spec.umax)
    err = np.array(errs).T  # [B][iters]
    B = P * S
    xstart = np.concatenate([u0b[:, None, :], ref["hist"][:-1].transpose(1, 0, 2)], axis=1)  # [B][iters][d]
    rs = O.ik_eval(rbo, orc_weights(), None, lib.CR_TASK_IK6, np.repeat(tg, S, 0).repeat(iters, 0), 1,
                   xstart.reshape(B * iters, -1), want=("r",))["r"].reshape(B, iters, -1)
    tie = near_ties(ref["Fstart"], ref["Ftrial"], EPS[prec], pose_operand_scale(spec))
    first = first_true(tie | kink_or_pi(xstart, spec, rs[:, :, 3:6], prec))
    checked = np.arange(iters)[None, :] < first[:, None]
    tol = 1e-10 if prec == lib.CR_F64 else 1e-4
    excl = int((first < iters).sum())
    print(f"LM {'f64' if prec == lib.CR_F64 else 'f32'}: max error {err[checked].max():.2e} of the bound over "
          f"{int(checked.sum())} compared iterations; {excl} of {len(first)} seeds reach a near-tie "
          f"(median first at iteration {np.median(first[first < iters]) if excl else '-'}); "
          f"error of those after it: max {err[~checked].max() if (~checked).any() else 0:.2e}")
    assert err[checked].max() <= tol, np.sort(err[checked])[-5:]
    assert checked[:, 0].mean() >= 0.9  # the first iteration is compared for (almost) every seed
    assert np.mean(ref["F"] < 1e-12) > 0.5  # most seeds converge in 20 iterations


def _solve(spec, ik, kind, tg, prec, plain=False, spheres=None, p0=0):
    s = api.IkSolver(spec, ik, synth.WEIGHTS, kind, len(tg), api.Scene(spheres), prec, plain)
    s.prm.p0 = p0
    o = s.solve(targets_dev(tg), p0=p0)
    torch.cuda.synchronize()
    return dict(u=host_aos(o.u), F=o.cost.cpu().numpy(), pos=o.pos_err.cpu().numpy(),
                rot=o.rot_err.cpu().numpy(), success=o.success.cpu().numpy().astype(bool),
                status=s.status())


def _oracle_solve(spec, ik, kind, tg, spheres=None, p0=0):
    cfg = O.IkConfig(S=ik.S, n_final=ik.n_final, k_init=ik.k_init, k_final=ik.k_final, lambda0=ik.lambda0,
                     alpha0=ik.alpha0, dedup_eps=ik.dedup_eps, lim_tol=ik.lim_tol, pos_tol=ik.pos_tol,
                     rot_tol=ik.rot_tol, seed=ik.seed, p0=p0)
    return O.solve_ik(orc_robot(spec), orc_weights(), spheres, kind, tg, cfg)


def test_solve_ik_1seg_fp64_full_size():
    """The 1-segment 5-DoF workload at full size (256 targets, 32 seeds, 50 LM iterations, FP64,
    single stage): same solutions as the oracle."""
    spec, ik, P = synth.ROBOT_1SEG, synth.IK_1SEG, synth.P_1SEG
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "axis", lambda x: O.fk(rbo, x)[0], seed=0)
    g = _solve(spec, ik, lib.CR_TASK_IK5, tg, lib.CR_F64)
    o = _oracle_solve(spec, ik, lib.CR_TASK_IK5, tg)
    assert abs(g["success"].mean() - o["success"].mean()) <= 0.01
    assert g["success"].mean() >= 0.99
    close = np.abs(g["u"] - o["u"]).max(axis=1) <= 1e-9
    assert close.mean() >= 0.98
    assert g["status"] == 0


@pytest.mark.parametrize("prec", [lib.CR_F64, lib.CR_F32])
def test_solve_ik_3seg_two_stage(prec):
    spec = synth.ROBOT_3SEG
    ik = synth.IK_3SEG
    P = 48
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=3)
    g = _solve(spec, ik, lib.CR_TASK_IK6, tg, prec)
    o = _oracle_solve(spec, ik, lib.CR_TASK_IK6, tg)
    assert abs(g["success"].mean() - o["success"].mean()) <= 0.01 + 1.0 / P
    # Several candidates may converge to different exact solutions (cost ~1e-30); which one the
    # argmin keeps is then decided by rounding, so the unique part is checked instead: the
    # success flags and the validity of every GPU solution under the oracle's own acceptance.
    pos, rot, lim, col = O.accept(orc_robot(spec), None, lib.CR_TASK_IK6, tg, g["u"], ik.lim_tol)
    np.testing.assert_allclose(g["pos"], pos, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(g["rot"], rot, rtol=1e-6, atol=1e-12)
    ok = (pos <= ik.pos_tol) & (rot <= ik.rot_tol) & lim & col
    assert np.array_equal(ok, g["success"])
    if prec == lib.CR_F64:
        # where the oracle's best cost is not an exact solution the argmin is meaningful: equal costs
        sep = o["F"] > 1e-20
        np.testing.assert_allclose(g["F"][sep], o["F"][sep], rtol=1e-8)
    assert np.all(g["pos"][g["success"]] <= 1e-3)


def test_solve_ik_full_size_sampled():
    """The 3-segment two-stage workload at full size (4096 targets) in the launch configuration of
    the benchmark; a contiguous sample of 48 targets is solved by the oracle (same seed counters)."""
    spec, ik, P = synth.ROBOT_3SEG, synth.IK_3SEG, synth.P_3SEG
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=0)
    g = _solve(spec, ik, lib.CR_TASK_IK6, tg, lib.CR_F32)
    lo = 1000
    o = _oracle_solve(spec, ik, lib.CR_TASK_IK6, tg[lo:lo + 48], p0=lo)
    gs = g["success"][lo:lo + 48]
    assert np.sum(gs != o["success"]) <= 1
    assert g["success"].mean() >= o["success"].mean() - 0.01 - 1.0 / 48
    assert g["status"] == 0


def test_plain_form_matches_optimised_fp64():
    spec = synth.ROBOT_3SEG
    ik = synth.IkSpec(S=64, n_final=4, k_init=16, k_final=10)
    P = 6
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=4)
    a = _solve(spec, ik, lib.CR_TASK_IK6, tg, lib.CR_F64)
    b = _solve(spec, ik, lib.CR_TASK_IK6, tg, lib.CR_F64, plain=True)
    assert np.array_equal(a["success"], b["success"])
    np.testing.assert_allclose(b["u"], a["u"], atol=1e-10)


def test_solve_ik_ragged_and_obstacles():
    """Seeds not a multiple of the warp size, a 2-segment robot, obstacles, and a non-finite target."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=45, n_final=5, k_init=20, k_final=20)
    P = 9
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=5)
    sph = np.array([[0.03, 0.0, 0.12, 0.01], [-0.02, 0.03, 0.08, 0.008]])
    g = _solve(spec, ik, lib.CR_TASK_IK6, tg, lib.CR_F64, spheres=sph)
    o = _oracle_solve(spec, ik, lib.CR_TASK_IK6, tg, spheres=sph)
    assert np.sum(g["success"] != o["success"]) <= 1
    tg[2, 0] = np.nan
    g2 = _solve(spec, ik, lib.CR_TASK_IK6, tg, lib.CR_F32, spheres=sph)
    assert not g2["success"][2] and np.isnan(g2["F"][2])
    assert g2["status"] & (1 << lib.CR_ENONFINITE)


@pytest.mark.parametrize("K,prec", [(5, lib.CR_F64), (10, lib.CR_F64), (5, lib.CR_F32), (10, lib.CR_F32)])
def test_solve_ik_per_problem_spheres(K, prec):
    """Each target with its own sphere set, 30 targets (a partial last block), against the oracle run
    target by target with that target's spheres. FP64: one candidate per thread, 5 candidates (one
    target per warp) or 10 (three targets per warp, 2 idle lanes). FP32: 5 candidates take the
    warp-cooperative refine (one warp per candidate), 10 the packed form. One target is non-finite
    (its candidates are skipped, its result NaN and flagged)."""
    spec = synth.RobotSpec(L=(0.1, 0.08), rc=0.005, umax=0.01, nb=8)
    ik = synth.IkSpec(S=40, n_final=K, k_init=12, k_final=15)
    P, no = 30, 3
    rbo = orc_robot(spec)
    tg, _ = synth.ik_workload(spec, P, "pose", lambda x: O.fk(rbo, x)[0], seed=7)
    rng = np.random.default_rng(8)
    sph = np.concatenate([rng.uniform(-0.05, 0.05, (P, no, 2)), rng.uniform(0.05, 0.15, (P, no, 1)),
                          rng.uniform(0.005, 0.012, (P, no, 1))], axis=2)
    s = api.IkSolver(spec, ik, synth.WEIGHTS, lib.CR_TASK_IK6, P, api.Scene(sph, per_problem=True), prec)
    o = s.solve(targets_dev(tg))
    torch.cuda.synchronize()
    gu, gs = host_aos(o.u), o.success.cpu().numpy().astype(bool)
    assert s.status() == 0
    bad = tg.copy()
    bad[4, 0] = np.nan
    o2 = s.solve(targets_dev(bad))
    torch.cuda.synchronize()
    assert not o2.success[4].item() and np.isnan(o2.cost[4].item())
    assert s.status() & (1 << lib.CR_ENONFINITE)
    assert np.array_equal(o2.success.cpu().numpy().astype(bool)[5:], gs[5:])
    agree = 0
    for p in range(P):
        r = _oracle_solve(spec, ik, lib.CR_TASK_IK6, tg[p:p + 1], spheres=sph[p], p0=p)
        agree += int(bool(r["success"][0]) == gs[p])
        if r["success"][0] and gs[p]:
            pos, rot, lim, col = O.accept(rbo, sph[p], lib.CR_TASK_IK6, tg[p:p + 1], gu[p:p + 1], ik.lim_tol)
            assert lim[0] and col[0] and pos[0] <= ik.pos_tol
    assert agree >= P - 1


def test_peak_kernels_run():
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    for kind in range(4):
        assert lib.cr_peak_launch(kind, buf, 2) > 0
    torch.cuda.synchronize()
