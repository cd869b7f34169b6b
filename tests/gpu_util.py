"""Shared helpers of the GPU parity tests: oracle structs from the workload specs, SoA transfers,
and the norm-wise error measures the tolerances are stated in."""
import numpy as np
import torch

import oracle as O
from paper_2607_11340_gb300 import api, lib, synth

# FP64: 1e-12 relative; FP32: 1e-5 relative (norm-wise per state and quantity)
TOL = {lib.CR_F64: 1e-12, lib.CR_F32: 1e-5}
TDT = {lib.CR_F64: torch.float64, lib.CR_F32: torch.float32}


def orc_robot(spec: synth.RobotSpec, thmax=None):
    return O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax if thmax is None else thmax,
                        nb=spec.nb, rbody=spec.body_radius, lmin=spec.lmin, lmax=spec.lmax, coupled=spec.coupled)


def orc_weights(w: synth.WeightSpec = synth.WEIGHTS):
    return O.make_weights(**w.as_dict())


def dev_soa(x, dtype):
    """[B][k] numpy -> device [k][B]."""
    return torch.as_tensor(np.ascontiguousarray(np.asarray(x).T), dtype=dtype).cuda().contiguous()


def host_aos(t):
    """device [k][B] -> numpy [B][k] float64."""
    return t.double().cpu().numpy().T.copy()


def targets_dev(tg):
    return dev_soa(tg, torch.float64)


def rowwise_rel(gpu, ref, floor=0.0):
    """max over states of max_q |gpu - ref| / max(max_q |ref|, floor)."""
    gpu = np.asarray(gpu, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    scale = np.maximum(np.abs(ref).max(axis=1), floor)
    return np.abs(gpu - ref).max(axis=1) / scale


def edge_states(spec, rng, count):
    """Hexagon-uniform states plus the degenerate ones: straight, nearly straight, on the bound."""
    u = synth.hexagon_states(rng, count, spec.n, spec.umax)
    u[0] = 0.0
    u[1] = 1e-9 * u[2]
    u[3] = u[3] / np.abs(u[3]).max() * spec.umax
    return u


# Unit roundoff of the arithmetic that takes an accept decision (FP64, or FP32 for the bulk form).
EPS = {lib.CR_F64: 2.0 ** -53, lib.CR_F32: 2.0 ** -24}


def pose_operand_scale(spec: synth.RobotSpec, w: synth.WeightSpec = synth.WEIGHTS) -> float:
    """Magnitude of the operands whose differences form the pose rows: w_p times the reach plus
    w_R times the largest rotation angle. A residual computed in precision eps carries an absolute
    error of a modest multiple of eps times this scale, however small the residual itself."""
    reach = sum(spec.L) if spec.lmax is None else spec.n * spec.lmax
    return w.wp * reach + w.wR * np.pi


def consequential_ties(F_start, F_trial, eps, scale, tol_state, sigma_min=1.0, k=64.0):
    """near_ties whose outcome can move the iterate by more than tol_state: a step decided at a cost
    F is no longer than about |r| / sigma_min = sqrt(2 F) / sigma_min (sigma_min: a lower bound on the
    Jacobian's smallest singular value in the weighted units, 1 here, where entries are 1e2-1e3), so
    a tie between two costs below (sigma_min tol_state)^2 / 2 -- an LM that has converged to the
    rounding level -- cannot separate the iterates by more than tol_state and is not counted."""
    F_start, F_trial = np.asarray(F_start), np.asarray(F_trial)
    big = np.sqrt(2 * np.maximum(np.abs(F_start), np.abs(np.nan_to_num(F_trial)))) > sigma_min * tol_state
    return near_ties(F_start, F_trial, eps, scale, k) & big


def near_ties(F_start, F_trial, eps, scale, k=64.0):
    """Accept decisions F_trial < F_start that rounding can flip. With F = |r|^2 / 2 and each
    residual known to within k eps scale, F is known to within k eps scale |r| + (k eps scale)^2 / 2,
    so the sign of F_trial - F_start is decided by the arithmetic, not by the method, when
    |F_trial - F_start| is below the sum of the two bounds. Elementwise; NaN trials (a failed
    Cholesky on the reference side) count as ties."""
    F_start, F_trial = np.asarray(F_start), np.asarray(F_trial)
    e = k * eps * scale
    band = e * (np.sqrt(2 * np.abs(F_start)) + np.sqrt(2 * np.abs(np.nan_to_num(F_trial)))) + e * e
    return ~np.isfinite(F_trial) | (np.abs(F_trial - F_start) <= band)


def first_true(mask):
    """[B][T] -> per row the first index where mask is set (T if none)."""
    mask = np.asarray(mask, bool)
    return np.where(mask.any(axis=1), mask.argmax(axis=1), mask.shape[1])


def cost_errors(F_gpu, F_ref, r_norm, scale):
    """Errors of a least-squares cost F = |r|^2 / 2: (plain relative |dF| / F, norm-wise relative to
    the data |dF| / (F + |r| scale)). Each residual row is a difference of operands of magnitude
    up to `scale` (pose_operand_scale), which a precision of unit roundoff eps represents only to
    eps scale; F is then known to within about eps scale |r|, so its attainable relative accuracy,
    2 eps scale / |r|, degrades without bound as the residual vanishes. The norm-wise measure
    divides by the size of the data instead, and is the one bounded for every state."""
    F_gpu, F_ref, r_norm = (np.asarray(x, np.float64) for x in (F_gpu, F_ref, r_norm))
    d = np.abs(F_gpu - F_ref)
    return d / np.maximum(F_ref, 1e-300), d / (F_ref + r_norm * scale)


def grad_errors(g_gpu, g_ref, J_ref, r_norm, scale):
    """Errors of g = J^T r per state: (plain, max_q |dg| / max_q |g|; norm-wise relative to the data,
    max_q |dg| / (max_q |g| + max |J| (|r| + scale))): an error of eps scale in each residual row and
    of eps |J| in each Jacobian entry moves g by about eps |J| (scale + |r|)."""
    g_gpu, g_ref = np.asarray(g_gpu, np.float64), np.asarray(g_ref, np.float64)
    B = len(g_ref)
    d = np.abs(g_gpu - g_ref).reshape(B, -1).max(axis=1)
    gm = np.abs(g_ref).reshape(B, -1).max(axis=1)
    Jm = np.abs(np.asarray(J_ref)).reshape(B, -1).max(axis=1)
    return d / np.maximum(gm, 1e-300), d / (gm + Jm * (np.asarray(r_norm) + scale))


def kink_or_pi(states, spec: synth.RobotSpec, rot_rows, prec, k=64.0, w: synth.WeightSpec = synth.WEIGHTS):
    """Per state [..., d]: does an iteration starting there depend on rounding in a way the
    iterate comparison cannot follow? (b) a bound or curvature hinge sits at its kink to within
    k eps of its scale, so one precision may take the row as active and the other not (their
    Jacobians then differ by a whole penalty row); (c) in FP32, a rotation error within 0.05 rad of
    pi, where the FP32 SO(3) log (error ~ eps / sin(angle)) cannot resolve the axis. rot_rows: the
    oracle's rotation rows [..., 3] (w_R Log), or None for the 5-DoF task. A hinge argument of
    exactly zero (a state the projection clamped onto its bound) is on the kink in both precisions
    and is not flagged."""
    x = np.asarray(states, np.float64)
    eps = EPS[prec]
    # a state exactly on the kink (a projection's clamp) is on it in both precisions: not ambiguous
    band = lambda v, s: (np.abs(v) <= k * eps * s) & (v != 0)
    n = spec.n
    kink = np.zeros(x.shape[:-1], bool)
    for i in range(n):
        a, b_, c = x[..., 3 * i], x[..., 3 * i + 1], x[..., 3 * i + 2]
        if spec.lmin is not None:  # arc model: (theta cos phi, theta sin phi, L)
            th = np.hypot(a, b_)
            kink |= band(c - spec.lmax, spec.lmax) | band(spec.lmin - c, spec.lmax)
        else:  # tendon model: |u_ij| <= u_max on the state, theta from the inverse of Eq. 4
            if spec.coupled and i > 0:  # coupled routing: the segment bends with u_i = q_i - q_{i-1}
                a_, b2, c_ = a - x[..., 3 * i - 3], b_ - x[..., 3 * i - 2], c - x[..., 3 * i - 1]
            else:
                a_, b2, c_ = a, b_, c
            th = (2.0 / (3.0 * spec.rc)) * np.hypot(a_ - 0.5 * (b2 + c_), (np.sqrt(3.0) / 2.0) * (b2 - c_))
            # a state the FP32 projection clamped holds the FP32 bound itself, exactly on the kink
            # for that precision (inactive on both sides): not ambiguous either
            bnd = float(np.float32(spec.umax)) if prec == lib.CR_F32 else spec.umax
            for u in (a, b_, c):
                kink |= band(np.abs(u) - spec.umax, spec.umax) & (np.abs(u) != bnd)
        kink |= band(th - spec.thmax, spec.thmax)
    if rot_rows is not None and prec == lib.CR_F32:
        ang = np.linalg.norm(np.asarray(rot_rows, np.float64), axis=-1) / w.wR
        kink |= ang > np.pi - 0.05
    return kink
