"""FP64 CPU oracle of the CR-Solver hot path (test infrastructure only).

This package wraps ``cr_oracle.cpp`` (plain C++17, double precision, complex-step derivatives)
through ctypes. It is the slow reference the CUDA library is checked against: only the tests, the
smoke check and the CPU-baseline leg of the benchmark may import it. It shares no code with the
CUDA path, and the CUDA path never imports it.

Arrays here are row-major "array of structures": states ``u[B][d]`` with ``d = 3 n`` and the
tendons of segment i at ``u[:, 3 i : 3 i + 3]``; targets ``[P][7]`` = position then unit
quaternion (w, x, y, z) for full-pose IK, or position then tip axis (and a zero) for 5-DoF IK;
obstacles either spheres ``[N_o][4]`` = centre then radius, or a pair ``(spheres, prims)`` adding
primitive records ``[N_p][16]`` (``OBS`` doubles each: kind, radius, then the kind's parameters;
see ``obstacle_records``). Per-problem obstacle sets carry a leading ``[P]`` axis on both.

Functions with no independent pin say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cr_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcr_oracle.so")
# A prebuilt oracle library to load instead (the mutation tests point this at a copy of the oracle
# with one planted mistake, built in a temporary directory, to show that a pin catches it).
_SO_OVERRIDE = os.environ.get("CR_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

MAXSEG = 8
IK6, IK5 = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no fast-math, no FMA contraction)."""
    if _SO_OVERRIDE:
        return _SO_OVERRIDE
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Robot(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nb", C.c_int32), ("model", C.c_int32),
                ("L", C.c_double * MAXSEG), ("rc", C.c_double * MAXSEG),
                ("umax", C.c_double * MAXSEG), ("thmax", C.c_double * MAXSEG),
                ("rbody", C.c_double), ("lmin", C.c_double * MAXSEG), ("lmax", C.c_double * MAXSEG)]


MODEL_TENDON, MODEL_ARC, MODEL_COUPLED = 0, 1, 2


class Weights(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("wp", "wR", "rho_b", "rho_eq", "rho_k", "rho_c", "w_s", "w_len", "rho_v",
                 "rho_a", "dt", "vmax", "amax", "delta", "rho_s")]


class IkParams(C.Structure):
    _fields_ = [("S", C.c_int32), ("n_final", C.c_int32), ("k_init", C.c_int32),
                ("k_final", C.c_int32), ("lambda0", C.c_double), ("alpha0", C.c_double),
                ("dedup_eps", C.c_double), ("lim_tol", C.c_double), ("pos_tol", C.c_double),
                ("rot_tol", C.c_double), ("seed", C.c_uint64), ("p0", C.c_int64)]


def make_robot(L, rc, umax, thmax=None, nb=16, rbody=None, m=3, lmin=None, lmax=None, coupled=False) -> Robot:
    """Tendon model; with lmin/lmax given, the arc model (per segment (theta cos phi, theta sin phi,
    L) with lmin <= L <= lmax; L then only sets the nominal length); with coupled, the tendon model
    with coupled routing (the state holds the actuator displacements, model B)."""
    n = len(L)
    r = Robot()
    r.n, r.m, r.nb = n, m, nb
    r.model = MODEL_ARC if lmin is not None else (MODEL_COUPLED if coupled else MODEL_TENDON)
    if lmin is not None:
        lmin = list(lmin) if np.ndim(lmin) else [lmin] * n
        lmax = list(lmax) if np.ndim(lmax) else [lmax] * n
        for i in range(n):
            r.lmin[i], r.lmax[i] = lmin[i], lmax[i]
    rc = list(rc) if np.ndim(rc) else [rc] * n
    umax = list(umax) if np.ndim(umax) else [umax] * n
    thmax = [np.pi] * n if thmax is None else (list(thmax) if np.ndim(thmax) else [thmax] * n)
    for i in range(n):
        r.L[i], r.rc[i], r.umax[i], r.thmax[i] = L[i], rc[i], umax[i], thmax[i]
    r.rbody = rc[0] if rbody is None else rbody
    return r


def make_weights(**kw) -> Weights:
    """Weights from keyword values; rho_s (the self-contact rows) defaults to 0 (rows left out)."""
    w = Weights()
    for f, _ in Weights._fields_:
        setattr(w, f, float(kw.get(f, 0.0) if f == "rho_s" else kw[f]))
    return w


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_splitmix64_at.restype = C.c_uint64
            L.orc_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
        return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _threads(threads):
    return os.cpu_count() if threads is None else threads


def fk(robot: Robot, u, backbone: bool = False):
    """Forward kinematics (Eq. 1-3 chained). Returns (T[B,12], backbone[B, n*nb, 3] or None)."""
    u = _f64(u)
    B = u.shape[0]
    T = np.zeros((B, 12))
    bb = np.zeros((B, robot.n * robot.nb, 3)) if backbone else None
    lib().orc_fk(C.byref(robot), _dp(u), C.c_int64(B), _dp(T), _dp(bb))
    return T, bb


def fk_rodrigues(robot: Robot, u):
    """Forward kinematics through the Rodrigues form of Eq. 2-3 (no backbone)."""
    u = _f64(u)
    T = np.zeros((u.shape[0], 12))
    lib().orc_fk_rodrigues(C.byref(robot), _dp(u), C.c_int64(u.shape[0]), _dp(T))
    return T


def bend(robot: Robot, u):
    """(theta_i, phi_i) of every segment from the inverse of Eq. 4: [B, n, 2]."""
    u = _f64(u)
    out = np.zeros((u.shape[0], robot.n, 2))
    lib().orc_bend(C.byref(robot), _dp(u), C.c_int64(u.shape[0]), _dp(out))
    return out


def tendon_lengths(rc, L, theta, phi, m=3):
    """Eq. 4: l_j = L - r_c theta cos(alpha_j - phi), j = 1..m."""
    out = np.zeros(m)
    lib().orc_tendon_lengths(C.c_double(rc), C.c_double(L), C.c_double(theta), C.c_double(phi),
                             C.c_int(m), _dp(out))
    return out


def tip_jacobian(robot: Robot, u):
    """Tip Jacobian [B, 6, d] by complex step: d p/d u and world angular velocity per du."""
    u = _f64(u)
    d = robot.n * robot.m
    J = np.zeros((u.shape[0], 6, d))
    lib().orc_tip_jacobian(C.byref(robot), _dp(u), C.c_int64(u.shape[0]), _dp(J))
    return J


def so3_log(E):
    E = _f64(E).reshape(-1, 9)
    w = np.zeros((E.shape[0], 3))
    lib().orc_so3_log(_dp(E), C.c_int64(E.shape[0]), _dp(w))
    return w


def quat_to_R(q):
    q = _f64(q).reshape(-1, 4)
    R = np.zeros((q.shape[0], 9))
    lib().orc_quat_to_R(_dp(q), C.c_int64(q.shape[0]), _dp(R))
    return R.reshape(-1, 3, 3)


def ik_rows(robot: Robot, n_spheres: int, weights: Weights | None = None) -> int:
    w = weights if weights is not None else make_weights(**{f: 0.0 for f, _ in Weights._fields_})
    return lib().orc_ik_rows(C.byref(robot), C.byref(w), C.c_int(n_spheres))


OBS = 16  # doubles per obstacle record
SPHERE, CAPSULE, BOX = 0, 1, 2


def obstacle_records(spheres=None, prims=None, P=None):
    """Obstacle records as the oracle reads them (Eq. ik_coll's clearance rows, with Sec. IV-C's
    convex pieces): ``[n][OBS]`` = kind, radius r, then
      sphere  (0): centre;
      capsule (1): end points a, b;
      box     (2): centre, half extents, orientation quaternion (w, x, y, z), box frame to world;
    zeros elsewhere. Spheres ``[n_o][4]`` become kind-0 records ahead of the primitive records
    ``[n_p][OBS]``. With P, both inputs carry a leading ``[P]`` axis and so does the result."""
    lead = () if P is None else (P,)
    parts = []
    if spheres is not None:
        s = _f64(spheres).reshape(lead + (-1, 4))
        rec = np.zeros(s.shape[:-1] + (OBS,))
        rec[..., 1] = s[..., 3]
        rec[..., 2:5] = s[..., 0:3]
        parts.append(rec)
    if prims is not None:
        parts.append(_f64(prims).reshape(lead + (-1, OBS)))
    if not parts:
        return np.zeros(lead + (0, OBS))
    return np.ascontiguousarray(np.concatenate(parts, axis=-2))


def obstacle_sd(record, x, gradient=False):
    """Signed distance of points x [B][3] to the core of one obstacle record [OBS] (a sphere's
    centre, a capsule's segment, a solid box), and with gradient its derivative in x [B][3]."""
    rec = _f64(record).reshape(OBS)
    x = _f64(x).reshape(-1, 3)
    sd = np.zeros(x.shape[0])
    g = np.zeros_like(x) if gradient else None
    lib().orc_obstacle_sd(_dp(rec), _dp(x), C.c_int64(x.shape[0]), _dp(sd), _dp(g))
    return (sd, g) if gradient else sd


def _split_obstacles(obs):
    if isinstance(obs, tuple):
        return obs
    return obs, None


def _spheres(obs):
    """obs: None, spheres [no][4], or (spheres or None, prims [np][OBS] or None) -> (n, records)."""
    sp, pr = _split_obstacles(obs)
    rec = obstacle_records(sp, pr)
    if rec.shape[0] == 0:
        return 0, None
    return rec.shape[0], rec


def ik_eval(robot, weights, spheres, kind, targets, S, u, want=("F",), threads=None):
    """IK residuals / cost / collision cost / gradient / Jacobian of every seed.

    ``targets[P][7]``, seed b aims at target b // S. ``want`` picks among r, F, coll, g, J.
    """
    no, sp = _spheres(spheres)
    u = _f64(u)
    tg = _f64(targets).reshape(-1, 7)
    B, d = u.shape
    nr = ik_rows(robot, no, weights)
    out = {}
    r = np.zeros((B, nr)) if "r" in want else None
    F = np.zeros(B) if "F" in want else None
    coll = np.zeros(B) if "coll" in want else None
    g = np.zeros((B, d)) if "g" in want else None
    J = np.zeros((B, nr, d)) if "J" in want else None
    lib().orc_ik_eval(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind),
                      _dp(tg), C.c_int64(S), _dp(u), C.c_int64(B), _dp(r), _dp(F), _dp(coll),
                      _dp(g), _dp(J), C.c_int(_threads(threads)))
    for k, v in (("r", r), ("F", F), ("coll", coll), ("g", g), ("J", J)):
        if v is not None:
            out[k] = v
    return out


def ik_param_grad(robot, weights, spheres, kind, targets, S, u):
    """d(sum_b F_b)/d(L_1..n, r_c,1..n) by complex step: [2n]."""
    no, sp = _spheres(spheres)
    u = _f64(u)
    tg = _f64(targets).reshape(-1, 7)
    out = np.zeros(2 * robot.n)
    lib().orc_ik_param_grad(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind),
                            _dp(tg), C.c_int64(S), _dp(u), C.c_int64(u.shape[0]), _dp(out))
    return out


def ik_lm(robot, weights, spheres, kind, targets, S, u0, iters, lambda0=1e-3, history=False,
          threads=None):
    """Run ``iters`` LM iterations per seed. Returns dict u, lam, nu, F, acc[, hist, Fstart, Ftrial]:
    with history, the iterate after every iteration [iters][B][d] and, per seed and iteration, the
    cost where the iteration started and at its trial point [B][iters] (NaN if its Cholesky failed)."""
    no, sp = _spheres(spheres)
    u = _f64(u0).copy()
    tg = _f64(targets).reshape(-1, 7)
    B, d = u.shape
    lam = np.full(B, lambda0)
    nu = np.full(B, 2.0)
    F = np.zeros(B)
    acc = np.zeros((B, iters), dtype=np.uint8)
    hist = np.zeros((iters, B, d)) if history else None
    trace = np.zeros((B, iters, 2)) if history else None
    lib().orc_ik_lm(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind), _dp(tg),
                    C.c_int64(S), _dp(u), C.c_int64(B), C.c_int(iters), _dp(lam), _dp(nu), _dp(F),
                    _dp(hist), acc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(trace),
                    C.c_int(_threads(threads)))
    out = dict(u=u, lam=lam, nu=nu, F=F, acc=acc)
    if history:
        out["hist"] = hist
        out["Fstart"] = trace[:, :, 0].copy()
        out["Ftrial"] = trace[:, :, 1].copy()
    return out


def lm_linear(A, y, x0, iters, lambda0=1e-3):
    A = _f64(A)
    y = _f64(y)
    x = _f64(x0).copy()
    lam = C.c_double(lambda0)
    nu = C.c_double(2.0)
    F = C.c_double(0.0)
    lib().orc_lm_linear(_dp(A), _dp(y), C.c_int(A.shape[0]), C.c_int(A.shape[1]), _dp(x),
                        C.c_int(iters), C.byref(lam), C.byref(nu), C.byref(F))
    return x, lam.value, nu.value, F.value


def pg_quadratic(c, b, u0, steps, alpha0):
    """The stage-one step rule on F(u) = 1/2 |u - c|^2 over per-segment hexagons (3 tendons each,
    bounds b[i]). Returns (u, F, hist) with hist [steps][3 n + 3] = iterate, alpha, F and the
    trial's cost after each step."""
    c = _f64(c)
    u = _f64(u0).copy()
    b = _f64(np.atleast_1d(b))
    F = C.c_double(0)
    hist = np.zeros((steps, u.size + 3))
    lib().orc_pg_quadratic(_dp(c), C.c_int(b.size), _dp(b), _dp(u), C.c_int(steps), C.c_double(alpha0),
                           C.byref(F), _dp(hist))
    return u, F.value, hist


def lm_scalar(a, x0, iters, lambda0=1e-3):
    """LM on r(x) = x^2 - a. Returns dict of per-iteration x, lam, nu, F (at the iteration's start), acc."""
    out = {k: np.zeros(iters) for k in ("x", "lam", "nu", "F")}
    acc = np.zeros(iters, np.uint8)
    lib().orc_lm_scalar(C.c_double(a), C.c_double(x0), C.c_int(iters), C.c_double(lambda0), _dp(out["x"]),
                        _dp(out["lam"]), _dp(out["nu"]), _dp(out["F"]), acc.ctypes.data_as(C.POINTER(C.c_uint8)))
    out["acc"] = acc
    return out


def opcount_lm_update(nx):
    """(flops, special calls) of steps 2-5 of one LM iteration on nx unknowns (no cost evaluation)."""
    out = (C.c_longlong * 2)()
    lib().orc_opcount_lm_update(C.c_int(nx), out)
    return int(out[0]), int(out[1])


def opcount_pg_step(nx):
    """(flops, special calls) of the step of one projected-gradient iteration on nx unknowns: the
    gradient norm, the step length and the move (no projection, no cost evaluation)."""
    out = (C.c_longlong * 2)()
    lib().orc_opcount_pg_step(C.c_int(nx), out)
    return int(out[0]), int(out[1])


def opcount_probe(which):
    """Op counts (fwd flop, fwd sfu, tangent flop, tangent sfu) of a small hand-countable program."""
    out = (C.c_longlong * 4)()
    if lib().orc_opcount_probe(C.c_int(which), out) != 0:
        raise ValueError(which)
    return tuple(int(v) for v in out)


def cholesky(A):
    A = _f64(A)
    Lm = np.zeros_like(A)
    rc = lib().orc_cholesky(C.c_int(A.shape[0]), _dp(A), _dp(Lm))
    return (Lm if rc == 0 else None)


def project(v, b):
    """Projection of each row of v[B][m] onto {|u_j| <= b, sum_j u_j = 0}."""
    v = _f64(v)
    u = np.zeros_like(v)
    lib().orc_project(_dp(v), C.c_int64(v.shape[0]), C.c_int(v.shape[1]), C.c_double(b), _dp(u))
    return u


def project_arc(v, thmax, lmin, lmax):
    """Arc model: projection of each row (tx, ty, L) of v[B][3] onto {|(tx, ty)| <= thmax} x
    [lmin, lmax]."""
    v = _f64(v)
    u = np.zeros_like(v)
    lib().orc_project_arc(_dp(v), C.c_int64(v.shape[0]), C.c_double(thmax), C.c_double(lmin), C.c_double(lmax),
                          _dp(u))
    return u


def ik_pg(robot, weights, spheres, kind, targets, S, u0, steps, alpha0, threads=None, history=False):
    """Stage-one projected gradient on every seed. Returns (u, F), or with history (u, F, hist):
    hist [B][steps][d + 3] = the iterate, alpha, F and the trial's cost after every step. alpha0: one
    starting step length, or one per seed."""
    no, sp = _spheres(spheres)
    u = _f64(u0).copy()
    tg = _f64(targets).reshape(-1, 7)
    F = np.zeros(u.shape[0])
    hist = np.zeros((u.shape[0], steps, u.shape[1] + 3)) if history else None
    a_per = None if np.ndim(alpha0) == 0 else np.ascontiguousarray(_f64(alpha0).reshape(-1))
    lib().orc_ik_pg(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind), _dp(tg),
                    C.c_int64(S), _dp(u), C.c_int64(u.shape[0]), C.c_int(steps),
                    C.c_double(0.0 if a_per is not None else alpha0), _dp(a_per), _dp(F), _dp(hist),
                    C.c_int(_threads(threads)))
    return (u, F, hist) if history else (u, F)


def splitmix64_at(s0: int, k: int) -> int:
    return int(lib().orc_splitmix64_at(C.c_uint64(s0), C.c_uint64(k)))


def seeds(robot, weights, spheres, base, p0, P, S):
    """SampleSeeds: hexagon-uniform seeds from the counter-based generator, [P, S, d]."""
    no, sp = _spheres(spheres)
    d = robot.n * robot.m
    u = np.zeros((P, S, d))
    lib().orc_seeds(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_uint64(base),
                    C.c_int64(p0), C.c_int64(P), C.c_int64(S), _dp(u))
    return u


def topk(cost, coll, u, k, dedup_eps):
    """SelectTop of one problem on float32 keys: indices [k] (-1 where fewer candidates)."""
    cost = np.ascontiguousarray(cost, dtype=np.float32)
    coll = np.ascontiguousarray(coll, dtype=np.float32)
    u = _f64(u)
    out = np.zeros(k, dtype=np.int32)
    lib().orc_topk(cost.ctypes.data_as(C.POINTER(C.c_float)),
                   coll.ctypes.data_as(C.POINTER(C.c_float)), _dp(u), C.c_int64(u.shape[0]),
                   C.c_int(u.shape[1]), C.c_int(k), C.c_double(dedup_eps),
                   out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


@dataclasses.dataclass
class IkConfig:
    S: int = 32
    n_final: int = 8
    k_init: int = 0
    k_final: int = 30
    lambda0: float = 1e-3
    alpha0: float = 1e-3
    dedup_eps: float = 1e-4
    lim_tol: float = 1e-5
    pos_tol: float = 1e-3
    rot_tol: float = float(np.deg2rad(1.0))
    seed: int = 0
    p0: int = 0

    def c(self) -> IkParams:
        p = IkParams()
        for f, _ in IkParams._fields_:
            setattr(p, f, getattr(self, f))
        return p


def solve_ik(robot, weights, spheres, kind, targets, cfg: IkConfig, threads=None, extra=False):
    """Algorithm 1 per target. Returns dict u, F, pos, rot, success[, cand, stage1_F]."""
    no, sp = _spheres(spheres)
    tg = _f64(targets).reshape(-1, 7)
    P = tg.shape[0]
    d = robot.n * robot.m
    u = np.zeros((P, d))
    F = np.zeros(P)
    pos = np.zeros(P)
    rot = np.zeros(P)
    suc = np.zeros(P, dtype=np.uint8)
    cand = np.zeros((P, cfg.n_final), dtype=np.int32) if extra else None
    s1 = np.zeros((P, cfg.S)) if extra else None
    lib().orc_solve_ik(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind),
                       _dp(tg), C.c_int64(P), C.byref(cfg.c()), _dp(u), _dp(F), _dp(pos),
                       _dp(rot), suc.ctypes.data_as(C.POINTER(C.c_uint8)),
                       cand.ctypes.data_as(C.POINTER(C.c_int32)) if extra else None, _dp(s1),
                       C.c_int(_threads(threads)))
    out = dict(u=u, F=F, pos=pos, rot=rot, success=suc.astype(bool))
    if extra:
        out.update(cand=cand, stage1_F=s1)
    return out


def accept(robot, spheres, kind, targets, u, tol=1e-5, self_contact=False):
    """Final acceptance metrics: (pos err m, rot err rad, limits ok, collision-free); with
    self_contact, collision-free also covers the robot's own segments two or more apart."""
    no, sp = _spheres(spheres)
    tg = _f64(targets).reshape(-1, 7)
    u = _f64(u)
    P = u.shape[0]
    pos, rot = np.zeros(P), np.zeros(P)
    lo, co = np.zeros(P, dtype=np.uint8), np.zeros(P, dtype=np.uint8)
    lib().orc_accept(C.byref(robot), C.c_int(no), _dp(sp), C.c_int(kind), _dp(tg), _dp(u),
                     C.c_int64(P), C.c_double(tol), _dp(pos), _dp(rot),
                     lo.ctypes.data_as(C.POINTER(C.c_uint8)), co.ctypes.data_as(C.POINTER(C.c_uint8)),
                     C.c_int(1 if self_contact else 0))
    return pos, rot, lo.astype(bool), co.astype(bool)


def opcount_ik(robot, weights, spheres, kind, target, u, box=True):
    """Algorithmic op counts of one IK state evaluation (Rodrigues form):
    (forward flops, forward special calls, tangent flops, tangent special calls). box=False leaves
    out the tendon model's bound and sum-zero rows (a projected trial point needs none)."""
    no, sp = _spheres(spheres)
    out = (C.c_longlong * 4)()
    lib().orc_opcount_ik_form(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), C.c_int(kind),
                              _dp(_f64(target).reshape(7)), _dp(_f64(u)), C.c_int(1 if box else 0), out)
    return tuple(int(x) for x in out)


# ---------------------------------------------------------------------------------------------
# Trajectory planning, path following, calibration
# ---------------------------------------------------------------------------------------------
def _per_problem_spheres(obs, P):
    """obs: None, spheres [P][no][4], or (spheres or None, prims [P][np][OBS] or None)
    -> (obstacles per problem, records [P][n][OBS])."""
    sp, pr = _split_obstacles(obs)
    rec = obstacle_records(sp, pr, P=P)
    if rec.shape[1] == 0:
        return 0, None
    return rec.shape[1], rec


def traj_rows(robot, n_spheres, Tn, weights=None):
    w = weights if weights is not None else make_weights(**{f: 0.0 for f, _ in Weights._fields_})
    return lib().orc_traj_rows(C.byref(robot), C.byref(w), C.c_int(n_spheres), C.c_int(Tn))


def traj_eval(robot, weights, spheres, u_start, goal, x, want=("F",), threads=None):
    """Trajectory cost F [P], gradient g [P][Tn-1][d], residuals r [P][rows].
    x: free states [P][Tn-1][d]; u_start [P][d]; goal [P][7]; spheres [P][no][4], a (spheres, prims) pair
    with a leading [P] axis on both, or None."""
    x = _f64(x)
    P, Tm1, d = x.shape
    no, sp = _per_problem_spheres(spheres, P)
    us, gl = _f64(u_start).reshape(P, d), _f64(goal).reshape(P, 7)
    F = np.zeros(P) if "F" in want else None
    g = np.zeros((P, Tm1, d)) if "g" in want else None
    r = np.zeros((P, traj_rows(robot, no, Tm1 + 1, weights))) if "r" in want else None
    rc = lib().orc_traj_eval(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(us), _dp(gl),
                             C.c_int(Tm1 + 1), _dp(x), C.c_int64(P), _dp(F), _dp(g), _dp(r),
                             C.c_int(_threads(threads)))
    assert rc == 0
    return {k: v for k, v in (("F", F), ("g", g), ("r", r)) if v is not None}


def traj_pg(robot, weights, spheres, u_start, goal, x0, steps, alpha0, threads=None):
    x = _f64(x0).copy()
    P, Tm1, d = x.shape
    no, sp = _per_problem_spheres(spheres, P)
    F = np.zeros(P)
    lib().orc_traj_pg(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(_f64(u_start)), _dp(_f64(goal)),
                      C.c_int(Tm1 + 1), _dp(x), C.c_int64(P), C.c_int(steps), C.c_double(alpha0), _dp(F),
                      C.c_int(_threads(threads)))
    return x, F


def solve_traj(robot, weights, spheres, u_start, goal, Tn, ik_cfg: "IkConfig", k_traj, alpha0, threads=None):
    us = _f64(u_start)
    P, d = us.shape
    no, sp = _per_problem_spheres(spheres, P)
    X = np.zeros((P, Tn, d))
    F, gp, gr, sv, sa = (np.zeros(P) for _ in range(5))
    lo, co = np.zeros(P, np.uint8), np.zeros(P, np.uint8)
    lib().orc_solve_traj(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(us), _dp(_f64(goal)),
                         C.c_int64(P), C.c_int(Tn), C.byref(ik_cfg.c()), C.c_int(k_traj), C.c_double(alpha0),
                         _dp(X), _dp(F), _dp(gp), _dp(gr), _dp(sv), _dp(sa),
                         lo.ctypes.data_as(C.POINTER(C.c_uint8)), co.ctypes.data_as(C.POINTER(C.c_uint8)),
                         C.c_int(_threads(threads)))
    return dict(x=X, F=F, goal_pos=gp, goal_rot=gr, speed=sv, accel=sa, lim_ok=lo.astype(bool),
                col_ok=co.astype(bool))


def traj_refine(robot, weights, spheres, u_start, goal, X0, k_traj, alpha0, lim_tol=1e-5, threads=None):
    """Refinement and metrics of orc_solve_traj from the initial states X0 [P][Tn][d]."""
    X = _f64(X0).copy()
    P, Tn, d = X.shape
    no, sp = _per_problem_spheres(spheres, P)
    F, gp, gr, sv, sa = (np.zeros(P) for _ in range(5))
    lo, co = np.zeros(P, np.uint8), np.zeros(P, np.uint8)
    lib().orc_traj_refine(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(_f64(u_start)),
                          _dp(_f64(goal)), C.c_int64(P), C.c_int(Tn), C.c_int(k_traj), C.c_double(alpha0),
                          C.c_double(lim_tol), _dp(X), _dp(F), _dp(gp), _dp(gr), _dp(sv), _dp(sa),
                          lo.ctypes.data_as(C.POINTER(C.c_uint8)), co.ctypes.data_as(C.POINTER(C.c_uint8)),
                          C.c_int(_threads(threads)))
    return dict(x=X, F=F, goal_pos=gp, goal_rot=gr, speed=sv, accel=sa, lim_ok=lo.astype(bool),
                col_ok=co.astype(bool))


# ---------------------------------------------------------------------------------------------
# PRM exploration (Algorithm 2): roadmap build and queries
# ---------------------------------------------------------------------------------------------
def _u8p(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _i32p(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _sph_flat(spheres):
    """PRM obstacles: spheres [no][4] only."""
    if isinstance(spheres, tuple):
        raise ValueError("the PRM functions take sphere obstacles only")
    if spheres is None or len(spheres) == 0:
        return 0, None
    s = np.ascontiguousarray(_f64(spheres).reshape(-1, 4))
    return s.shape[0], s


def prm_sample(robot, delta, spheres, key, r, N, attempts):
    """ParallelSample of roadmap r: nodes [N][d], ok [N] (bool)."""
    d = robot.n * robot.m
    no, sp = _sph_flat(spheres)
    nodes = np.zeros((N, d))
    ok = np.zeros(N, np.uint8)
    lib().orc_prm_sample(C.byref(robot), C.c_double(delta), C.c_int(no), _dp(sp), C.c_uint64(key), C.c_int64(r),
                         C.c_int(N), C.c_int(attempts), _dp(nodes), _u8p(ok))
    return nodes, ok.astype(bool)


def prm_knn(nodes, ok, k):
    nodes = np.ascontiguousarray(_f64(nodes))
    N, d = nodes.shape
    okb = np.ascontiguousarray(np.asarray(ok, np.uint8))
    nbr = np.zeros((N, k), np.int32)
    lib().orc_prm_knn(_dp(nodes), _u8p(okb), C.c_int(N), C.c_int(d), C.c_int(k), _i32p(nbr))
    return nbr


def prm_segment_free(robot, delta, spheres, xa, xb, n_check):
    no, sp = _sph_flat(spheres)
    return bool(lib().orc_prm_segment_free(C.byref(robot), C.c_double(delta), C.c_int(no), _dp(sp),
                                           _dp(np.ascontiguousarray(_f64(xa))), _dp(np.ascontiguousarray(_f64(xb))),
                                           C.c_int(n_check)))


def prm_connect(robot, delta, spheres, nodes, ok, nbr, n_check):
    """ParallelConnect: CSR (row [N+1], col [E], wt [E]) of the roadmap graph."""
    nodes = np.ascontiguousarray(_f64(nodes))
    N, d = nodes.shape
    k = nbr.shape[1]
    no, sp = _sph_flat(spheres)
    row = np.zeros(N + 1, np.int32)
    col = np.zeros(2 * N * k, np.int32)
    wt = np.zeros(2 * N * k)
    lib().orc_prm_connect(C.byref(robot), C.c_double(delta), C.c_int(no), _dp(sp), _dp(nodes),
                          _u8p(np.ascontiguousarray(np.asarray(ok, np.uint8))),
                          _i32p(np.ascontiguousarray(nbr, np.int32)), C.c_int(N), C.c_int(k), C.c_int(n_check),
                          _i32p(row), _i32p(col), _dp(wt))
    E = int(row[N])
    return row, col[:E].copy(), wt[:E].copy()


def prm_build(robot, delta, spheres, key, r, N, k, n_check, attempts):
    """The roadmap of Algorithm 2's offline stage: dict(nodes, ok, nbr, row, col, wt)."""
    nodes, ok = prm_sample(robot, delta, spheres, key, r, N, attempts)
    nbr = prm_knn(nodes, ok, k)
    row, col, wt = prm_connect(robot, delta, spheres, nodes, ok, nbr, n_check)
    return dict(nodes=nodes, ok=ok, nbr=nbr, row=row, col=col, wt=wt)


def prm_query(robot, delta, spheres, rm, k, n_check, u_start, u_goal, T):
    """ConnectToRoadmap, Dijkstra and ResampleLinear of one query: (X [T][d], length, hops, path)."""
    nodes = np.ascontiguousarray(_f64(rm["nodes"]))
    N, d = nodes.shape
    no, sp = _sph_flat(spheres)
    col = np.ascontiguousarray(rm["col"], np.int32)
    wt = np.ascontiguousarray(_f64(rm["wt"]))
    if len(col) == 0:
        col, wt = np.zeros(1, np.int32), np.zeros(1)
    X = np.zeros((T, d))
    length = C.c_double(0)
    hops = C.c_int32(0)
    path = np.full(N + 2, -1, np.int32)
    lib().orc_prm_query(C.byref(robot), C.c_double(delta), C.c_int(no), _dp(sp), _dp(nodes),
                        _u8p(np.ascontiguousarray(np.asarray(rm["ok"], np.uint8))),
                        _i32p(np.ascontiguousarray(rm["row"], np.int32)), _i32p(col), _dp(wt), C.c_int(N),
                        C.c_int(k), C.c_int(n_check), _dp(np.ascontiguousarray(_f64(u_start))),
                        _dp(np.ascontiguousarray(_f64(u_goal))), C.c_int(T), _dp(X), C.byref(length),
                        C.byref(hops), _i32p(path))
    return X, length.value, hops.value, path[:hops.value + 1].copy() if hops.value > 0 else path[:0].copy()


def self_rows(robot, rho_s, delta, u, gradient=False):
    """Self-contact rows r [B][rows], cost F [B] and (gradient=True) dF/du [B][d] of states u [B][d]."""
    u = np.ascontiguousarray(_f64(u).reshape(-1, robot.n * robot.m))
    B, d = u.shape
    nr = lib().orc_self_row_count(C.byref(robot))
    r = np.zeros((B, max(nr, 1)))
    F = np.zeros(B)
    g = np.zeros((B, d)) if gradient else None
    lib().orc_self_rows(C.byref(robot), C.c_double(rho_s), C.c_double(delta), _dp(u), C.c_int64(B), _dp(r), _dp(F),
                        _dp(g))
    return r[:, :nr], F, g


def routing_b_from_a(robot, u):
    """Model A per-segment displacements u [B][n m] -> model B actuator displacements q (prefix sums)."""
    u = np.ascontiguousarray(_f64(u).reshape(-1, robot.n * robot.m))
    q = np.zeros_like(u)
    lib().orc_routing_b_from_a(C.byref(robot), _dp(u), C.c_int64(len(u)), _dp(q))
    return q


def routing_b_grad(robot, g_u):
    """Gradient with respect to model B actuator displacements from the model A gradient g_u."""
    g_u = np.ascontiguousarray(_f64(g_u).reshape(-1, robot.n * robot.m))
    g_q = np.zeros_like(g_u)
    lib().orc_routing_b_grad(C.byref(robot), _dp(g_u), C.c_int64(len(g_u)), _dp(g_q))
    return g_q


def routing_a_from_b(robot, q):
    """Model B actuator displacements q [B][n m] -> model A per-segment displacements u."""
    q = np.ascontiguousarray(_f64(q).reshape(-1, robot.n * robot.m))
    u = np.zeros_like(q)
    lib().orc_routing_a_from_b(C.byref(robot), _dp(q), C.c_int64(len(q)), _dp(u))
    return u


def calibrate(robot, U, Pm, theta0, iters, lambda0=1e-3, history=False):
    """LM on theta = (L_1..n, r_c,1..n) from known displacements U [K][d] and tip positions Pm [K][3]."""
    U, Pm = _f64(U), _f64(Pm)
    th = _f64(theta0).copy()
    F = C.c_double(0)
    hist = np.zeros((iters, th.size)) if history else None
    lib().orc_calibrate(C.byref(robot), _dp(U), _dp(Pm), C.c_int(U.shape[0]), _dp(th), C.c_int(iters),
                        C.c_double(lambda0), C.byref(F), _dp(hist))
    out = dict(theta=th, F=F.value)
    if history:
        out["hist"] = hist
    return out


def calib_residual(robot, U, Pm, theta):
    """The calibration residual [3K] (tip position minus measurement per pose) at theta."""
    U, Pm = _f64(U), _f64(Pm)
    r = np.zeros(3 * U.shape[0])
    lib().orc_calib_residual(C.byref(robot), _dp(U), _dp(Pm), C.c_int(U.shape[0]), _dp(_f64(theta)), _dp(r))
    return r


def calib_jacobian(robot, U, Pm, theta):
    U, Pm = _f64(U), _f64(Pm)
    J = np.zeros((3 * U.shape[0], 2 * robot.n))
    lib().orc_calib_jacobian(C.byref(robot), _dp(U), _dp(Pm), C.c_int(U.shape[0]), _dp(_f64(theta)), _dp(J))
    return J


def path_rows(robot, n_spheres, H, weights=None):
    w = weights if weights is not None else make_weights(**{f: 0.0 for f, _ in Weights._fields_})
    return lib().orc_path_rows(C.byref(robot), C.byref(w), C.c_int(n_spheres), C.c_int(H))


def path_residual(robot, weights, spheres, wp, x, jacobian=False):
    """One path: spheres [no][4] (or a (spheres, prims) pair) or None, wp [H][7], x [H][d] -> r (and the full J by complex step)."""
    no, sp = _spheres(spheres)
    x = _f64(x)
    H, d = x.shape
    nr = path_rows(robot, no, H, weights)
    r = np.zeros(nr)
    J = np.zeros((nr, H * d)) if jacobian else None
    lib().orc_path_residual(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(_f64(wp)), C.c_int(H),
                            _dp(x), _dp(r), _dp(J))
    return (r, J) if jacobian else r


def path_lm(robot, weights, spheres, wp, x0, iters, lambda0=1e-3, history=False):
    """Joint LM of one path from x0 [H][d]. With history: the iterates and, per iteration, the cost at
    its start and at its trial point (Fstart, Ftrial)."""
    no, sp = _spheres(spheres)
    x = _f64(x0).copy()
    H, d = x.shape
    lam, nu, F = C.c_double(lambda0), C.c_double(2.0), C.c_double(0)
    hist = np.zeros((iters, H, d)) if history else None
    acc = np.zeros(iters, np.uint8)
    trace = np.zeros((iters, 2)) if history else None
    lib().orc_path_lm(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(_f64(wp)), C.c_int(H), _dp(x),
                      C.c_int(iters), C.byref(lam), C.byref(nu), C.byref(F), _dp(hist),
                      acc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(trace))
    out = dict(x=x, lam=lam.value, nu=nu.value, F=F.value, acc=acc)
    if history:
        out["hist"] = hist
        out["Fstart"], out["Ftrial"] = trace[:, 0].copy(), trace[:, 1].copy()
    return out


def solve_path(robot, weights, spheres, wp, ik_cfg: "IkConfig", k_warm, k_joint, threads=None, trace=False):
    """Path following for P paths: spheres [P][no][4] (or a per-problem (spheres, prims) pair) or None, wp [P][H][7]. With trace, also the
    start and trial costs of every LM iteration (the warm sweep waypoint by waypoint, then the joint
    stage) [P][(H-1) k_warm + k_joint][2]."""
    wp = _f64(wp)
    P, H, _ = wp.shape
    no, sp = _per_problem_spheres(spheres, P)
    d = robot.n * robot.m
    X = np.zeros((P, H, d))
    SX = np.zeros((P, H, d))
    F = np.zeros(P)
    pos, rot = np.zeros((P, H)), np.zeros((P, H))
    lo, co = np.zeros(P, np.uint8), np.zeros(P, np.uint8)
    TR = np.zeros((P, (H - 1) * k_warm + k_joint, 2)) if trace else None
    lib().orc_solve_path(C.byref(robot), C.byref(weights), C.c_int(no), _dp(sp), _dp(wp), C.c_int64(P), C.c_int(H),
                         C.byref(ik_cfg.c()), C.c_int(k_warm), C.c_int(k_joint), _dp(X), _dp(F), _dp(pos), _dp(rot),
                         _dp(SX), lo.ctypes.data_as(C.POINTER(C.c_uint8)), co.ctypes.data_as(C.POINTER(C.c_uint8)),
                         _dp(TR), C.c_int(_threads(threads)))
    out = dict(x=X, stage_x=SX, F=F, pos=pos, rot=rot, lim_ok=lo.astype(bool), col_ok=co.astype(bool))
    if trace:
        out["trace"] = TR
    return out
