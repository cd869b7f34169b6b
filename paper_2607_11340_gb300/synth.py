"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds workload definitions (robot geometry, penalty weights, solver settings) and
random-number recipes only. It contains none of the method's arithmetic. Forward kinematics,
costs and solvers live in the CUDA library and, separately, in the CPU oracle. Where an input
needs kinematics (targets = FK of random states), the caller passes the FK function in.

Recipes (all numpy PCG64, ``np.random.default_rng(seed)``):
  * in-bound tendon states: per segment, (u_1, u_2) ~ U[-b, b]^2 and u_3 = -u_1 - u_2, redrawn
    while |u_3| > b. This is uniform on the hexagon {|u_j| <= b, sum_j u_j = 0}, because the
    hexagon is a linear image of the accepted part of the square.
  * full-pose targets: FK of in-bound states, giving position plus unit quaternion (w >= 0).
  * 5-DoF targets: position plus tip axis (the third column of R).
  * spheres: centre uniform in a box, radius uniform in [r_lo, r_hi].
  * capsules and boxes: centre uniform in a box, direction / orientation uniformly random (a
    normalised Gaussian vector / quaternion), half lengths and radii uniform in ranges; shelves
    as boxes of a fixed layout.

The paper's benchmarks (1000 uniform IK targets, a 27-sphere lattice, shelf and cabinet scenes,
letter-shaped paths) are replaced by these synthetic stand-ins of the same shape.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

W_P_DEFAULT = math.pi / 0.18  # 1 mm of position error weighs as much as 1 degree of rotation


@dataclasses.dataclass(frozen=True)
class RobotSpec:
    L: tuple          # segment lengths (m)
    rc: float         # tendon radius (m)
    umax: float       # displacement bound |u| <= umax (m)
    nb: int = 16      # backbone samples per segment
    thmax: float = math.pi
    rbody: float | None = None  # backbone radius for clearance (defaults to rc)
    lmin: float | None = None   # arc model (the paper's (theta, phi, L) per segment): length bounds
    lmax: float | None = None
    coupled: bool = False       # coupled routing (model B): the state holds the actuator displacements

    @property
    def is_arc(self) -> bool:
        return self.lmin is not None

    @property
    def n(self) -> int:
        return len(self.L)

    @property
    def d(self) -> int:
        return 3 * len(self.L)

    @property
    def body_radius(self) -> float:
        return self.rc if self.rbody is None else self.rbody


@dataclasses.dataclass(frozen=True)
class WeightSpec:
    wp: float = W_P_DEFAULT
    wR: float = 1.0
    rho_b: float = 1e4
    rho_eq: float = 1e4
    rho_k: float = 1e4
    rho_c: float = 1e4
    w_s: float = 1.0
    w_len: float = 1.0
    rho_v: float = 1e4
    rho_a: float = 1e4
    dt: float = 0.05
    vmax: float = 0.05
    amax: float = 0.5
    delta: float = 1e-3
    rho_s: float = 0.0      # self-contact rows (segments two or more apart); 0 leaves them out

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass(frozen=True)
class IkSpec:
    S: int                 # seeds per target
    n_final: int           # candidates kept after stage one
    k_init: int            # stage-one projected-gradient steps
    k_final: int           # stage-two LM iterations
    lambda0: float = 1e-3
    alpha0: float = 1e-3   # first stage-one step length (m of tendon displacement)
    dedup_eps: float = 1e-4
    lim_tol: float = 1e-5
    pos_tol: float = 1e-3
    rot_tol: float = math.radians(1.0)
    seed: int = 0


# 1-segment, 3-tendon robot of the 5-DoF single-stage workload (256 targets, 32 seeds, 50 LM its).
ROBOT_1SEG = RobotSpec(L=(0.10,), rc=0.005, umax=0.008)
IK_1SEG = IkSpec(S=32, n_final=32, k_init=0, k_final=50)
P_1SEG = 256

# 3-segment, 9-tendon robot of the two-stage full-pose workload (4096 targets, 256 seeds -> 8).
ROBOT_3SEG = RobotSpec(L=(0.12, 0.10, 0.08), rc=0.005, umax=0.010)
IK_3SEG = IkSpec(S=256, n_final=8, k_init=64, k_final=30)
P_3SEG = 4096

WEIGHTS = WeightSpec()


def hexagon_states(rng: np.random.Generator, count: int, n_seg: int, umax: float) -> np.ndarray:
    """``count`` in-bound states [count, 3 n_seg], uniform on each segment's hexagon."""
    out = np.empty((count, n_seg, 3))
    for i in range(n_seg):
        filled = 0
        while filled < count:
            k = 2 * (count - filled) + 16
            a = rng.uniform(-umax, umax, size=(k, 2))
            c = -a.sum(axis=1)
            ok = np.abs(c) <= umax
            take = min(int(ok.sum()), count - filled)
            sel = np.nonzero(ok)[0][:take]
            out[filled:filled + take, i, 0:2] = a[sel]
            out[filled:filled + take, i, 2] = c[sel]
            filled += take
    return out.reshape(count, 3 * n_seg)


def rotation_to_quaternion(R: np.ndarray) -> np.ndarray:
    """Rotation matrices [N,3,3] -> unit quaternions (w, x, y, z) with w >= 0 (Shepperd)."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    q = np.empty((R.shape[0], 4))
    for b in range(R.shape[0]):
        m = R[b]
        tr = m[0, 0] + m[1, 1] + m[2, 2]
        cands = [tr, m[0, 0], m[1, 1], m[2, 2]]
        k = int(np.argmax(cands))
        if k == 0:
            s = math.sqrt(1.0 + tr) * 2
            q[b] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif k == 1:
            s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
            q[b] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif k == 2:
            s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
            q[b] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
            q[b] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
        q[b] /= np.linalg.norm(q[b])
        if q[b, 0] < 0:
            q[b] = -q[b]
    return q


def pose_targets(T12: np.ndarray, kind: str) -> np.ndarray:
    """Targets [P, 7] from FK output rows [P, 12] (R row-major, then p).

    kind "pose": position + quaternion (w >= 0); kind "axis": position + tip axis + 0.
    """
    T12 = np.asarray(T12, dtype=np.float64).reshape(-1, 12)
    R = T12[:, :9].reshape(-1, 3, 3)
    p = T12[:, 9:12]
    out = np.zeros((T12.shape[0], 7))
    out[:, :3] = p
    if kind == "pose":
        out[:, 3:7] = rotation_to_quaternion(R)
    elif kind == "axis":
        out[:, 3:6] = R[:, :, 2]
    else:
        raise ValueError(kind)
    return out


def ik_workload(robot: RobotSpec, P: int, kind: str, fk, seed: int = 0):
    """Targets for P IK problems: FK of hexagon-uniform states (seed), returns (targets, u_true).

    ``fk(u[P, d]) -> T[P, 12]`` is supplied by the caller (oracle or CUDA path).
    """
    rng = np.random.default_rng(seed)
    u_true = hexagon_states(rng, P, robot.n, robot.umax)
    T = np.asarray(fk(u_true))
    return pose_targets(T, kind), u_true


def spheres_uniform(rng: np.random.Generator, count: int, lo, hi, r_lo: float, r_hi: float):
    """``count`` spheres [count, 4]: centre uniform in the box [lo, hi], radius in [r_lo, r_hi]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = rng.uniform(lo, hi, size=(count, 3))
    r = rng.uniform(r_lo, r_hi, size=(count, 1))
    return np.concatenate([c, r], axis=1)


# Obstacle primitives (capsules, boxes): records of PRIM_DOUBLES values, the layout of the library's
# scene: kind, radius, then end points (capsule) or centre, half extents and orientation quaternion
# (w, x, y, z) (box). The paper's shelf and cabinet scenes are unions of such convex pieces.
PRIM_DOUBLES = 16
PRIM_CAPSULE, PRIM_BOX = 1, 2


def capsule_record(a, b, r: float) -> np.ndarray:
    rec = np.zeros(PRIM_DOUBLES)
    rec[0], rec[1] = PRIM_CAPSULE, r
    rec[2:5], rec[5:8] = a, b
    return rec


def box_record(c, h, q, r: float = 0.0) -> np.ndarray:
    rec = np.zeros(PRIM_DOUBLES)
    rec[0], rec[1] = PRIM_BOX, r
    rec[2:5], rec[5:8], rec[8:12] = c, h, q
    return rec


def random_quaternions(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform random rotations: normalised 4-D Gaussian vectors, w >= 0."""
    q = rng.normal(size=(count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def prims_uniform(rng: np.random.Generator, n_capsules: int, n_boxes: int, lo, hi, r_lo: float, r_hi: float,
                  half_lo: float, half_hi: float, rounded: float = 0.5) -> np.ndarray:
    """[n_capsules + n_boxes][PRIM_DOUBLES]: capsules with centre uniform in [lo, hi], a uniformly
    random direction, half length in [half_lo, half_hi] and radius in [r_lo, r_hi]; boxes with centre
    uniform in [lo, hi], half extents in [half_lo, half_hi] each, a uniformly random orientation and,
    with probability ``rounded``, an edge radius in [r_lo, r_hi] (else sharp)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = []
    for _ in range(n_capsules):
        c = rng.uniform(lo, hi)
        v = rng.normal(size=3)
        v *= rng.uniform(half_lo, half_hi) / np.linalg.norm(v)
        out.append(capsule_record(c - v, c + v, rng.uniform(r_lo, r_hi)))
    q = random_quaternions(rng, n_boxes)
    for k in range(n_boxes):
        c = rng.uniform(lo, hi)
        h = rng.uniform(half_lo, half_hi, size=3)
        r = rng.uniform(r_lo, r_hi) if rng.uniform() < rounded else 0.0
        out.append(box_record(c, h, q[k], r))
    return np.array(out).reshape(-1, PRIM_DOUBLES)


def prims_clear_of(rng: np.random.Generator, n_capsules: int, n_boxes: int, points: np.ndarray, margin_box: float,
                   r_lo: float, r_hi: float, half_lo: float, half_hi: float, clearance: float, sd,
                   max_tries: int = 100000) -> np.ndarray:
    """Primitives drawn as in ``prims_uniform`` inside the bounding box of ``points`` [M][3] dilated by
    ``margin_box``, each redrawn while its surface is closer than ``clearance`` to any of the points.
    ``sd(record, points) -> [M]`` is the caller's signed distance to the primitive's core."""
    lo = points.min(axis=0) - margin_box
    hi = points.max(axis=0) + margin_box
    out = []
    for nc, nbx in ((n_capsules, 0), (0, n_boxes)):
        got = 0
        tries = 0
        while got < nc + nbx and tries < max_tries:
            tries += 1
            rec = prims_uniform(rng, nc and 1, nbx and 1, lo, hi, r_lo, r_hi, half_lo, half_hi)[0]
            if np.min(sd(rec, points)) >= rec[1] + clearance:
                out.append(rec)
                got += 1
        if got < nc + nbx:
            raise RuntimeError("could not place the primitives")
    return np.array(out).reshape(-1, PRIM_DOUBLES)


def shelf_prims(centre, yaw: float, width: float, depth: float, height: float, n_boards: int,
                thickness: float) -> np.ndarray:
    """A shelf as boxes: two side walls, a back panel, top and bottom and n_boards - 2 boards in
    between, open towards -x in the shelf's frame (rotated by yaw about z, bottom at centre)."""
    cz, sz = math.cos(0.5 * yaw), math.sin(0.5 * yaw)
    q = np.array([cz, 0.0, 0.0, sz])
    rot = np.array([[math.cos(yaw), -math.sin(yaw), 0.0], [math.sin(yaw), math.cos(yaw), 0.0], [0.0, 0.0, 1.0]])
    centre = np.asarray(centre, dtype=np.float64)
    t = 0.5 * thickness
    parts = [((0.0, -0.5 * width + t, 0.5 * height), (0.5 * depth, t, 0.5 * height)),
             ((0.0, 0.5 * width - t, 0.5 * height), (0.5 * depth, t, 0.5 * height)),
             ((0.5 * depth - t, 0.0, 0.5 * height), (t, 0.5 * width, 0.5 * height))]
    for k in range(n_boards):
        z = t + k * (height - thickness) / max(n_boards - 1, 1)
        parts.append(((0.0, 0.0, z), (0.5 * depth, 0.5 * width, t)))
    return np.array([box_record(centre + rot @ np.array(c), h, q) for c, h in parts])


# Trajectories among shelves (stands in for the shelf scenes of Sec. V-C): per problem a shelf of
# 6 boxes (3 boards) 0.13 m from the base axis at a uniformly random azimuth, open towards the robot,
# plus capsules uniform around the robot; start and goal are the first two of 64 in-bound draws
# whose backbone clears every obstacle by r_body + delta.
N_SHELF_CAPS = 4


def shelf_traj_workload(robot: RobotSpec, P: int, clearance_cost, seed: int = 0, n_caps: int = N_SHELF_CAPS):
    """Returns u_start [P][d], goal states [P][d] and primitives [P][6 + n_caps][PRIM_DOUBLES].
    ``clearance_cost(states [M][d], prims [n][PRIM_DOUBLES]) -> [M]`` is the caller's clearance
    part of the cost (zero when every backbone sample clears every obstacle by r_body + delta)."""
    rng = np.random.default_rng(seed)
    reach = float(sum(robot.L))
    starts, goals, scenes = [], [], []
    while len(scenes) < P:
        psi = rng.uniform(0.0, 2.0 * math.pi)
        c = 0.13 * np.array([math.cos(psi), math.sin(psi), 0.0])
        shelf = shelf_prims(c, psi + math.pi, 0.22, 0.12, 0.32, 3, 0.008)
        caps = prims_uniform(rng, n_caps, 0, [-reach, -reach, 0.05], [reach, reach, reach], 0.004, 0.01, 0.02, 0.06)
        prims = np.concatenate([shelf, caps])
        cand = hexagon_states(rng, 64, robot.n, robot.umax)
        free = np.flatnonzero(np.asarray(clearance_cost(cand, prims)) == 0.0)
        if len(free) < 2:
            continue
        starts.append(cand[free[0]])
        goals.append(cand[free[1]])
        scenes.append(prims)
    return np.array(starts), np.array(goals), np.array(scenes)


# ---------------------------------------------------------------------------------------------
# Path following: 4-segment, 12-tendon robot; 512 paths of 64 waypoints; 32 spheres per path
# ---------------------------------------------------------------------------------------------
ROBOT_4SEG = RobotSpec(L=(0.10, 0.10, 0.10, 0.10), rc=0.005, umax=0.010, nb=16)
P_PATH, H_PATH, NO_PATH = 512, 64, 32
IK_PATH0 = IkSpec(S=64, n_final=8, k_init=32, k_final=30)   # the first waypoint
K_WARM, K_JOINT = 30, 20                                     # per-waypoint warm start, joint LM

# Trajectory planning: 3-segment robot; 256 problems of 32 states; 64 spheres per problem
P_TRAJ, T_TRAJ, NO_TRAJ = 256, 32, 64
IK_GOAL = IkSpec(S=64, n_final=4, k_init=32, k_final=30)     # IK to the goal pose
K_TRAJ, ALPHA_TRAJ = 100, 1e-3

# PRM initialiser of the trajectory workload (Algorithm 2): one roadmap per problem (each problem has
# its own spheres) of 256 nodes, 8 nearest neighbours, 8 interior states checked per edge, up to 8
# draws per node. The paper gives no roadmap size; these are readings.
@dataclasses.dataclass(frozen=True)
class PrmSpec:
    N: int = 256
    k: int = 8
    n_check: int = 8
    attempts: int = 8
    seed: int = 0x5052_0001


PRM_TRAJ = PrmSpec()

# Calibration: 1024 measured tip positions, noise sigma = 0.5 mm, parameters off by up to 5%
K_CALIB, SIGMA_CALIB, PERTURB_CALIB, ITERS_CALIB = 1024, 5e-4, 0.05, 20


def bezier_states(rng: np.random.Generator, P: int, H: int, n_seg: int, umax: float) -> np.ndarray:
    """[P][H][3 n_seg]: cubic Bezier curves in u-space through 4 hexagon-uniform control states,
    sampled at H uniform parameter values (a convex combination, so in bounds with sum zero)."""
    ctrl = hexagon_states(rng, 4 * P, n_seg, umax).reshape(P, 4, 3 * n_seg)
    s = np.linspace(0.0, 1.0, H)
    w = np.stack([(1 - s) ** 3, 3 * s * (1 - s) ** 2, 3 * s ** 2 * (1 - s), s ** 3], axis=1)  # [H][4]
    return np.einsum("hk,pkd->phd", w, ctrl)


def spheres_clear_of(rng: np.random.Generator, count: int, points: np.ndarray, margin_box: float,
                     r_lo: float, r_hi: float, clearance: float, max_tries: int = 100000) -> np.ndarray:
    """``count`` spheres [count][4] with centres uniform in the bounding box of ``points`` [M][3]
    dilated by ``margin_box``, radius uniform in [r_lo, r_hi], each redrawn while its surface is
    closer than ``clearance`` to any of the points."""
    lo = points.min(axis=0) - margin_box
    hi = points.max(axis=0) + margin_box
    out = []
    tries = 0
    while len(out) < count and tries < max_tries:
        tries += 1
        c = rng.uniform(lo, hi)
        r = rng.uniform(r_lo, r_hi)
        if np.min(np.linalg.norm(points - c, axis=1)) >= r + clearance:
            out.append(np.concatenate([c, [r]]))
    if len(out) < count:
        raise RuntimeError("could not place the spheres")
    return np.array(out)


def path_workload(robot: RobotSpec, P: int, H: int, n_spheres: int, fk_backbone, seed: int = 0,
                  weights: WeightSpec = WEIGHTS):
    """Reference paths: wp [P][H][7] (position + quaternion of FK of a Bezier curve in u-space),
    the ground-truth states [P][H][d], spheres [P][n_spheres][4] clear of the ground-truth backbone
    by r_body + delta. ``fk_backbone(u [N][d]) -> (T [N][12], backbone [N][n*nb][3])``."""
    rng = np.random.default_rng(seed)
    states = bezier_states(rng, P, H, robot.n, robot.umax)
    T, bb = fk_backbone(states.reshape(P * H, -1))
    wp = pose_targets(T, "pose").reshape(P, H, 7)
    bb = np.asarray(bb).reshape(P, -1, 3)
    sph = np.stack([spheres_clear_of(rng, n_spheres, bb[p], 0.02, 0.005, 0.015,
                                     robot.body_radius + weights.delta) for p in range(P)]) if n_spheres else None
    return wp, states, sph


def traj_workload(robot: RobotSpec, P: int, n_spheres: int, fk_backbone, seed: int = 0,
                  weights: WeightSpec = WEIGHTS):
    """Trajectory problems: u_start [P][d] (uniform in bounds), goal [P][7] (full pose of FK of
    another uniform state), spheres [P][n_spheres][4] clear of the start and goal backbones."""
    rng = np.random.default_rng(seed)
    us = hexagon_states(rng, P, robot.n, robot.umax)
    ug = hexagon_states(rng, P, robot.n, robot.umax)
    T, bb = fk_backbone(np.concatenate([us, ug]))
    goal = pose_targets(np.asarray(T)[P:], "pose")
    bb = np.asarray(bb)
    sph = None
    if n_spheres:
        sph = np.stack([spheres_clear_of(rng, n_spheres, np.concatenate([bb[p], bb[P + p]]), 0.03, 0.005, 0.015,
                                         robot.body_radius + weights.delta) for p in range(P)])
    return us, goal, sph, ug


def calib_workload(robot: RobotSpec, K: int, fk_with_params, seed: int = 0, sigma: float = SIGMA_CALIB,
                   perturb: float = PERTURB_CALIB):
    """Calibration data: U [K][d] uniform in bounds, true parameters theta_true = (L, r_c) scaled by
    1 + U(-perturb, perturb) each, measured tip positions FK(U; theta_true) + N(0, sigma^2).
    ``fk_with_params(U, L [n], rc [n]) -> T [K][12]``. Returns (U, Pm, theta_true, theta_nominal)."""
    rng = np.random.default_rng(seed)
    U = hexagon_states(rng, K, robot.n, robot.umax)
    nominal = np.concatenate([np.array(robot.L, float), np.full(robot.n, robot.rc)])
    true = nominal * (1.0 + rng.uniform(-perturb, perturb, nominal.shape))
    T = np.asarray(fk_with_params(U, true[:robot.n], true[robot.n:]))
    Pm = T[:, 9:12] + rng.normal(0.0, sigma, (K, 3))
    return U, Pm, true, nominal


# Ragged serving batch: 16384 items, each an IK (H = 1) or a path with probability 1/2; segment count
# U{1..6}, waypoints U{1..128} (paths), seeds U{16..256}, spheres U{0..64}; every segment of the
# family is L = 0.10 m, r_c = 5 mm, |u| <= 10 mm.
ROBOT_FAMILY = RobotSpec(L=(0.10,) * 6, rc=0.005, umax=0.010, nb=16)
N_RAGGED = 16384
IK_RAGGED = IkSpec(S=0, n_final=8, k_init=64, k_final=30)  # S per item


def ragged_items(rng: np.random.Generator, N: int) -> np.ndarray:
    """[N][5] int: (kind 0 IK / 1 path, n, H, S, n_o) drawn from the distributions above."""
    kind = rng.integers(0, 2, N)
    n = rng.integers(1, 7, N)
    H = np.where(kind == 1, rng.integers(1, 129, N), 1)
    S = rng.integers(16, 257, N)
    no = rng.integers(0, 65, N)
    return np.stack([kind, n, H, S, no], axis=1).astype(np.int64)


def spheres_clear_fast(rng: np.random.Generator, count: int, points: np.ndarray, margin_box: float, r_lo: float,
                       r_hi: float, clearance: float) -> np.ndarray:
    """As spheres_clear_of (same distribution: centres uniform in the dilated bounding box, radii
    uniform, rejected while closer than ``clearance`` to a point), drawing candidates in blocks and
    testing them against a k-d tree of the points."""
    from scipy.spatial import cKDTree

    if count == 0:
        return np.zeros((0, 4))
    lo, hi = points.min(axis=0) - margin_box, points.max(axis=0) + margin_box
    tree = cKDTree(points)
    out = []
    for _ in range(1000):
        c = rng.uniform(lo, hi, (4 * count, 3))
        r = rng.uniform(r_lo, r_hi, 4 * count)
        d, _ = tree.query(c)
        ok = d >= r + clearance
        out.extend(np.concatenate([c[ok], r[ok, None]], axis=1))
        if len(out) >= count:
            return np.array(out[:count])
    raise RuntimeError("could not place the spheres")


def ragged_workload(N: int, fk_backbone_n, seed: int = 0, items: np.ndarray | None = None,
                    robot: RobotSpec = ROBOT_FAMILY, weights: WeightSpec = WEIGHTS):
    """Items [N][5], targets [W][7] (W = sum H; item i's waypoints follow those of item i - 1),
    spheres [sum n_o][4] (item-packed) and the ground-truth states (list of [H][3n] arrays). IK
    targets are FK poses of hexagon-uniform states, path waypoints FK poses along a Bezier curve in
    u-space; an item's spheres are clear of its ground-truth backbone by r_body + delta.
    ``fk_backbone_n(n, u [M][3n]) -> (T [M][12], backbone [M][n*nb][3])``."""
    rng = np.random.default_rng(seed)
    if items is None:
        items = ragged_items(rng, N)
    N = len(items)
    states = [None] * N
    for i, (kind, n, H, S, no) in enumerate(items):
        states[i] = (bezier_states(rng, 1, int(H), int(n), robot.umax)[0] if kind == 1
                     else hexagon_states(rng, 1, int(n), robot.umax))
    Hs = items[:, 2]
    woff = np.concatenate([[0], np.cumsum(Hs)])
    targets = np.zeros((int(woff[-1]), 7))
    backbones = [None] * N
    for n in range(1, 7):
        idx = np.nonzero(items[:, 1] == n)[0]
        if len(idx) == 0:
            continue
        U = np.concatenate([states[i] for i in idx])
        T, bb = fk_backbone_n(n, U)
        T, bb = np.asarray(T), np.asarray(bb)
        poses = pose_targets(T, "pose")
        o = 0
        for i in idx:
            h = int(Hs[i])
            targets[woff[i]:woff[i] + h] = poses[o:o + h]
            backbones[i] = bb[o:o + h].reshape(-1, 3)
            o += h
    clear = robot.body_radius + weights.delta
    sph = [spheres_clear_fast(rng, int(items[i, 4]), backbones[i], 0.02, 0.005, 0.015, clear) for i in range(N)]
    spheres = np.concatenate(sph) if sum(len(s) for s in sph) else np.zeros((0, 4))
    return items, targets, spheres, states


# ---------------------------------------------------------------------------------------------
# The paper's own IK benchmarks, arc model (Sec. V-B): segments of 1.0 m and radius 0.1 m,
# theta in [0, pi], phi in [0, 2 pi], L fixed at 1.0 m or extendable in [0.5, 1.5] m, 10 backbone
# points per segment, 128 seeds -> top 8 within a budget of 200 iterations.
# ---------------------------------------------------------------------------------------------
def arc_robot(n: int, extendable: bool) -> RobotSpec:
    lo, hi = (0.5, 1.5) if extendable else (1.0, 1.0)
    return RobotSpec(L=(1.0,) * n, rc=0.1, umax=0.01, nb=10, thmax=math.pi, rbody=0.1, lmin=lo, lmax=hi)


ROBOT_E1 = arc_robot(3, True)
ROBOT_E2_FIXED, ROBOT_E2_EXT = arc_robot(3, False), arc_robot(4, True)
P_E1, P_E2 = 1000, 100
# 200 iterations split as 150 projected-gradient steps and 50 LM iterations; the step length and the
# near-duplicate radius are in the arc state's units (rad, m)
IK_E1 = IkSpec(S=128, n_final=8, k_init=150, k_final=50, alpha0=0.05, dedup_eps=1e-3)
LATTICE_R = 0.2


def arc_states(rng: np.random.Generator, count: int, spec: RobotSpec) -> np.ndarray:
    """Configurations uniform in the paper's parameters, theta ~ U[0, theta_max], phi ~ U[0, 2 pi),
    L ~ U[lmin, lmax], as arc states (theta cos phi, theta sin phi, L) [count][3n]."""
    th = rng.uniform(0.0, spec.thmax, (count, spec.n))
    ph = rng.uniform(0.0, 2 * math.pi, (count, spec.n))
    L = rng.uniform(spec.lmin, spec.lmax, (count, spec.n))
    return np.stack([th * np.cos(ph), th * np.sin(ph), L], axis=2).reshape(count, 3 * spec.n)


def lattice_spheres(radius: float = LATTICE_R) -> np.ndarray:
    """Sec. V-B's 3 x 3 x 3 lattice of spheres of radius 0.2 m, 0.8 m apart in x and y and 1.0 m in z.
    The paper does not place it; here it is centred on the base axis at heights 1, 2 and 3 m, so the
    robot's straight configuration runs through its middle column. [27][4]"""
    g = [(x, y, z, radius) for z in (1.0, 2.0, 3.0) for y in (-0.8, 0.0, 0.8) for x in (-0.8, 0.0, 0.8)]
    return np.array(g, dtype=np.float64)


def e1_workload(spec: RobotSpec, P: int, fk, seed: int = 0):
    """Sec. V-B without obstacles: P full-pose targets from FK of uniform configurations.
    ``fk(q [N][3n]) -> T [N][12]``. Returns (targets [P][7], configurations [P][3n])."""
    rng = np.random.default_rng(seed)
    q = arc_states(rng, P, spec)
    return pose_targets(fk(q), "pose"), q


def e2_workload(spec: RobotSpec, P: int, fk_backbone, seed: int = 0, weights: WeightSpec = WEIGHTS):
    """Sec. V-B with the sphere lattice: P collision-free targets, FK of uniform configurations
    whose backbone samples all stay r_s + r_body + delta clear of every sphere (rejection).
    ``fk_backbone(q [N][3n]) -> (T [N][12], backbone [N][n*nb][3])``. Returns (targets [P][7],
    configurations [P][3n], spheres [27][4])."""
    rng = np.random.default_rng(seed)
    sph = lattice_spheres()
    reach = sph[:, 3] + spec.body_radius + weights.delta
    got_T, got_q = [], []
    while sum(len(t) for t in got_T) < P:
        q = arc_states(rng, 4 * P, spec)
        T, bb = fk_backbone(q)
        d2 = ((bb[:, :, None, :] - sph[None, None, :, :3]) ** 2).sum(-1)
        ok = (d2 >= reach[None, None, :] ** 2).all(axis=(1, 2))
        got_T.append(T[ok])
        got_q.append(q[ok])
    T = np.concatenate(got_T)[:P]
    q = np.concatenate(got_q)[:P]
    return pose_targets(T, "pose"), q, sph



# Self-contact IK (Eq. ik_coll over the robot itself): a 4-segment robot that can curl into a loop
# (up to 2 rad per segment), 1024 full-pose targets, half of them the poses of curled states whose
# segments two or more apart intersect (the solver must find another, contact-free configuration),
# half FK of hexagon-uniform states; self-contact rows weighted rho_s = 1e4.
ROBOT_SELF = RobotSpec(L=(0.10,) * 4, rc=0.005, umax=0.010, nb=8)
IK_SELF = IkSpec(S=128, n_final=8, k_init=32, k_final=30)
P_SELF = 1024
WEIGHTS_SELF = dataclasses.replace(WEIGHTS, rho_s=1e4)


def curled_states(rng: np.random.Generator, B: int, spec: RobotSpec) -> np.ndarray:
    """[B][3n] states bent in nearly one plane by 1.6-2.0 rad per segment (within the bounds at any
    azimuth; an azimuth drift of N(0, 0.08) rad per segment), so that the robot curls into a loop whose
    ends meet: the tendon displacements of
    Eq. 4, u_j = -r_c theta cos(alpha_j - phi), plus N(0, 0.2 mm) noise, re-centred to sum zero and
    clipped to the bounds."""
    n = spec.n
    u = np.zeros((B, 3 * n))
    alpha = np.array([0.0, 2 * np.pi / 3, 4 * np.pi / 3])
    for b in range(B):
        phi0 = rng.uniform(0, 2 * np.pi)
        for i in range(n):
            th = rng.uniform(1.6, 2.0)
            phi = phi0 + rng.normal(0, 0.08)
            u[b, 3 * i:3 * i + 3] = -spec.rc * th * np.cos(alpha - phi)
    u += rng.normal(0, 2e-4, u.shape)
    u -= u.reshape(B, n, 3).mean(axis=2).repeat(3, axis=1)
    return np.clip(u, -spec.umax, spec.umax)


def self_contact_workload(spec: RobotSpec, P: int, fk, seed: int = 0):
    """Targets [P][7]: the first half FK of curled states, the rest FK of hexagon-uniform states;
    returns (targets, states)."""
    rng = np.random.default_rng(seed)
    u = np.concatenate([curled_states(rng, P // 2, spec), hexagon_states(rng, P - P // 2, spec.n, spec.umax)])
    return pose_targets(fk(u), "pose"), u
