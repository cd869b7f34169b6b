"""User-facing API over the C ABI: builds the host structs, lets torch allocate device outputs and
workspaces, and calls the library. No arithmetic of the method happens here."""
from __future__ import annotations

import dataclasses

import torch

from . import lib
from . import synth


def robot_struct(spec: synth.RobotSpec) -> lib.cr_robot:
    r = lib.cr_robot()
    r.n, r.m, r.n_b = spec.n, 3, spec.nb
    r.model = lib.CR_MODEL_ARC if spec.is_arc else (lib.CR_MODEL_COUPLED if spec.coupled else lib.CR_MODEL_TENDON)
    for i in range(spec.n):
        r.L[i] = spec.L[i]
        r.r_c[i] = spec.rc
        r.u_max[i] = spec.umax
        r.theta_max[i] = spec.thmax
        if spec.is_arc:
            r.l_min[i], r.l_max[i] = spec.lmin, spec.lmax
    r.r_body = spec.body_radius
    return r


def weights_struct(w: synth.WeightSpec) -> lib.cr_weights:
    s = lib.cr_weights()
    s.w_p, s.w_R = w.wp, w.wR
    s.rho_b, s.rho_eq, s.rho_k, s.rho_c = w.rho_b, w.rho_eq, w.rho_k, w.rho_c
    s.w_s, s.w_len, s.rho_v, s.rho_a = w.w_s, w.w_len, w.rho_v, w.rho_a
    s.dt, s.v_max, s.a_max, s.delta = w.dt, w.vmax, w.amax, w.delta
    s.rho_s = w.rho_s
    return s


class Scene:
    """Obstacles resident on the device in FP64: spheres [n_o][4] (centre, radius) and primitive
    records [n_p][CR_PRIM_DOUBLES] (capsules, boxes) shared by all problems, or [P][n_o][4] and
    [P][n_p][CR_PRIM_DOUBLES] with per_problem=True (each problem its own set)."""

    def __init__(self, spheres=None, device="cuda", per_problem=False, prims=None):
        def resident(a, width):
            if a is None or len(a) == 0:
                return None, 0
            t = torch.as_tensor(a, dtype=torch.float64, device=device)
            t = (t.reshape(t.shape[0], -1, width) if per_problem else t.reshape(-1, width)).contiguous()
            return (t, t.shape[-2]) if t.shape[-2] > 0 else (None, 0)

        self.spheres, self.n_o = resident(spheres, 4)
        self.prims, self.n_p = resident(prims, lib.CR_PRIM_DOUBLES)
        self.c = lib.cr_scene()
        self.c.spheres = self.spheres.data_ptr() if self.spheres is not None else None
        self.c.n_o = self.n_o
        self.c.prims = self.prims.data_ptr() if self.prims is not None else None
        self.c.n_p = self.n_p
        self.c.per_problem = 1 if (per_problem and self.n_o + self.n_p > 0) else 0


def task_struct(kind: int, targets_soa: torch.Tensor, S: int, weights: synth.WeightSpec) -> lib.cr_task:
    """targets_soa: device FP64 [7][P]. The struct keeps a reference to the tensor, so the device
    memory its pointer names stays allocated while the struct is alive."""
    if targets_soa.dtype != torch.float64 or not targets_soa.is_cuda or not targets_soa.is_contiguous():
        raise ValueError("targets must be a contiguous CUDA float64 tensor [7][P]")
    t = lib.cr_task()
    t._targets = targets_soa
    t.kind = kind
    t.seeds_per_target = S
    t.targets = targets_soa.data_ptr()
    t.n_targets = targets_soa.shape[1]
    t.w = weights_struct(weights)
    return t


def ik_params_struct(spec: synth.IkSpec, precision: int = lib.CR_F32, p0: int = 0) -> lib.cr_ik_params:
    p = lib.cr_ik_params()
    p.S, p.n_final, p.k_init, p.k_final = spec.S, spec.n_final, spec.k_init, spec.k_final
    p.lambda0, p.alpha0, p.dedup_eps = spec.lambda0, spec.alpha0, spec.dedup_eps
    p.lim_tol, p.pos_tol, p.rot_tol = spec.lim_tol, spec.pos_tol, spec.rot_tol
    p.seed, p.p0, p.precision, p.reserved = spec.seed, p0, precision, 0
    return p


def _soa(x, dtype, device="cuda"):
    """[B][k] host/array -> device [k][B]."""
    return torch.as_tensor(x, dtype=dtype).T.contiguous().to(device)


def fk(robot: lib.cr_robot, u: torch.Tensor, backbone: bool = False):
    """u [d][B] (float32/float64, CUDA) -> (T [12][B], backbone [n*n_b][3][B] or None)."""
    B = u.shape[1]
    T = torch.empty((12, B), dtype=u.dtype, device=u.device)
    bb = torch.empty((robot.n * robot.n_b, 3, B), dtype=u.dtype, device=u.device) if backbone else None
    lib.cr_fk(robot, u, T, bb)
    return T, bb


def fk_jac(robot: lib.cr_robot, u: torch.Tensor):
    J = torch.empty((6, u.shape[0], u.shape[1]), dtype=u.dtype, device=u.device)
    lib.cr_fk_jac(robot, u, J)
    return J


def cost_grad(robot, scene: Scene, task, u: torch.Tensor, grad: bool = True, param_grad: bool = False,
              coll: bool = False):
    B = u.shape[1]
    cost = torch.empty(B, dtype=u.dtype, device=u.device)
    cl = torch.empty(B, dtype=u.dtype, device=u.device) if coll else None
    gu = torch.empty_like(u) if (grad or param_grad) else None
    gp = torch.empty((2 * robot.n, B), dtype=u.dtype, device=u.device) if param_grad else None
    lib.cr_cost_grad(robot, scene.c, task, u, cost, cl, gu, gp)
    return cost, cl, gu, gp


def reduce_rows(x: torch.Tensor) -> torch.Tensor:
    out = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
    lib.cr_reduce_rows(x, out)
    return out


@dataclasses.dataclass
class IkResult:
    u: torch.Tensor        # [d][P] FP64
    cost: torch.Tensor     # [P]
    pos_err: torch.Tensor  # [P] m
    rot_err: torch.Tensor  # [P] rad
    success: torch.Tensor  # [P] uint8


class IkSolver:
    """Algorithm 1 for batches of P targets; owns its device workspace and outputs."""

    def __init__(self, robot_spec: synth.RobotSpec, ik_spec: synth.IkSpec, weights: synth.WeightSpec,
                 kind: int, P: int, scene: Scene | None = None, precision: int = lib.CR_F32,
                 plain: bool = False, device="cuda"):
        self.robot = robot_struct(robot_spec)
        self.weights = weights
        self.kind = kind
        self.P = P
        self.scene = scene or Scene(None)
        self.plain = plain
        self.prm = ik_params_struct(ik_spec, lib.CR_F64 if plain else precision)
        d = robot_spec.d
        nbytes = lib.cr_ik_workspace_size(self.robot, P, self.prm)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.out = IkResult(torch.empty((d, P), dtype=torch.float64, device=device),
                            torch.empty(P, dtype=torch.float64, device=device),
                            torch.empty(P, dtype=torch.float64, device=device),
                            torch.empty(P, dtype=torch.float64, device=device),
                            torch.empty(P, dtype=torch.uint8, device=device))

    def solve(self, targets_soa: torch.Tensor, p0: int = 0) -> IkResult:
        """targets_soa: device FP64 [7][P]."""
        task = task_struct(self.kind, targets_soa, 1, self.weights)
        self._task = task
        self.prm.p0 = p0
        o = self.out
        f = lib.cr_solve_ik_plain if self.plain else lib.cr_solve_ik
        f(self.robot, self.scene.c, task, self.prm, o.u, o.cost, o.pos_err, o.rot_err, o.success, self.workspace)
        return o

    def stage1(self, targets_soa: torch.Tensor, p0: int = 0):
        """Exploration only (SampleSeeds, projected gradient, SelectTop) into the workspace."""
        self._task = task_struct(self.kind, targets_soa, 1, self.weights)
        self.prm.p0 = p0
        lib.cr_ik_stage1(self.robot, self.scene.c, self._task, self.prm, self.workspace)

    def stage2(self) -> IkResult:
        """Refinement of the candidates stage1 left in the workspace."""
        o = self.out
        lib.cr_ik_stage2(self.robot, self.scene.c, self._task, self.prm, o.u, o.cost, o.pos_err, o.rot_err,
                         o.success, self.workspace)
        return o

    def solve_host(self, targets_host: torch.Tensor, out_host: dict | None = None, p0: int = 0) -> dict:
        """End-to-end call with host buffers: copies pinned host targets [7][P] to the device, solves,
        and copies the results back into (pinned) host tensors; returns them after a sync."""
        if not hasattr(self, "_targets_dev") or self._targets_dev.shape != targets_host.shape:
            self._targets_dev = torch.empty(targets_host.shape, dtype=torch.float64, device=self.workspace.device)
        self._targets_dev.copy_(targets_host, non_blocking=True)
        o = self.solve(self._targets_dev, p0)
        if out_host is None:
            out_host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                        for k, v in dataclasses.asdict(o).items()}
        for k, v in dataclasses.asdict(o).items():
            out_host[k].copy_(v, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return out_host

    def pg_accepted(self) -> int:
        """Accepted projected-gradient steps of the last solve's stage one, over all seeds (the
        workspace counter the kernels add to; reading it synchronises the stream)."""
        return int(self.workspace[8:16].view(torch.int64).item())

    def status(self) -> int:
        return lib.cr_poll_status(self.workspace)


def solve_ik(robot_spec, ik_spec, weights, kind, targets_soa, scene=None, precision=lib.CR_F32, plain=False):
    s = IkSolver(robot_spec, ik_spec, weights, kind, targets_soa.shape[1], scene, precision, plain,
                 device=targets_soa.device)
    return s.solve(targets_soa)


# ---------------------------------------------------------------------------------------------
# Differentiation: the hand-written adjoint behind torch.autograd.Function (recompute-in-backward)
# ---------------------------------------------------------------------------------------------
class IkCost(torch.autograd.Function):
    """Per-state IK cost F_b(u_b; L, r_c). forward(u [d][B], L [n], r_c [n], ctx_data) -> cost [B].

    backward recomputes the forward sweep inside the adjoint kernel (nothing but the inputs is
    saved) and returns dF/du (scaled by the upstream gradient) and sum_b upstream_b dF_b/d(L, r_c).
    ``ctx_data`` = (RobotSpec, Scene, task struct); L and r_c are host tensors (small).
    """

    @staticmethod
    def forward(ctx, u, L, rc, ctx_data):
        spec, scene, task = ctx_data
        robot = robot_struct(spec)
        for i in range(spec.n):
            robot.L[i] = float(L[i])
            robot.r_c[i] = float(rc[i])
        cost = torch.empty(u.shape[1], dtype=u.dtype, device=u.device)
        lib.cr_cost_grad(robot, scene.c, task, u.contiguous(), cost)
        ctx.save_for_backward(u)
        ctx.robot, ctx.scene, ctx.task, ctx.n = robot, scene, task, spec.n
        ctx.param_dtype, ctx.param_device = L.dtype, L.device
        return cost

    @staticmethod
    def backward(ctx, gcost):
        (u,) = ctx.saved_tensors
        gu = torch.empty_like(u)
        gp = torch.empty(2 * ctx.n, dtype=torch.float64, device=u.device)
        ws = torch.empty((2 * ctx.n, u.shape[1]), dtype=u.dtype, device=u.device)
        lib.cr_cost_vjp(ctx.robot, ctx.scene.c, ctx.task, u.contiguous(), gcost.contiguous().to(u.dtype), gu, gp, ws)
        gp = gp.to(ctx.param_device, ctx.param_dtype)
        return gu, gp[:ctx.n], gp[ctx.n:], None


class TrajCost(torch.autograd.Function):
    """Trajectory cost per problem: forward(x [d][P*(T-1)], ctx_data) -> cost [P] (free states only;
    u_0 = u_start is fixed). backward recomputes the kinematics in the adjoint kernel."""

    @staticmethod
    def forward(ctx, x, ctx_data):
        robot, scene, task = ctx_data
        cost = torch.empty(task.P, dtype=x.dtype, device=x.device)
        lib.cr_traj_cost(robot, scene.c, task, x.contiguous(), cost)
        ctx.save_for_backward(x)
        ctx.data = ctx_data
        return cost

    @staticmethod
    def backward(ctx, gcost):
        (x,) = ctx.saved_tensors
        robot, scene, task = ctx.data
        cost = torch.empty(task.P, dtype=x.dtype, device=x.device)
        g = torch.empty_like(x)
        lib.cr_traj_cost(robot, scene.c, task, x.contiguous(), cost, g, gcost.contiguous().to(x.dtype))
        return g, None


def traj_task_struct(u_start_soa, goal_soa, T: int, weights: synth.WeightSpec) -> lib.cr_traj_task:
    """u_start_soa [d][P], goal_soa [7][P]: contiguous CUDA float64 (kept alive by the struct)."""
    t = lib.cr_traj_task()
    t._keep = (u_start_soa, goal_soa)
    t.u_start = u_start_soa.data_ptr()
    t.goal = goal_soa.data_ptr()
    t.P = u_start_soa.shape[1]
    t.T = T
    t.w = weights_struct(weights)
    return t


def prm_params_struct(spec: synth.PrmSpec) -> lib.cr_prm_params:
    p = lib.cr_prm_params()
    p.N, p.k, p.n_check, p.attempts, p.seed = spec.N, spec.k, spec.n_check, spec.attempts, spec.seed
    return p


class Roadmap:
    """R PRM roadmaps resident on the device (Algorithm 2's offline stage): nodes [d][R*N], node_ok
    [R*N], nbr [R*N][k], the graphs in CSR form row [R][N+1], col / wt [R][2Nk]."""

    def __init__(self, robot_spec, spec: synth.PrmSpec, R: int, device="cuda"):
        self.spec, self.R = spec, R
        self.robot = robot_struct(robot_spec)
        self.params = prm_params_struct(spec)
        N, k, d = spec.N, spec.k, robot_spec.d
        self.nodes = torch.empty(d, R * N, dtype=torch.float64, device=device)
        self.node_ok = torch.empty(R * N, dtype=torch.uint8, device=device)
        self.nbr = torch.empty(R * N, k, dtype=torch.int32, device=device)
        self.row = torch.empty(R, N + 1, dtype=torch.int32, device=device)
        self.col = torch.empty(R, 2 * N * k, dtype=torch.int32, device=device)
        self.wt = torch.empty(R, 2 * N * k, dtype=torch.float64, device=device)
        self.workspace = torch.empty(lib.cr_prm_workspace_size(self.robot, R, self.params), dtype=torch.uint8,
                                     device=device)
        self.c = lib.cr_roadmap()
        self.c.R = R
        for f in ("nodes", "node_ok", "nbr", "row", "col", "wt"):
            setattr(self.c, f, getattr(self, f).data_ptr())

    def build(self, scene: Scene | None, weights: synth.WeightSpec):
        scene = scene or Scene(None)
        self._scene = scene
        lib.cr_prm_build(self.robot, scene.c, weights_struct(weights), self.params, self.c, self.workspace)
        return self

    def graph(self, r: int):
        """Roadmap r on the host: dict(nodes [N][d], ok, nbr, row, col, wt) as numpy arrays."""
        N = self.spec.N
        row = self.row[r].cpu().numpy()
        E = int(row[N])
        return dict(nodes=self.nodes[:, r * N:(r + 1) * N].T.cpu().numpy(),
                    ok=self.node_ok[r * N:(r + 1) * N].cpu().numpy().astype(bool),
                    nbr=self.nbr[r * N:(r + 1) * N].cpu().numpy(), row=row,
                    col=self.col[r, :E].cpu().numpy(), wt=self.wt[r, :E].cpu().numpy())

    def query(self, scene: Scene | None, weights, u_start_soa, u_goal_soa, T: int):
        """ConnectToRoadmap, shortest path, ResampleLinear: X [d][P*T], length [P], hops [P]."""
        scene = scene or Scene(None)
        d, P = u_start_soa.shape
        dev = u_start_soa.device
        X = torch.empty(d, P * T, dtype=torch.float64, device=dev)
        length = torch.empty(P, dtype=torch.float64, device=dev)
        hops = torch.empty(P, dtype=torch.int32, device=dev)
        lib.cr_prm_query(self.robot, scene.c, weights_struct(weights), self.params, self.c, u_start_soa, u_goal_soa,
                         P, T, X, length, hops)
        return X, length, hops


class TrajSolver:
    """Trajectory planning for P problems of T states (goal IK, linear initialisation or, with a
    roadmap, the PRM initialiser of Algorithm 2, projected gradient refinement)."""

    def __init__(self, robot_spec, goal_ik: synth.IkSpec, weights, P, T, scene: Scene | None = None,
                 precision=lib.CR_F32, k_traj=synth.K_TRAJ, alpha0=synth.ALPHA_TRAJ, device="cuda",
                 roadmap: Roadmap | None = None):
        self.robot = robot_struct(robot_spec)
        self.weights = weights
        self.P, self.T, self.k_traj, self.alpha0 = P, T, k_traj, alpha0
        self.scene = scene or Scene(None)
        self.prm = ik_params_struct(goal_ik, precision)
        self.roadmap = roadmap
        d = robot_spec.d
        wsb = (lib.cr_traj_prm_workspace_size(self.robot, P, T, self.prm) if roadmap is not None
               else lib.cr_traj_workspace_size(self.robot, P, self.prm))
        self.workspace = torch.empty(wsb, dtype=torch.uint8, device=device)
        z = lambda *s, dt=torch.float64: torch.empty(s, dtype=dt, device=device)
        self.X, self.cost, self.goal_pos, self.goal_rot = z(d, P * T), z(P), z(P), z(P)
        self.speed, self.accel = z(P), z(P)
        self.lim_ok, self.col_ok = z(P, dt=torch.uint8), z(P, dt=torch.uint8)
        self.length, self.hops = z(P), z(P, dt=torch.int32)

    def solve(self, u_start_soa, goal_soa, p0: int = 0):
        task = traj_task_struct(u_start_soa, goal_soa, self.T, self.weights)
        self._task = task
        self.prm.p0 = p0
        if self.roadmap is not None:
            lib.cr_solve_traj_prm(self.robot, self.scene.c, task, self.prm, self.roadmap.params, self.roadmap.c,
                                  self.k_traj, self.alpha0, self.X, self.cost, self.goal_pos, self.goal_rot,
                                  self.speed, self.accel, self.lim_ok, self.col_ok, self.length, self.hops,
                                  self.workspace)
            return self
        lib.cr_solve_traj(self.robot, self.scene.c, task, self.prm, self.k_traj, self.alpha0, self.X, self.cost,
                          self.goal_pos, self.goal_rot, self.speed, self.accel, self.lim_ok, self.col_ok,
                          self.workspace)
        return self


def calibrate(robot_spec, U_soa, P_meas_soa, theta0, iters=synth.ITERS_CALIB, lambda0=1e-3, history=False):
    """LM calibration of (L, r_c): U_soa [d][K] (float32/64 CUDA), P_meas_soa [3][K] FP64 CUDA.
    Returns (theta [2n], F, hist or None) as device tensors."""
    robot = robot_struct(robot_spec)
    theta = torch.as_tensor(theta0, dtype=torch.float64, device=U_soa.device).clone()
    F = torch.empty(1, dtype=torch.float64, device=U_soa.device)
    hist = torch.empty((iters, 2 * robot_spec.n), dtype=torch.float64, device=U_soa.device) if history else None
    ws = torch.empty(lib.cr_calibrate_workspace_size(robot, U_soa.shape[-1]), dtype=torch.uint8, device=U_soa.device)
    lib.cr_calibrate(robot, U_soa, P_meas_soa, theta, iters, lambda0, F, hist, ws)
    return theta, F, hist


def calibrate_lm_sharded(ops, theta, state, iters, allreduce):
    """The LM iterations of the calibration when the poses are spread over processes (the one place
    where processes exchange data: a sum over all poses): per iteration this process's partial sums (J^T J, J^T r, F) are all-reduced, every
    process forms the same trial parameters, the partial trial costs are all-reduced and every process
    applies the same rule, so theta stays identical everywhere. ``ops`` holds the four pieces (the
    library's cr_calib_* calls in CalibShard), ``allreduce(t)`` sums a tensor over the processes in
    place. theta and state (lambda, nu, ok, pred) are updated in place."""
    for _ in range(iters):
        sums = ops.sums(theta)
        allreduce(sums)
        theta_trial = ops.trial(sums, theta, state)
        F_trial = ops.cost(theta_trial)
        allreduce(F_trial)
        ops.accept(sums, F_trial, theta_trial, theta, state)
    return theta, state


class CalibShard:
    """One process's share of the calibration poses on its GPU: U_soa [d][K] (float32/64 CUDA),
    P_meas_soa [3][K] FP64 CUDA; the four pieces of an iteration as library calls."""

    def __init__(self, robot_spec, U_soa, P_meas_soa):
        self.robot = robot_struct(robot_spec)
        self.U, self.P = U_soa, P_meas_soa
        dev = U_soa.device
        self.nv = lib.cr_calib_nv(robot_spec.n)
        self.ws = torch.empty(lib.cr_calibrate_workspace_size(self.robot, U_soa.shape[-1]), dtype=torch.uint8,
                              device=dev)
        self.theta_trial = torch.empty(2 * robot_spec.n, dtype=torch.float64, device=dev)

    def sums(self, theta):
        out = torch.empty(self.nv, dtype=torch.float64, device=self.U.device)
        lib.cr_calib_sums(self.robot, self.U, self.P, theta, out, self.ws)
        return out

    def trial(self, sums, theta, state):
        lib.cr_calib_trial(self.robot, sums, theta, state, self.theta_trial)
        return self.theta_trial

    def cost(self, theta_trial):
        F = torch.empty(1, dtype=torch.float64, device=self.U.device)
        lib.cr_calib_cost(self.robot, self.U, self.P, theta_trial, F)
        return F

    def accept(self, sums, F_trial, theta_trial, theta, state):
        lib.cr_calib_accept(self.robot, sums, F_trial, theta_trial, theta, state)


def calibrate_sharded(robot_spec, U_soa, P_meas_soa, theta0, iters=synth.ITERS_CALIB, lambda0=1e-3, group=None):
    """calibrate() over the poses of all processes of ``group`` (torch.distributed, NCCL on GPUs), this
    process holding U_soa / P_meas_soa; without a process group it is calibrate() itself, iteration
    for iteration. Returns theta [2n] (device), identical on every process."""
    import torch.distributed as dist

    dev = U_soa.device
    theta = torch.as_tensor(theta0, dtype=torch.float64, device=dev).clone()
    state = torch.tensor([lambda0, 2.0, 0.0, 0.0], dtype=torch.float64, device=dev)
    multi = dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1

    def allreduce(t):
        if multi:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

    return calibrate_lm_sharded(CalibShard(robot_spec, U_soa, P_meas_soa), theta, state, iters, allreduce)[0]


# ---------------------------------------------------------------------------------------------
# Path following
# ---------------------------------------------------------------------------------------------
def path_task_struct(wp_soa, H: int, weights: synth.WeightSpec) -> lib.cr_path_task:
    """wp_soa [7][P*H] contiguous CUDA float64 (kept alive by the struct)."""
    t = lib.cr_path_task()
    t._keep = wp_soa
    t.waypoints = wp_soa.data_ptr()
    t.P = wp_soa.shape[1] // H
    t.H = H
    t.w = weights_struct(weights)
    return t


def waypoints_soa(wp, device="cuda"):
    """wp [P][H][7] host -> device [7][P*H]."""
    wp = torch.as_tensor(wp, dtype=torch.float64)
    P, H, _ = wp.shape
    return wp.reshape(P * H, 7).T.contiguous().to(device)


class PathSolver:
    """Path following for P paths of H waypoints (exploration sweep, joint LM refinement)."""

    def __init__(self, robot_spec, first_ik: synth.IkSpec, weights, P, H, scene: Scene | None = None,
                 precision=lib.CR_F32, k_warm=synth.K_WARM, k_joint=synth.K_JOINT, device="cuda"):
        self.robot = robot_struct(robot_spec)
        self.weights = weights
        self.P, self.H, self.k_warm, self.k_joint = P, H, k_warm, k_joint
        self.scene = scene or Scene(None)
        self.prm = ik_params_struct(first_ik, precision)
        d = robot_spec.d
        self.workspace = torch.empty(lib.cr_path_workspace_size(self.robot, P, H, self.prm), dtype=torch.uint8,
                                     device=device)
        z = lambda *s, dt=torch.float64: torch.empty(s, dtype=dt, device=device)
        self.X, self.cost, self.pos, self.rot = z(d, P * H), z(P), z(P * H), z(P * H)
        self.lim_ok, self.col_ok = z(P, dt=torch.uint8), z(P, dt=torch.uint8)

    def solve(self, wp_soa, p0: int = 0):
        self._task = path_task_struct(wp_soa, self.H, self.weights)
        self.prm.p0 = p0
        lib.cr_solve_path(self.robot, self.scene.c, self._task, self.prm, self.k_warm, self.k_joint, self.X, self.cost,
                          self.pos, self.rot, self.lim_ok, self.col_ok, self.workspace)
        return self


# ------------------------------------------------------------------------------------------------
# Ragged batch
# ------------------------------------------------------------------------------------------------
class BatchSolver:
    """A ragged batch of items (kind, n, H, S, n_o) -- IK (H = 1) or path -- solved by one CUDA-graph
    launch of persistent kernels. Inputs stay resident: targets [7][W] and spheres [sum n_o][4] on the
    device; ``plan()`` builds the queue and graph once, ``run()`` re-solves from the current inputs."""

    def __init__(self, family: synth.RobotSpec, items, ik: synth.IkSpec, weights: synth.WeightSpec,
                 k_warm: int = synth.K_WARM, k_joint: int = synth.K_JOINT, seeds_per_unit: int = 0,
                 device="cuda", p0: int = 0, seed_regs: int = 0):
        import numpy as np

        self.family = robot_struct(family)
        self.weights = weights_struct(weights)
        self.items_np = np.asarray(items, dtype=np.int64).reshape(-1, 5)
        self.items = lib._batch_items(self.items_np)
        self.prm = self.params(ik, k_warm, k_joint, seeds_per_unit, seed_regs)
        self.seed_regs = 0  # the plan's register budget of the seeds phase (1 wide, 2 tight) once planned
        self.prm.ik.p0 = p0  # item i draws its seeds as problem p0 + i (a process's share of a larger batch)
        it = self.items_np
        self.N = len(it)
        self.W = int(it[:, 2].sum())
        self.n_sph = int(it[:, 4].sum())
        self.n_states = int((3 * it[:, 1] * it[:, 2]).sum())
        self.device = device
        z = lambda n, dt=torch.float64: torch.empty(max(n, 1), dtype=dt, device=device)
        self.targets = torch.zeros((7, self.W), dtype=torch.float64, device=device)
        self.spheres = torch.zeros((max(self.n_sph, 1), 4), dtype=torch.float64, device=device)
        self.u, self.cost, self.pos, self.rot = z(self.n_states), z(self.N), z(self.W), z(self.W)
        self.flags, self.t_done = z(self.N, torch.uint8), z(self.N, torch.int64)
        self.workspace = torch.empty(lib.cr_batch_workspace_size(self.family, self.items, self.prm),
                                     dtype=torch.uint8, device=device)
        self._plan = None

    @staticmethod
    def params(ik: synth.IkSpec, k_warm: int = synth.K_WARM, k_joint: int = synth.K_JOINT,
               seeds_per_unit: int = 0, seed_regs: int = 0) -> lib.cr_batch_params:
        prm = lib.cr_batch_params()
        prm.ik = ik_params_struct(ik, lib.CR_F32)
        prm.k_warm, prm.k_joint, prm.seeds_per_unit = k_warm, k_joint, seeds_per_unit
        prm.seed_regs = seed_regs
        return prm

    def set_inputs(self, targets, spheres):
        """targets [W][7] (position + quaternion per waypoint, items in order), spheres [sum n_o][4]."""
        self.targets.copy_(torch.as_tensor(targets, dtype=torch.float64).T)
        if self.n_sph:
            self.spheres[: self.n_sph].copy_(torch.as_tensor(spheres, dtype=torch.float64))

    def plan(self):
        if self._plan is not None:
            lib.cr_batch_plan_destroy(self._plan)
        self._plan = lib.cr_batch_plan_create(self.family, self.weights, self.items, self.prm, self.targets,
                                              self.spheres, self.u, self.cost, self.pos, self.rot, self.flags,
                                              self.t_done, self.workspace)
        spu, units, workers, self.seed_regs = lib.cr_batch_plan_info(self._plan)
        return spu, units, workers

    def run(self):
        if self._plan is None:
            self.plan()
        lib.cr_batch_plan_run(self._plan)
        return self

    def solve_plain(self):
        """The plain per-problem form into fresh outputs: dict of u, cost, pos, rot, flags, t_done."""
        out = {k: torch.empty_like(v) for k, v in
               dict(u=self.u, cost=self.cost, pos=self.pos, rot=self.rot, flags=self.flags, t_done=self.t_done).items()}
        ws = torch.empty(lib.cr_batch_plain_workspace_size(self.family, self.items, self.prm), dtype=torch.uint8,
                         device=self.device)
        lib.cr_solve_batch_plain(self.family, self.weights, self.items, self.prm, self.targets, self.spheres,
                                 out["u"], out["cost"], out["pos"], out["rot"], out["flags"], out["t_done"], ws)
        return out

    def item_states(self, i: int, u=None):
        """[H][3n] states of item i from an item-packed output (default: the batch result)."""
        u = self.u if u is None else u
        it = self.items_np
        off = int((3 * it[:i, 1] * it[:i, 2]).sum())
        d, H = 3 * int(it[i, 1]), int(it[i, 2])
        return u[off:off + d * H].reshape(d, H).T

    def __del__(self):
        try:
            if self._plan is not None:
                lib.cr_batch_plan_destroy(self._plan)
        except Exception:
            pass


def family_fk_backbone(family: synth.RobotSpec, device="cuda"):
    """fk_backbone_n(n, U [M][3n]) for ragged_workload: FK of the family's first n segments."""
    def f(n, U):
        spec = dataclasses.replace(family, L=family.L[:n])
        T, bb = fk(robot_struct(spec), torch.as_tensor(U.T.copy(), dtype=torch.float64, device=device), True)
        return T.cpu().numpy().T, bb.cpu().numpy().transpose(2, 0, 1)
    return f
