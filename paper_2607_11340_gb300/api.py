"""User-facing API over the C ABI: builds the host structs, lets torch allocate device outputs and
workspaces, and calls the library. No arithmetic of the method happens here."""
from __future__ import annotations

import dataclasses

import torch

from . import lib
from . import synth


def robot_struct(spec: synth.RobotSpec) -> lib.cr_robot:
    r = lib.cr_robot()
    r.n, r.m, r.n_b, r.reserved = spec.n, 3, spec.nb, 0
    for i in range(spec.n):
        r.L[i] = spec.L[i]
        r.r_c[i] = spec.rc
        r.u_max[i] = spec.umax
        r.theta_max[i] = spec.thmax
    r.r_body = spec.body_radius
    return r


def weights_struct(w: synth.WeightSpec) -> lib.cr_weights:
    s = lib.cr_weights()
    s.w_p, s.w_R = w.wp, w.wR
    s.rho_b, s.rho_eq, s.rho_k, s.rho_c = w.rho_b, w.rho_eq, w.rho_k, w.rho_c
    s.w_s, s.w_len, s.rho_v, s.rho_a = w.w_s, w.w_len, w.rho_v, w.rho_a
    s.dt, s.v_max, s.a_max, s.delta = w.dt, w.vmax, w.amax, w.delta
    return s


class Scene:
    """Spheres [n_o][4] (centre, radius) resident on the device in FP64."""

    def __init__(self, spheres=None, device="cuda"):
        if spheres is None or len(spheres) == 0:
            self.spheres = None
            self.n_o = 0
        else:
            self.spheres = torch.as_tensor(spheres, dtype=torch.float64, device=device).reshape(-1, 4).contiguous()
            self.n_o = self.spheres.shape[0]
        self.c = lib.cr_scene()
        self.c.spheres = self.spheres.data_ptr() if self.spheres is not None else None
        self.c.n_o = self.n_o


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

    def status(self) -> int:
        return lib.cr_poll_status(self.workspace)


def solve_ik(robot_spec, ik_spec, weights, kind, targets_soa, scene=None, precision=lib.CR_F32, plain=False):
    s = IkSolver(robot_spec, ik_spec, weights, kind, targets_soa.shape[1], scene, precision, plain,
                 device=targets_soa.device)
    return s.solve(targets_soa)
