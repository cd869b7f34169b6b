"""Thin ctypes binding of libcrsolver.so (include/cr.h), with the same entry-point names.

Only argument marshalling happens here: torch CUDA tensors are passed as raw device pointers, the
current torch stream as the cudaStream_t, and host structs as ctypes Structures. Every step of the
computation runs in the library's kernels. Loading fails loudly if the library was not built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcrsolver.so")

CR_OK, CR_EINVAL, CR_ECUDA, CR_ENONFINITE, CR_ETIMEOUT = 0, 1, 2, 3, 4
CR_F32, CR_F64 = 0, 1
CR_TASK_IK6, CR_TASK_IK5 = 0, 1
CR_MAX_SEG = 6
CR_MAX_SPHERES = 256
CR_MAX_NB = 64
CR_MAX_SEEDS = 256
CR_PRIM_DOUBLES = 16
CR_PRIM_SPHERE, CR_PRIM_CAPSULE, CR_PRIM_BOX = 0, 1, 2

EXPORTS = ("cr_fk", "cr_fk_jac", "cr_cost_grad", "cr_reduce_rows", "cr_lm_step", "cr_pg_steps",
           "cr_seeds", "cr_topk", "cr_ik_workspace_size", "cr_solve_ik", "cr_ik_stage1", "cr_ik_stage2",
           "cr_solve_ik_plain",
           "cr_poll_status", "cr_last_error_string", "cr_peak_launch", "cr_solve_ik_static",
           "cr_static_workspace_capacity", "cr_traj_cost", "cr_traj_workspace_size", "cr_solve_traj",
           "cr_calibrate", "cr_calibrate_workspace_size", "cr_cost_vjp", "cr_path_workspace_size", "cr_solve_path", "cr_device_check",
           "cr_batch_workspace_size", "cr_batch_plan_create", "cr_batch_plan_run", "cr_batch_plan_info",
           "cr_batch_plan_destroy", "cr_solve_batch", "cr_batch_plain_workspace_size", "cr_solve_batch_plain",
           "cr_batch_partition", "cr_calib_nv", "cr_calib_sums", "cr_calib_trial", "cr_calib_cost",
           "cr_calib_accept",
           "cr_prm_workspace_size", "cr_prm_build", "cr_prm_query", "cr_traj_prm_workspace_size",
           "cr_solve_traj_prm")


class CrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cr status {status}: {msg}")
        self.status = status


class cr_robot(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("n_b", C.c_int32), ("model", C.c_int32),
                ("L", C.c_double * CR_MAX_SEG), ("r_c", C.c_double * CR_MAX_SEG),
                ("u_max", C.c_double * CR_MAX_SEG), ("theta_max", C.c_double * CR_MAX_SEG),
                ("r_body", C.c_double), ("l_min", C.c_double * CR_MAX_SEG), ("l_max", C.c_double * CR_MAX_SEG)]


CR_MODEL_TENDON, CR_MODEL_ARC, CR_MODEL_COUPLED = 0, 1, 2
CR_MAX_SEG_ARC = 4


class cr_weights(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("w_p", "w_R", "rho_b", "rho_eq", "rho_k", "rho_c", "w_s",
                                          "w_len", "rho_v", "rho_a", "dt", "v_max", "a_max", "delta",
                                          "rho_s")]


class cr_scene(C.Structure):
    _fields_ = [("spheres", C.c_void_p), ("n_o", C.c_int32), ("per_problem", C.c_int32), ("prims", C.c_void_p),
                ("n_p", C.c_int32)]


class cr_task(C.Structure):
    _fields_ = [("kind", C.c_int32), ("seeds_per_target", C.c_int32), ("targets", C.c_void_p),
                ("n_targets", C.c_int64), ("w", cr_weights)]


class cr_traj_task(C.Structure):
    _fields_ = [("u_start", C.c_void_p), ("goal", C.c_void_p), ("P", C.c_int64), ("T", C.c_int32),
                ("reserved", C.c_int32), ("w", cr_weights)]


class cr_path_task(C.Structure):
    _fields_ = [("waypoints", C.c_void_p), ("P", C.c_int64), ("H", C.c_int32), ("reserved", C.c_int32),
                ("w", cr_weights)]


class cr_ik_params(C.Structure):
    _fields_ = [("S", C.c_int32), ("n_final", C.c_int32), ("k_init", C.c_int32), ("k_final", C.c_int32),
                ("lambda0", C.c_double), ("alpha0", C.c_double), ("dedup_eps", C.c_double),
                ("lim_tol", C.c_double), ("pos_tol", C.c_double), ("rot_tol", C.c_double),
                ("seed", C.c_uint64), ("p0", C.c_int64), ("precision", C.c_int32),
                ("reserved", C.c_int32)]


CR_ITEM_IK, CR_ITEM_PATH = 0, 1
CR_BATCH_MAX_SPHERES, CR_BATCH_MAX_H = 64, 128


class cr_batch_item(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("H", C.c_int32), ("S", C.c_int32), ("n_o", C.c_int32),
                ("reserved", C.c_int32)]


class cr_batch_params(C.Structure):
    _fields_ = [("ik", cr_ik_params), ("k_warm", C.c_int32), ("k_joint", C.c_int32),
                ("seeds_per_unit", C.c_int32), ("seed_regs", C.c_int32)]


CR_PRM_MAX_N, CR_PRM_MAX_K, CR_PRM_MAX_CHECK, CR_PRM_MAX_ATTEMPTS = 1024, 32, 64, 8


class cr_prm_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("k", C.c_int32), ("n_check", C.c_int32), ("attempts", C.c_int32),
                ("seed", C.c_uint64)]


class cr_roadmap(C.Structure):
    _fields_ = [("R", C.c_int64), ("nodes", C.c_void_p), ("node_ok", C.c_void_p), ("nbr", C.c_void_p),
                ("row", C.c_void_p), ("col", C.c_void_p), ("wt", C.c_void_p)]


_lib = None
_lock = threading.Lock()

_P = C.c_void_p
_SIGS = {
    "cr_fk": [C.POINTER(cr_robot), _P, C.c_int64, _P, _P, C.c_int32, _P],
    "cr_fk_jac": [C.POINTER(cr_robot), _P, C.c_int64, _P, C.c_int32, _P],
    "cr_cost_grad": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), _P, C.c_int64, _P, _P,
                     _P, _P, C.c_int32, _P],
    "cr_reduce_rows": [_P, C.c_int64, C.c_int64, _P, C.c_int32, _P],
    "cr_lm_step": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), _P, _P, _P, _P, _P,
                   C.c_int64, C.c_int32, C.c_int32, _P],
    "cr_pg_steps": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), _P, _P, _P, C.c_int64,
                    C.c_int32, C.c_int32, _P],
    "cr_seeds": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_weights), C.c_uint64, C.c_int64,
                 C.c_int64, C.c_int32, _P, C.c_int32, _P],
    "cr_topk": [_P, _P, _P, C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_double, _P, C.c_int32, _P],
    "cr_solve_ik": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), C.POINTER(cr_ik_params),
                    _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_ik_stage1": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), C.POINTER(cr_ik_params),
                     _P, C.c_size_t, _P],
    "cr_ik_stage2": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), C.POINTER(cr_ik_params),
                     _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_solve_ik_plain": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task),
                          C.POINTER(cr_ik_params), _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_solve_ik_static": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task),
                           C.POINTER(cr_ik_params), _P, _P, _P, _P, _P, _P],
    "cr_poll_status": [_P, C.POINTER(C.c_int32), _P],
    "cr_traj_cost": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_traj_task), _P, _P, _P, _P, C.c_int32, _P],
    "cr_solve_traj": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_traj_task), C.POINTER(cr_ik_params),
                      C.c_int32, C.c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_solve_path": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_path_task), C.POINTER(cr_ik_params),
                      C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_calibrate": [C.POINTER(cr_robot), _P, _P, C.c_int64, _P, C.c_int32, C.c_double, _P, _P, C.c_int32, _P,
                     C.c_size_t, _P],
    "cr_calib_sums": [C.POINTER(cr_robot), _P, _P, C.c_int64, _P, _P, C.c_int32, _P, C.c_size_t, _P],
    "cr_calib_trial": [C.POINTER(cr_robot), _P, _P, _P, _P, _P],
    "cr_calib_cost": [C.POINTER(cr_robot), _P, _P, C.c_int64, _P, _P, C.c_int32, _P],
    "cr_calib_accept": [C.POINTER(cr_robot), _P, _P, _P, _P, _P, _P],
    "cr_cost_vjp": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_task), _P, C.c_int64, _P, _P, _P, _P,
                    C.c_int32, _P],
    "cr_peak_launch": [C.c_int32, _P, C.c_size_t, C.c_int32, C.POINTER(C.c_double), _P],
    "cr_device_check": [C.c_int32, _P, _P, C.c_int64, _P],
    "cr_batch_plan_create": [C.POINTER(cr_robot), C.POINTER(cr_weights), C.POINTER(cr_batch_item), C.c_int64,
                             C.POINTER(cr_batch_params), _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P,
                             C.POINTER(C.c_void_p)],
    "cr_batch_plan_run": [_P, _P],
    "cr_batch_partition": [C.POINTER(cr_batch_item), C.c_int64, C.POINTER(cr_batch_params), C.c_int32,
                           C.POINTER(C.c_int64)],
    "cr_batch_plan_info": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                           C.POINTER(C.c_int32)],
    "cr_batch_plan_destroy": [_P],
    "cr_solve_batch": [C.POINTER(cr_robot), C.POINTER(cr_weights), C.POINTER(cr_batch_item), C.c_int64,
                       C.POINTER(cr_batch_params), _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_solve_batch_plain": [C.POINTER(cr_robot), C.POINTER(cr_weights), C.POINTER(cr_batch_item), C.c_int64,
                             C.POINTER(cr_batch_params), _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
    "cr_prm_build": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_weights), C.POINTER(cr_prm_params),
                     C.POINTER(cr_roadmap), _P, C.c_size_t, _P],
    "cr_prm_query": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_weights), C.POINTER(cr_prm_params),
                     C.POINTER(cr_roadmap), _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P],
    "cr_solve_traj_prm": [C.POINTER(cr_robot), C.POINTER(cr_scene), C.POINTER(cr_traj_task),
                          C.POINTER(cr_ik_params), C.POINTER(cr_prm_params), C.POINTER(cr_roadmap), C.c_int32,
                          C.c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P],
}


def load(path: str | None = None):
    """Load libcrsolver.so (raises if it is missing: build it with build_lib.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libcrsolver.so not found at {p}; run paper_2607_11340_gb300.build_lib.build()")
        L = C.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.cr_ik_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64, C.POINTER(cr_ik_params)]
        L.cr_ik_workspace_size.restype = C.c_size_t
        L.cr_traj_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64, C.POINTER(cr_ik_params)]
        L.cr_traj_workspace_size.restype = C.c_size_t
        L.cr_path_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64, C.c_int32, C.POINTER(cr_ik_params)]
        L.cr_path_workspace_size.restype = C.c_size_t
        L.cr_prm_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64, C.POINTER(cr_prm_params)]
        L.cr_prm_workspace_size.restype = C.c_size_t
        L.cr_traj_prm_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64, C.c_int32, C.POINTER(cr_ik_params)]
        L.cr_traj_prm_workspace_size.restype = C.c_size_t
        L.cr_calibrate_workspace_size.argtypes = [C.POINTER(cr_robot), C.c_int64]
        L.cr_calibrate_workspace_size.restype = C.c_size_t
        for nm in ("cr_batch_workspace_size", "cr_batch_plain_workspace_size"):
            getattr(L, nm).argtypes = [C.POINTER(cr_robot), C.POINTER(cr_batch_item), C.c_int64,
                                       C.POINTER(cr_batch_params)]
            getattr(L, nm).restype = C.c_size_t
        L.cr_calib_nv.argtypes = [C.c_int32]
        L.cr_calib_nv.restype = C.c_int32
        L.cr_static_workspace_capacity.argtypes = []
        L.cr_static_workspace_capacity.restype = C.c_size_t
        L.cr_last_error_string.argtypes = []
        L.cr_last_error_string.restype = C.c_char_p
        _lib = L
        return L


def last_error() -> str:
    return load().cr_last_error_string().decode()


def _check(st: int):
    if st != CR_OK:
        raise CrError(st, last_error())


def _ptr(t):
    """Device pointer of a tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("CUDA tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch

    if t.dtype == torch.float32:
        return CR_F32
    if t.dtype == torch.float64:
        return CR_F64
    raise ValueError(f"float32/float64 expected, got {t.dtype}")


# --------------------------------------------------------------------------------------------
# Same-name wrappers (tensors in, status checked)
# --------------------------------------------------------------------------------------------
def cr_fk(robot: cr_robot, u, T_out, backbone_out=None, stream=None):
    B = u.shape[-1]
    _check(load().cr_fk(C.byref(robot), _ptr(u), B, _ptr(T_out), _ptr(backbone_out), _dtype_code(u),
                        _stream(stream)))


def cr_fk_jac(robot: cr_robot, u, J_out, stream=None):
    _check(load().cr_fk_jac(C.byref(robot), _ptr(u), u.shape[-1], _ptr(J_out), _dtype_code(u), _stream(stream)))


def cr_cost_grad(robot, scene, task, u, cost_out, coll_out=None, grad_u_out=None, grad_param_out=None,
                 stream=None):
    _check(load().cr_cost_grad(C.byref(robot), C.byref(scene), C.byref(task), _ptr(u), u.shape[-1],
                               _ptr(cost_out), _ptr(coll_out), _ptr(grad_u_out), _ptr(grad_param_out),
                               _dtype_code(u), _stream(stream)))


def cr_reduce_rows(x, out, stream=None):
    _check(load().cr_reduce_rows(_ptr(x), x.shape[0], x.shape[1], _ptr(out), _dtype_code(x), _stream(stream)))


def cr_lm_step(robot, scene, task, u, lam, nu, F_out=None, accepted_out=None, n_iter=1, stream=None):
    _check(load().cr_lm_step(C.byref(robot), C.byref(scene), C.byref(task), _ptr(u), _ptr(lam), _ptr(nu),
                             _ptr(F_out), _ptr(accepted_out), u.shape[-1], n_iter, _dtype_code(u),
                             _stream(stream)))


def cr_pg_steps(robot, scene, task, u, alpha, F_out, steps, stream=None):
    _check(load().cr_pg_steps(C.byref(robot), C.byref(scene), C.byref(task), _ptr(u), _ptr(alpha), _ptr(F_out),
                              u.shape[-1], steps, _dtype_code(u), _stream(stream)))


def cr_seeds(robot, scene, weights, seed, p0, P, S, u_out, stream=None):
    _check(load().cr_seeds(C.byref(robot), C.byref(scene), C.byref(weights), C.c_uint64(seed), p0, P, S,
                           _ptr(u_out), _dtype_code(u_out), _stream(stream)))


def cr_topk(cost, coll, u, P, S, k, dedup_eps, idx_out, stream=None):
    _check(load().cr_topk(_ptr(cost), _ptr(coll), _ptr(u), u.shape[0], P, S, k, dedup_eps, _ptr(idx_out),
                          _dtype_code(u), _stream(stream)))


def cr_ik_workspace_size(robot, P, prm) -> int:
    return int(load().cr_ik_workspace_size(C.byref(robot), P, C.byref(prm)))


def cr_solve_ik(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, workspace, stream=None):
    _check(load().cr_solve_ik(C.byref(robot), C.byref(scene), C.byref(task), C.byref(prm), _ptr(u_out),
                              _ptr(cost_out), _ptr(pos_err), _ptr(rot_err), _ptr(success), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_ik_stage1(robot, scene, task, prm, workspace, stream=None):
    _check(load().cr_ik_stage1(C.byref(robot), C.byref(scene), C.byref(task), C.byref(prm), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_ik_stage2(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, workspace, stream=None):
    _check(load().cr_ik_stage2(C.byref(robot), C.byref(scene), C.byref(task), C.byref(prm), _ptr(u_out),
                               _ptr(cost_out), _ptr(pos_err), _ptr(rot_err), _ptr(success), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_solve_ik_plain(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, workspace,
                      stream=None):
    _check(load().cr_solve_ik_plain(C.byref(robot), C.byref(scene), C.byref(task), C.byref(prm), _ptr(u_out),
                                    _ptr(cost_out), _ptr(pos_err), _ptr(rot_err), _ptr(success),
                                    _ptr(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)))


def cr_solve_ik_static(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, stream=None):
    """cr_solve_ik without a workspace argument (scratch is a static device array; allocates nothing)."""
    _check(load().cr_solve_ik_static(C.byref(robot), C.byref(scene), C.byref(task), C.byref(prm), _ptr(u_out),
                                     _ptr(cost_out), _ptr(pos_err), _ptr(rot_err), _ptr(success),
                                     _stream(stream)))


def cr_static_workspace_capacity() -> int:
    return int(load().cr_static_workspace_capacity())


def cr_traj_cost(robot, scene, task, x, cost_out, grad_out=None, upstream=None, stream=None):
    _check(load().cr_traj_cost(C.byref(robot), C.byref(scene), C.byref(task), _ptr(x), _ptr(cost_out), _ptr(grad_out),
                               _ptr(upstream), _dtype_code(x), _stream(stream)))


def cr_traj_workspace_size(robot, P, goal_ik) -> int:
    return int(load().cr_traj_workspace_size(C.byref(robot), P, C.byref(goal_ik)))


def cr_solve_traj(robot, scene, task, goal_ik, k_traj, alpha0, X_out, cost_out, goal_pos, goal_rot, speed, accel,
                  lim_ok, col_ok, workspace, stream=None):
    _check(load().cr_solve_traj(C.byref(robot), C.byref(scene), C.byref(task), C.byref(goal_ik), k_traj, alpha0,
                                _ptr(X_out), _ptr(cost_out), _ptr(goal_pos), _ptr(goal_rot), _ptr(speed), _ptr(accel),
                                _ptr(lim_ok), _ptr(col_ok), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_prm_workspace_size(robot, R, prm) -> int:
    return int(load().cr_prm_workspace_size(C.byref(robot), R, C.byref(prm)))


def cr_prm_build(robot, scene, weights, prm, roadmap, workspace, stream=None):
    _check(load().cr_prm_build(C.byref(robot), C.byref(scene), C.byref(weights), C.byref(prm), C.byref(roadmap),
                               _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_prm_query(robot, scene, weights, prm, roadmap, u_start, u_goal, P, T, X, length, hops, stream=None):
    _check(load().cr_prm_query(C.byref(robot), C.byref(scene), C.byref(weights), C.byref(prm), C.byref(roadmap),
                               _ptr(u_start), _ptr(u_goal), P, T, _ptr(X), _ptr(length), _ptr(hops),
                               _stream(stream)))


def cr_traj_prm_workspace_size(robot, P, T, goal_ik) -> int:
    return int(load().cr_traj_prm_workspace_size(C.byref(robot), P, T, C.byref(goal_ik)))


def cr_solve_traj_prm(robot, scene, task, goal_ik, prm, roadmap, k_traj, alpha0, X_out, cost_out, goal_pos, goal_rot,
                      speed, accel, lim_ok, col_ok, length, hops, workspace, stream=None):
    _check(load().cr_solve_traj_prm(C.byref(robot), C.byref(scene), C.byref(task), C.byref(goal_ik), C.byref(prm),
                                    C.byref(roadmap), k_traj, alpha0, _ptr(X_out), _ptr(cost_out), _ptr(goal_pos),
                                    _ptr(goal_rot), _ptr(speed), _ptr(accel), _ptr(lim_ok), _ptr(col_ok),
                                    _ptr(length), _ptr(hops), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_path_workspace_size(robot, P, H, first_ik) -> int:
    return int(load().cr_path_workspace_size(C.byref(robot), P, H, C.byref(first_ik)))


def cr_solve_path(robot, scene, task, first_ik, k_warm, k_joint, X_out, cost_out, pos_err, rot_err, lim_ok, col_ok,
                  workspace, stream=None):
    _check(load().cr_solve_path(C.byref(robot), C.byref(scene), C.byref(task), C.byref(first_ik), k_warm, k_joint,
                                _ptr(X_out), _ptr(cost_out), _ptr(pos_err), _ptr(rot_err), _ptr(lim_ok), _ptr(col_ok),
                                _ptr(workspace), workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_calibrate_workspace_size(robot, K) -> int:
    return int(load().cr_calibrate_workspace_size(C.byref(robot), K))


def cr_calibrate(robot, U, P_meas, theta, iters, lambda0, F_out, hist, workspace, stream=None):
    _check(load().cr_calibrate(C.byref(robot), _ptr(U), _ptr(P_meas), U.shape[-1], _ptr(theta), iters, lambda0,
                               _ptr(F_out), _ptr(hist), _dtype_code(U), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream(stream)))


def cr_calib_nv(n: int) -> int:
    return int(load().cr_calib_nv(n))


def cr_calib_sums(robot, U, P_meas, theta, sums, workspace, stream=None):
    _check(load().cr_calib_sums(C.byref(robot), _ptr(U), _ptr(P_meas), U.shape[-1], _ptr(theta), _ptr(sums),
                                _dtype_code(U), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                _stream(stream)))


def cr_calib_trial(robot, sums, theta, state, theta_trial, stream=None):
    _check(load().cr_calib_trial(C.byref(robot), _ptr(sums), _ptr(theta), _ptr(state), _ptr(theta_trial),
                                 _stream(stream)))


def cr_calib_cost(robot, U, P_meas, theta_trial, F_trial, stream=None):
    _check(load().cr_calib_cost(C.byref(robot), _ptr(U), _ptr(P_meas), U.shape[-1], _ptr(theta_trial), _ptr(F_trial),
                                _dtype_code(U), _stream(stream)))


def cr_calib_accept(robot, sums, F_trial, theta_trial, theta, state, stream=None):
    _check(load().cr_calib_accept(C.byref(robot), _ptr(sums), _ptr(F_trial), _ptr(theta_trial), _ptr(theta),
                                  _ptr(state), _stream(stream)))


def cr_cost_vjp(robot, scene, task, u, upstream, grad_u_out, grad_param_out=None, workspace=None, stream=None):
    _check(load().cr_cost_vjp(C.byref(robot), C.byref(scene), C.byref(task), _ptr(u), u.shape[-1], _ptr(upstream),
                              _ptr(grad_u_out), _ptr(grad_param_out), _ptr(workspace), _dtype_code(u), _stream(stream)))


def cr_poll_status(workspace, stream=None) -> int:
    out = C.c_int32(0)
    _check(load().cr_poll_status(_ptr(workspace), C.byref(out), _stream(stream)))
    return out.value


CR_CHECK_RECIP, CR_CHECK_SIN, CR_CHECK_COS = 0, 1, 2


def cr_device_check(which: int, x, out, stream=None):
    _check(load().cr_device_check(which, _ptr(x), _ptr(out), x.numel(), _stream(stream)))


def cr_peak_launch(kind: int, buf, iters: int, stream=None) -> float:
    ops = C.c_double(0)
    _check(load().cr_peak_launch(kind, _ptr(buf), buf.numel() * buf.element_size(), iters, C.byref(ops),
                                 _stream(stream)))
    return ops.value


def _batch_items(items):
    """(N, 6) int array or a list of (kind, n, H, S, n_o) -> ctypes array of cr_batch_item."""
    arr = (cr_batch_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = cr_batch_item(int(it[0]), int(it[1]), int(it[2]), int(it[3]), int(it[4]), 0)
    return arr


def cr_batch_workspace_size(robot, items, prm) -> int:
    return load().cr_batch_workspace_size(C.byref(robot), items, len(items), C.byref(prm))


def cr_batch_plain_workspace_size(robot, items, prm) -> int:
    return load().cr_batch_plain_workspace_size(C.byref(robot), items, len(items), C.byref(prm))


def cr_batch_plan_create(robot, weights, items, prm, targets, spheres, u_out, cost, pos, rot, flags, t_done,
                         workspace, stream=None):
    plan = C.c_void_p()
    _check(load().cr_batch_plan_create(C.byref(robot), C.byref(weights), items, len(items), C.byref(prm),
                                       _ptr(targets), _ptr(spheres), _ptr(u_out), _ptr(cost), _ptr(pos), _ptr(rot),
                                       _ptr(flags), _ptr(t_done), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _stream(stream), C.byref(plan)))
    return plan


def cr_batch_partition(items, prm, parts: int):
    """Contiguous cost-balanced partition of the items over `parts` processes: list of parts + 1
    bounds (host only)."""
    b = (C.c_int64 * (parts + 1))()
    _check(load().cr_batch_partition(items, len(items), C.byref(prm), parts, b))
    return [int(v) for v in b]


def cr_batch_plan_run(plan, stream=None):
    _check(load().cr_batch_plan_run(plan, _stream(stream)))


def cr_batch_plan_info(plan):
    spu, units, workers, regs = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
    _check(load().cr_batch_plan_info(plan, C.byref(spu), C.byref(units), C.byref(workers), C.byref(regs)))
    return spu.value, units.value, workers.value, regs.value


def cr_batch_plan_destroy(plan):
    _check(load().cr_batch_plan_destroy(plan))


def cr_solve_batch(robot, weights, items, prm, targets, spheres, u_out, cost, pos, rot, flags, t_done, workspace,
                   stream=None):
    _check(load().cr_solve_batch(C.byref(robot), C.byref(weights), items, len(items), C.byref(prm), _ptr(targets),
                                 _ptr(spheres), _ptr(u_out), _ptr(cost), _ptr(pos), _ptr(rot), _ptr(flags),
                                 _ptr(t_done), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                 _stream(stream)))


def cr_solve_batch_plain(robot, weights, items, prm, targets, spheres, u_out, cost, pos, rot, flags, t_done,
                         workspace, stream=None):
    _check(load().cr_solve_batch_plain(C.byref(robot), C.byref(weights), items, len(items), C.byref(prm),
                                       _ptr(targets), _ptr(spheres), _ptr(u_out), _ptr(cost), _ptr(pos), _ptr(rot),
                                       _ptr(flags), _ptr(t_done), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _stream(stream)))
