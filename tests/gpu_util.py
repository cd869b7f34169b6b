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
                        nb=spec.nb, rbody=spec.body_radius, lmin=spec.lmin, lmax=spec.lmax)


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
