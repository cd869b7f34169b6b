"""Writes tests/golden/opcounts.json: algorithmic operation counts of one state evaluation of each
benchmark workload, counted by the oracle's op-counting scalar on the minimal (Rodrigues) form of
Eq. 2-3. "fwd" = cost (kinematics, pose log, penalty rows); "tan" = the linearised program whose
transpose is the adjoint (same multiply-add count), so one value-and-gradient evaluation costs
fwd + tan. "trial_*" counts leave out the rows that vanish at the projected trial points of stage
one (tendon model: bound and sum-zero rows; arc model: length and curvature rows). "pg_step_*" is
the step rule's own arithmetic per trial point (gradient norm, step length and move, without the
projection); "lm_update_*" that of one LM update of stage two (damping, Cholesky, the two
triangular solves, predicted decrease, gain ratio, damping rule) without its cost evaluations.
Calls only oracle/."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2607_11340_gb300 import synth  # noqa: E402


def counts(spec, kind, n_states=64):
    if spec.is_arc:
        rb = O.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius,
                          lmin=spec.lmin, lmax=spec.lmax)
    else:
        rb = O.make_robot(list(spec.L), spec.rc, spec.umax, nb=spec.nb)
    W = O.make_weights(**synth.WEIGHTS.as_dict())
    rng = np.random.default_rng(0)
    if spec.is_arc:
        u = synth.arc_states(rng, n_states + 1, spec)
    else:
        u = synth.hexagon_states(rng, n_states + 1, spec.n, spec.umax)
    tg = synth.pose_targets(O.fk(rb, u[:1])[0], "pose" if kind == O.IK6 else "axis")[0]
    c = np.array([O.opcount_ik(rb, W, None, kind, tg, u[1 + i]) for i in range(n_states)], dtype=float)
    m = c.mean(axis=0)  # branches (series vs closed form) make the count state-dependent
    out = {"fwd_flop": float(m[0]), "fwd_sfu": float(m[1]), "tan_flop": float(m[2]), "tan_sfu": float(m[3])}
    # a projected trial point of stage one (feasible: none of the rows that vanish there)
    c = np.array([O.opcount_ik(rb, W, None, kind, tg, u[1 + i], box=False) for i in range(n_states)], dtype=float)
    m = c.mean(axis=0)
    out.update({"trial_fwd_flop": float(m[0]), "trial_fwd_sfu": float(m[1]), "trial_tan_flop": float(m[2]),
                "trial_tan_sfu": float(m[3])})
    # the step rule's own arithmetic per trial (gradient norm, step length, move; not the projection)
    f, sf = O.opcount_pg_step(u.shape[1])
    out.update({"pg_step_flop": float(f), "pg_step_sfu": float(sf)})
    # one LM update of stage two without its cost evaluations (damping, Cholesky, solves, gain ratio)
    f, sf = O.opcount_lm_update(u.shape[1])
    out.update({"lm_update_flop": float(f), "lm_update_sfu": float(sf)})
    return out


def main():
    out = {
        "ik_3seg_pose": counts(synth.ROBOT_3SEG, O.IK6),
        "ik_1seg_axis": counts(synth.ROBOT_1SEG, O.IK5),
        "ik_arc_3seg_pose": counts(synth.ROBOT_E1, O.IK6),
    }
    path = os.path.join(HERE, "opcounts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(path, out)


if __name__ == "__main__":
    main()
