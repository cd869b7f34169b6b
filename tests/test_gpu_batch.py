"""GPU tests of the ragged batch (persistent kernels over a work queue, one CUDA graph): agreement
with the plain per-problem form on the same items, determinism, validity of every result under the
FP64 oracle, success-rate agreement with the oracle's own solves, the edge cases of the item
ranges, and the full-size 16384-item batch on a sampled subset."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import orc_robot, orc_weights
from paper_2607_11340_gb300 import api, lib, synth

pytestmark = pytest.mark.gpu

FAM = synth.ROBOT_FAMILY
IK = dataclasses.replace(synth.IK_RAGGED, k_init=24, k_final=15)
K_WARM, K_JOINT = 10, 6

# kind, n, H, S, n_o: both kinds, every segment count, H = 1 paths, a ragged tail over 32 and 64
# waypoints, fewer seeds than n_final, one full seed group, the maximum of every range
EDGE_ITEMS = [
    (0, 1, 1, 16, 0), (0, 2, 1, 5, 3), (0, 3, 1, 256, 64), (0, 4, 1, 40, 10), (0, 5, 1, 33, 0), (0, 6, 1, 64, 7),
    (1, 1, 1, 20, 4), (1, 2, 2, 17, 0), (1, 3, 33, 48, 12), (1, 4, 65, 24, 5), (1, 5, 9, 70, 64),
    (1, 6, 128, 16, 2), (1, 6, 5, 1, 0), (0, 1, 1, 1, 1), (1, 2, 31, 32, 9), (1, 4, 32, 96, 0),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_11340_gb300 import build_lib

    build_lib.build()
    O.build()


def _batch(items, seed=0, spu=32, ik=IK, k_warm=K_WARM, k_joint=K_JOINT, seed_regs=0):
    items, targets, spheres, states = synth.ragged_workload(len(items), api.family_fk_backbone(FAM), seed=seed,
                                                            items=np.asarray(items))
    s = api.BatchSolver(FAM, items, ik, synth.WEIGHTS, k_warm, k_joint, seeds_per_unit=spu, seed_regs=seed_regs)
    s.set_inputs(targets, spheres)
    return s, targets, spheres


def _item_views(s, targets, spheres, i):
    it = s.items_np
    w0 = int(it[:i, 2].sum())
    o0 = int(it[:i, 4].sum())
    H, no = int(it[i, 2]), int(it[i, 4])
    return targets[w0:w0 + H], (spheres[o0:o0 + no] if no else None), w0


def test_batch_matches_plain_form_and_is_deterministic():
    s, targets, spheres = _batch(EDGE_ITEMS, seed=1)
    spu, units, workers = s.plan()
    assert spu == 32 and units == sum((S + 31) // 32 for _, _, _, S, _ in EDGE_ITEMS) and workers > 0
    s.run()
    torch.cuda.synchronize()
    first = {k: getattr(s, k).clone() for k in ("u", "cost", "pos", "rot", "flags", "t_done")}
    s.run()
    torch.cuda.synchronize()
    for k in ("u", "cost", "pos", "rot", "flags"):
        assert torch.equal(first[k].nan_to_num(-7), getattr(s, k).nan_to_num(-7)), k
    plain = s.solve_plain()
    torch.cuda.synchronize()
    # the same problems, seeds and settings. The states are not bit-identical: the batch kernel and
    # the per-problem kernels are separate compilation units whose FP32 code (contractions, register
    # allocation) differs in the last bits, and stage one carries that into other local minima. Both
    # are compared on the unique part: the verdict per item; their states are each valid under the
    # oracle (test_batch_results_valid_under_oracle).
    fb = s.flags.cpu().numpy() & 1
    fp = plain["flags"].cpu().numpy() & 1
    du = [float(np.abs(s.item_states(i).cpu().numpy() - s.item_states(i, plain["u"]).cpu().numpy()).max())
          for i in range(len(fb))]
    print(f"batch vs per-problem form: verdicts agree on {int((fb == fp).sum())} of {len(fb)} items; "
          f"items with states within 2e-5 (m): {sum(d <= 2e-5 for d in du)}; largest state difference {max(du):.2e}")
    assert np.sum(fb != fp) <= 1, (fb, fp)
    assert fb.sum() >= len(fb) // 2


def test_batch_results_valid_under_oracle():
    """The reported per-waypoint errors and the flags equal the oracle's FP64 evaluation of the
    batch's own states."""
    s, targets, spheres = _batch(EDGE_ITEMS, seed=2)
    s.plan()
    s.run()
    torch.cuda.synchronize()
    it = s.items_np
    pos_all, rot_all = s.pos.cpu().numpy(), s.rot.cpu().numpy()
    for i in range(len(it)):
        n = int(it[i, 1])
        tg, sp, w0 = _item_views(s, targets, spheres, i)
        rbo = orc_robot(dataclasses.replace(FAM, L=FAM.L[:n]))
        u = s.item_states(i).cpu().numpy()
        pos, rot, lim, col = O.accept(rbo, sp, 0, tg, u)
        H = len(tg)
        np.testing.assert_allclose(pos_all[w0:w0 + H], pos, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(rot_all[w0:w0 + H], rot, rtol=1e-9, atol=1e-12)
        f = s.flags[i].item()
        assert bool(f & 2) == bool(lim.all()) and bool(f & 4) == bool(col.all()), i
        succ = (pos <= IK.pos_tol).all() and (rot <= IK.rot_tol).all() and lim.all() and col.all()
        assert bool(f & 1) == bool(succ), i
        assert s.t_done[i].item() > 0


def test_batch_success_rate_matches_oracle():
    """Success at <= 1 mm / <= 1 degree (every waypoint, limits and clearance) against the oracle's
    own solves of the same items with the same seeds and settings."""
    rng = np.random.default_rng(5)
    items = synth.ragged_items(rng, 40)
    items[:, 2] = np.where(items[:, 0] == 1, rng.integers(2, 12, 40), 1)
    items[:, 3] = rng.integers(16, 65, 40)
    items[:, 4] = rng.integers(0, 9, 40)
    s, targets, spheres = _batch(items, seed=3)
    s.plan()
    s.run()
    torch.cuda.synchronize()
    succ_g = (s.flags.cpu().numpy() & 1).astype(bool)
    succ_o = np.zeros(len(items), bool)
    for i, (kind, n, H, S, no) in enumerate(items):
        tg, sp, _ = _item_views(s, targets, spheres, i)
        rbo = orc_robot(dataclasses.replace(FAM, L=FAM.L[:n]))
        cfg = O.IkConfig(S=int(S), n_final=min(IK.n_final, int(S)), k_init=IK.k_init, k_final=IK.k_final,
                         lambda0=IK.lambda0, alpha0=IK.alpha0, p0=i)
        if kind == 1 and H > 1:
            o = O.solve_path(rbo, orc_weights(), None if sp is None else sp[None], tg[None], cfg, K_WARM, K_JOINT)
            succ_o[i] = ((o["pos"][0] <= IK.pos_tol).all() and (o["rot"][0] <= IK.rot_tol).all()
                         and o["lim_ok"][0] and o["col_ok"][0])
        else:
            o = O.solve_ik(rbo, orc_weights(), sp, 0, tg, cfg)
            succ_o[i] = bool(o["success"][0])
    print(f"40 items: success GPU {succ_g.mean():.3f} oracle {succ_o.mean():.3f}, mismatches {int((succ_g != succ_o).sum())}")
    # the 1-point comparison runs on 200 items in tests/test_gpu_success_parity.py
    assert np.sum(succ_g != succ_o) <= 2


def test_seed_register_budgets_agree():
    """The two register budgets of the seeds phase: the same method, but ptxas contracts multiplies
    and adds into FMAs differently under the two caps, so results agree to the consequences of FP32
    rounding (success flags of all but one item), each budget is deterministic run to run, and with
    the budget left open the planner picks one of the two by timing."""
    out = {}
    for regs in (1, 2, 0):
        s, _, _ = _batch(EDGE_ITEMS, seed=2, seed_regs=regs)
        s.plan()
        assert s.seed_regs == (regs if regs else s.seed_regs) and s.seed_regs in (1, 2)
        runs = []
        for _ in range(2):
            s.run()
            torch.cuda.synchronize()
            runs.append({k: getattr(s, k).cpu().numpy() for k in ("u", "cost", "flags")})
        for k in ("u", "cost", "flags"):
            np.testing.assert_array_equal(runs[0][k], runs[1][k])
        out[regs] = runs[0]
    ok = {r: (o["flags"] & 1).astype(bool) for r, o in out.items()}
    print(f"seed-phase register budgets: success wide {ok[1].mean():.3f} tight {ok[2].mean():.3f}, "
          f"flag mismatches {int((ok[1] != ok[2]).sum())}")
    assert int((ok[1] != ok[2]).sum()) <= 1
    assert np.array_equal(out[0]["flags"], out[1]["flags"] if s.seed_regs == 1 else out[2]["flags"])


def test_batch_autotuned_plan_full_size_sample():
    """The 16384-item batch of the serving workload with the seeds per unit picked by timing: every
    item completes, and a sampled subset is valid under the oracle."""
    items, targets, spheres, _ = synth.ragged_workload(synth.N_RAGGED, api.family_fk_backbone(FAM), seed=0)
    s = api.BatchSolver(FAM, items, synth.IK_RAGGED, synth.WEIGHTS, seeds_per_unit=0)
    s.set_inputs(targets, spheres)
    spu, units, workers = s.plan()
    assert spu in (32, 64, 128, 256)
    s.run()
    torch.cuda.synchronize()
    t = s.t_done.cpu().numpy()
    assert (t > 0).all()
    cost = s.cost.cpu().numpy()
    assert np.isfinite(cost).mean() > 0.999
    rng = np.random.default_rng(0)
    for i in rng.choice(len(items), 24, replace=False):
        n = int(items[i, 1])
        tg, sp, w0 = _item_views(s, targets, spheres, i)
        rbo = orc_robot(dataclasses.replace(FAM, L=FAM.L[:n]))
        pos, rot, lim, col = O.accept(rbo, sp, 0, tg, s.item_states(i).cpu().numpy())
        np.testing.assert_allclose(s.pos[w0:w0 + len(tg)].cpu().numpy(), pos, rtol=1e-9, atol=1e-12)
    # success over the batch: a serving workload of feasible targets
    assert (s.flags.cpu().numpy() & 1).mean() > 0.8
