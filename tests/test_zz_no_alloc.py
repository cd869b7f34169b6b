"""The allocation-free entry point cr_solve_ik_static.

It serves callers that must not allocate device memory, for instance a robot's real-time control
loop that reserves everything at start-up (cudaMalloc can block or synchronise the device at a
moment the loop cannot afford). Its scratch is a static device array inside the library. The
test calls it twice in a row through the C ABI and checks both results against the ordinary
cr_solve_ik (workspace passed by the caller) on the same inputs, at the FP32 tolerance of the
other GPU tests; it also checks that an oversize problem is refused with CR_EINVAL.
This file is collected last so that a run stopping at its first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 relative tolerance of the parity tests


@pytest.fixture(scope="module")
def setup():
    from paper_2607_11340_gb300 import api, build_lib, lib, synth

    build_lib.build()
    spec, ik = synth.ROBOT_3SEG, synth.IkSpec(S=256, n_final=8, k_init=32, k_final=20)
    P = 512
    rng = np.random.default_rng(900)
    u_true = synth.hexagon_states(rng, P, spec.n, spec.umax)
    T, _ = api.fk(api.robot_struct(spec), torch.as_tensor(u_true.T.copy(), dtype=torch.float64).cuda())
    tg = synth.pose_targets(T.cpu().numpy().T, "pose")
    tgd = torch.as_tensor(tg.T.copy(), dtype=torch.float64).cuda()
    return api, lib, synth, spec, ik, P, tgd


def _outputs(P, d):
    return [torch.empty((d, P), dtype=torch.float64, device="cuda")] + \
        [torch.empty(P, dtype=torch.float64, device="cuda") for _ in range(3)] + \
        [torch.empty(P, dtype=torch.uint8, device="cuda")]


def test_static_matches_workspace_version_twice(setup):
    api, lib, synth, spec, ik, P, tgd = setup
    robot = api.robot_struct(spec)
    scene = api.Scene(None)
    task = api.task_struct(lib.CR_TASK_IK6, tgd, 1, synth.WEIGHTS)
    prm = api.ik_params_struct(ik, lib.CR_F32)
    assert lib.cr_ik_workspace_size(robot, P, prm) <= lib.cr_static_workspace_capacity()
    ref = _outputs(P, spec.d)
    ws = torch.empty(lib.cr_ik_workspace_size(robot, P, prm), dtype=torch.uint8, device="cuda")
    lib.cr_solve_ik(robot, scene.c, task, prm, *ref, ws)
    for _ in range(2):
        out = _outputs(P, spec.d)
        lib.cr_solve_ik_static(robot, scene.c, task, prm, *out)
        torch.cuda.synchronize()
        u, cost, pos, rot, suc = [x.cpu().numpy() for x in out]
        ru, rcost, rpos, rrot, rsuc = [x.cpu().numpy() for x in ref]
        assert np.array_equal(suc, rsuc)
        np.testing.assert_allclose(u, ru, rtol=TOL, atol=TOL * spec.umax)
        np.testing.assert_allclose(cost, rcost, rtol=TOL, atol=1e-20)
        np.testing.assert_allclose(pos, rpos, rtol=TOL, atol=1e-12)
        np.testing.assert_allclose(rot, rrot, rtol=TOL, atol=1e-12)
        assert suc.mean() > 0.95


def test_static_refuses_oversize(setup):
    api, lib, synth, spec, ik, P, tgd = setup
    robot = api.robot_struct(spec)
    prm = api.ik_params_struct(ik, lib.CR_F32)
    big = 1
    while lib.cr_ik_workspace_size(robot, big, prm) <= lib.cr_static_workspace_capacity():
        big *= 2
    tg = torch.zeros((7, big), dtype=torch.float64, device="cuda")
    tg[3] = 1.0
    task = api.task_struct(lib.CR_TASK_IK6, tg, 1, synth.WEIGHTS)
    out = _outputs(big, spec.d)
    with pytest.raises(lib.CrError) as e:
        lib.cr_solve_ik_static(robot, api.Scene(None).c, task, prm, *out)
    assert e.value.status == lib.CR_EINVAL
    assert "static array" in str(e.value)
