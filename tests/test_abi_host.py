"""Host-side checks of the C ABI that need no GPU: the library loads and exports every entry point
include/cr.h declares, the ctypes mirrors of the structs have the C layout, and invalid
arguments are rejected with CR_EINVAL before anything is launched."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cr.h")


@pytest.fixture(scope="module")
def crlib():
    from paper_2607_11340_gb300 import build_lib, lib

    build_lib.build()
    return lib


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^CR_API\s+[\w\s\*]+?\b(cr_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(crlib):
    names = declared_functions()
    assert len(names) >= 14
    L = crlib.load()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(crlib.EXPORTS)


def test_struct_layout_matches_c(crlib, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "cr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(cr_robot), sizeof(cr_weights), sizeof(cr_scene), sizeof(cr_task), sizeof(cr_ik_params));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(cr_robot, r_body), offsetof(cr_robot, l_max), offsetof(cr_task, w), offsetof(cr_ik_params, seed), offsetof(cr_ik_params, precision));
  printf("%zu %zu %d\\n", offsetof(cr_scene, prims), offsetof(cr_scene, n_p), CR_PRIM_DOUBLES);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    L = crlib
    py = [C.sizeof(L.cr_robot), C.sizeof(L.cr_weights), C.sizeof(L.cr_scene), C.sizeof(L.cr_task),
          C.sizeof(L.cr_ik_params), L.cr_robot.r_body.offset, L.cr_robot.l_max.offset, L.cr_task.w.offset,
          L.cr_ik_params.seed.offset,
          L.cr_ik_params.precision.offset, L.cr_scene.prims.offset, L.cr_scene.n_p.offset, L.CR_PRIM_DOUBLES]
    assert [int(x) for x in out] == py


def _robot(crlib, n=3):
    r = crlib.cr_robot()
    r.n, r.m, r.n_b = n, 3, 16
    for i in range(n):
        r.L[i], r.r_c[i], r.u_max[i], r.theta_max[i] = 0.1, 0.005, 0.01, 3.14
    r.r_body = 0.005
    return r


def test_invalid_arguments_are_rejected(crlib):
    L = crlib.load()
    r = _robot(crlib)
    dummy = C.c_void_p(256)
    assert L.cr_fk(C.byref(r), dummy, 4, dummy, None, 0, None) == crlib.CR_OK or True  # never launched here
    bad = _robot(crlib)
    bad.n = 0
    assert L.cr_fk(C.byref(bad), dummy, 4, dummy, None, 0, None) == crlib.CR_EINVAL
    assert "robot.n" in crlib.last_error()
    bad = _robot(crlib)
    bad.m = 4
    assert L.cr_fk(C.byref(bad), dummy, 4, dummy, None, 0, None) == crlib.CR_EINVAL
    bad = _robot(crlib)
    bad.L[1] = -1
    assert L.cr_fk_jac(C.byref(bad), dummy, 4, dummy, 0, None) == crlib.CR_EINVAL
    assert L.cr_fk(C.byref(r), None, 4, dummy, None, 0, None) == crlib.CR_EINVAL            # null u
    assert L.cr_fk(C.byref(r), C.c_void_p(257), 4, dummy, None, 0, None) == crlib.CR_EINVAL  # misaligned
    assert L.cr_fk(C.byref(r), dummy, -1, dummy, None, 0, None) == crlib.CR_EINVAL           # negative B
    assert L.cr_fk(C.byref(r), dummy, 4, dummy, None, 7, None) == crlib.CR_EINVAL            # bad dtype
    assert L.cr_fk(C.byref(r), None, 0, None, None, 0, None) == crlib.CR_OK                  # empty batch
    # tasks: too few targets for the batch, bad kind
    t = crlib.cr_task()
    t.kind, t.seeds_per_target, t.targets, t.n_targets = 0, 4, 256, 2
    sc = crlib.cr_scene()
    assert L.cr_cost_grad(C.byref(r), C.byref(sc), C.byref(t), dummy, 9, dummy, None, None, None, 0, None) \
        == crlib.CR_EINVAL
    t.kind = 9
    assert L.cr_cost_grad(C.byref(r), C.byref(sc), C.byref(t), dummy, 8, dummy, None, None, None, 0, None) \
        == crlib.CR_EINVAL
    sc.n_o = 300
    t.kind = 0
    assert L.cr_cost_grad(C.byref(r), C.byref(sc), C.byref(t), dummy, 8, dummy, None, None, None, 0, None) \
        == crlib.CR_EINVAL
    # solver params and workspace size
    p = crlib.cr_ik_params()
    p.S, p.n_final, p.k_init, p.k_final, p.lambda0 = 256, 8, 64, 30, 1e-3
    ws = crlib.cr_ik_workspace_size(r, 100, p)
    assert ws > 0 and ws % 256 == 0
    assert crlib.cr_ik_workspace_size(r, 200, p) > ws
    t = crlib.cr_task()
    t.kind, t.seeds_per_target, t.targets, t.n_targets = 0, 1, 256, 100
    outs = [dummy] * 4
    assert L.cr_solve_ik(C.byref(r), None, C.byref(t), C.byref(p), *outs, dummy, dummy, ws - 256, None) \
        == crlib.CR_EINVAL
    assert "workspace" in crlib.last_error()
    p.n_final = 40
    assert L.cr_solve_ik(C.byref(r), None, C.byref(t), C.byref(p), *outs, dummy, dummy, ws, None) \
        == crlib.CR_EINVAL
    p.n_final, p.S = 8, 300
    assert L.cr_solve_ik(C.byref(r), None, C.byref(t), C.byref(p), *outs, dummy, dummy, ws, None) \
        == crlib.CR_EINVAL


def test_batch_items_are_validated(crlib):
    """Ragged batch: every out-of-range item field, a bad seeds_per_unit and an IK item with H != 1
    are rejected before any device call; the struct layout matches the header."""
    L = crlib.load()
    r = _robot(crlib, n=6)
    w = crlib.cr_weights()
    p = crlib.cr_batch_params()
    p.ik.n_final, p.ik.k_init, p.ik.k_final, p.ik.lambda0 = 8, 16, 10, 1e-3
    p.k_warm, p.k_joint, p.seeds_per_unit = 5, 5, 64
    dummy = C.c_void_p(256)
    good = [(0, 3, 1, 64, 4), (1, 6, 128, 256, 64)]
    bad = [(2, 3, 1, 64, 0), (0, 0, 1, 64, 0), (0, 7, 1, 64, 0), (0, 3, 2, 64, 0), (1, 3, 129, 64, 0),
           (1, 3, 0, 64, 0), (0, 3, 1, 0, 0), (0, 3, 1, 257, 0), (0, 3, 1, 64, 65), (0, 3, 1, 64, -1)]
    outs = [dummy] * 8
    for it in bad:
        items = crlib._batch_items(good + [it])
        assert L.cr_solve_batch(C.byref(r), C.byref(w), items, 3, C.byref(p), *outs, dummy, 1 << 30, None) \
            == crlib.CR_EINVAL, it
        assert crlib.cr_batch_workspace_size(r, items, p) == 0
        assert L.cr_solve_batch_plain(C.byref(r), C.byref(w), items, 3, C.byref(p), *outs, dummy, 1 << 30, None) \
            == crlib.CR_EINVAL, it
    items = crlib._batch_items(good)
    p.seeds_per_unit = 48
    assert L.cr_solve_batch(C.byref(r), C.byref(w), items, 2, C.byref(p), *outs, dummy, 1 << 30, None) \
        == crlib.CR_EINVAL
    assert "seeds_per_unit" in crlib.last_error()
    p.seeds_per_unit, p.seed_regs = 64, 3
    assert L.cr_solve_batch(C.byref(r), C.byref(w), items, 2, C.byref(p), *outs, dummy, 1 << 30, None) \
        == crlib.CR_EINVAL
    assert "seed_regs" in crlib.last_error()
    p.seed_regs = 0
    assert C.sizeof(crlib.cr_batch_item) == 24
    assert crlib.cr_batch_params.k_warm.offset == C.sizeof(crlib.cr_ik_params)


def test_arc_model_is_validated(crlib):
    """Arc model: up to CR_MAX_SEG_ARC segments, 0 < l_min <= l_max, a known model code; the entry
    points that take the tendon model only refuse it; all before any device call."""
    L = crlib.load()
    dummy = C.c_void_p(256)

    def arc(n=3):
        r = _robot(crlib, n)
        r.model = crlib.CR_MODEL_ARC
        for i in range(n):
            r.l_min[i], r.l_max[i] = 0.5, 1.5
        return r

    r = arc()
    for bad in (arc(5), arc()):
        if bad.n == 3:
            bad.l_min[1], bad.l_max[1] = 1.0, 0.9
        assert L.cr_fk(C.byref(bad), dummy, 4, dummy, None, 0, None) == crlib.CR_EINVAL
    bad = arc()
    bad.model = 7
    assert L.cr_fk(C.byref(bad), dummy, 4, dummy, None, 0, None) == crlib.CR_EINVAL
    assert "model" in crlib.last_error()
    # coupled routing (model B): a valid model code, refused by the tendon-only entry points
    rc_ = _robot(crlib, 3)
    rc_.model = crlib.CR_MODEL_COUPLED
    assert L.cr_calibrate(C.byref(rc_), dummy, dummy, 4, dummy, 2, 1e-3, dummy, None, 0, dummy, 1 << 20, None) \
        == crlib.CR_EINVAL
    assert "tendon model" in crlib.last_error()
    # tendon-only entry points
    assert L.cr_calibrate(C.byref(r), dummy, dummy, 4, dummy, 2, 1e-3, dummy, None, 0, dummy, 1 << 20, None) \
        == crlib.CR_EINVAL
    assert "tendon model" in crlib.last_error()
    w = crlib.cr_weights()
    p = crlib.cr_batch_params()
    p.ik.n_final, p.ik.k_init, p.ik.k_final, p.ik.lambda0 = 8, 16, 10, 1e-3
    p.seeds_per_unit = 64
    items = crlib._batch_items([(0, 3, 1, 64, 4)])
    assert L.cr_solve_batch(C.byref(r), C.byref(w), items, 1, C.byref(p), *([dummy] * 8), dummy, 1 << 30, None) \
        == crlib.CR_EINVAL
    assert C.sizeof(crlib.cr_robot) == crlib.cr_robot.l_max.offset + 8 * crlib.CR_MAX_SEG


def test_prm_layout_and_validation(crlib, tmp_path):
    """PRM structs match the C layout; bad roadmap settings, a roadmap count that fits neither a
    shared nor a per-query roadmap, and the arc model are refused before any device call."""
    prog = tmp_path / "prm_layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "cr.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(cr_prm_params), offsetof(cr_prm_params, seed), sizeof(cr_roadmap),
         offsetof(cr_roadmap, wt));
  return 0;
}
""")
    exe = tmp_path / "prm_layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out == [C.sizeof(crlib.cr_prm_params), crlib.cr_prm_params.seed.offset, C.sizeof(crlib.cr_roadmap),
                   crlib.cr_roadmap.wt.offset]
    L = crlib.load()
    dummy = C.c_void_p(256)
    r = _robot(crlib)
    sc = crlib.cr_scene()
    w = crlib.cr_weights()

    def prm(N=64, k=8, nc=4, at=8):
        p = crlib.cr_prm_params()
        p.N, p.k, p.n_check, p.attempts, p.seed = N, k, nc, at, 1
        return p

    m = crlib.cr_roadmap()
    m.R = 2
    for f in ("nodes", "node_ok", "nbr", "row", "col", "wt"):
        setattr(m, f, 256)
    for bad in (prm(N=1), prm(N=2048), prm(k=0), prm(k=64), prm(N=8, k=8), prm(nc=0), prm(nc=65), prm(at=9)):
        assert L.cr_prm_build(C.byref(r), C.byref(sc), C.byref(w), C.byref(bad), C.byref(m), dummy, 1 << 30,
                              None) == crlib.CR_EINVAL
        assert L.cr_prm_workspace_size(C.byref(r), 2, C.byref(bad)) == 0
    good = prm()
    assert L.cr_prm_workspace_size(C.byref(r), 2, C.byref(good)) >= 2 * 64 * 8 + 2 * 64 * 2 * 4
    assert L.cr_prm_build(C.byref(r), C.byref(sc), C.byref(w), C.byref(good), C.byref(m), dummy, 16,
                          None) == crlib.CR_EINVAL  # workspace too small
    assert "workspace" in crlib.last_error()
    # R = 2 roadmaps serve neither 3 queries (needs R = 1 or R = P) ...
    assert L.cr_prm_query(C.byref(r), C.byref(sc), C.byref(w), C.byref(good), C.byref(m), dummy, dummy, 3, 8,
                          dummy, dummy, dummy, None) == crlib.CR_EINVAL
    assert "roadmap count" in crlib.last_error()
    # ... nor a horizon T outside 2..256
    assert L.cr_prm_query(C.byref(r), C.byref(sc), C.byref(w), C.byref(good), C.byref(m), dummy, dummy, 2, 1,
                          dummy, dummy, dummy, None) == crlib.CR_EINVAL
    r.model = crlib.CR_MODEL_ARC
    for i in range(3):
        r.l_min[i], r.l_max[i] = 0.5, 1.5
    assert L.cr_prm_build(C.byref(r), C.byref(sc), C.byref(w), C.byref(good), C.byref(m), dummy, 1 << 30,
                          None) == crlib.CR_EINVAL
    assert "tendon model" in crlib.last_error()


def test_self_contact_weight_is_validated(crlib):
    """weights.rho_s: negative values are rejected by every entry point that takes weights, and the
    solvers built without the self-contact rows (path, batch, plain, PRM) refuse rho_s > 0, all before
    any device call."""
    L = crlib.load()
    r = _robot(crlib, n=4)
    dummy = C.c_void_p(256)
    t = crlib.cr_task()
    t.kind, t.seeds_per_target, t.targets, t.n_targets = 0, 1, 256, 4
    t.w.rho_s = -1.0
    assert L.cr_cost_grad(C.byref(r), None, C.byref(t), dummy, 4, dummy, None, None, None, 0, None) == crlib.CR_EINVAL
    assert "rho_s" in crlib.last_error()
    p = crlib.cr_ik_params()
    p.S, p.n_final, p.k_init, p.k_final, p.lambda0 = 64, 8, 8, 8, 1e-3
    pt = crlib.cr_path_task()
    pt.waypoints, pt.P, pt.H = 256, 2, 4
    pt.w.rho_s = 1.0
    outs = [dummy] * 6
    assert L.cr_solve_path(C.byref(r), None, C.byref(pt), C.byref(p), 5, 5, *outs, dummy, 1 << 30, None) \
        == crlib.CR_EINVAL
    assert "self-contact" in crlib.last_error()
    t.w.rho_s = 1.0
    assert L.cr_solve_ik_plain(C.byref(r), None, C.byref(t), C.byref(p), *([dummy] * 5), dummy, 1 << 30, None) \
        == crlib.CR_EINVAL
    w = crlib.cr_weights()
    w.rho_s = 1.0
    bp = crlib.cr_batch_params()
    bp.ik.n_final, bp.ik.k_init, bp.ik.k_final, bp.ik.lambda0 = 8, 16, 10, 1e-3
    bp.k_warm, bp.k_joint, bp.seeds_per_unit = 5, 5, 64
    items = crlib._batch_items([(0, 3, 1, 64, 0)])
    assert L.cr_solve_batch(C.byref(r), C.byref(w), items, 1, C.byref(bp), *([dummy] * 8), dummy, 1 << 30, None) \
        == crlib.CR_EINVAL


def test_scene_primitives_are_validated(crlib):
    """n_p outside 0..CR_MAX_SPHERES - n_o, a NULL or misaligned primitive array, and primitives given
    to the PRM entry points are rejected before any device call."""
    L = crlib.load()
    dummy = C.c_void_p(256)
    r = _robot(crlib)
    t = crlib.cr_task()
    t.kind, t.seeds_per_target, t.targets, t.n_targets = 0, 1, 256, 8

    def cost_grad(sc):
        return L.cr_cost_grad(C.byref(r), C.byref(sc), C.byref(t), dummy, 8, dummy, None, None, None, 0, None)

    sc = crlib.cr_scene()
    sc.n_p = -1
    assert cost_grad(sc) == crlib.CR_EINVAL
    sc.n_o, sc.spheres, sc.n_p, sc.prims = 200, 256, 57, 256
    assert cost_grad(sc) == crlib.CR_EINVAL and "n_p" in crlib.last_error()
    sc.n_o, sc.n_p, sc.prims = 0, 4, None
    assert cost_grad(sc) == crlib.CR_EINVAL and "prims" in crlib.last_error()
    sc.prims = 260
    assert cost_grad(sc) == crlib.CR_EINVAL
    sc.prims = 256
    w = crlib.cr_weights()
    p = crlib.cr_prm_params()
    p.N, p.k, p.n_check, p.attempts, p.seed = 64, 8, 4, 8, 1
    m = crlib.cr_roadmap()
    m.R = 1
    for f in ("nodes", "node_ok", "nbr", "row", "col", "wt"):
        setattr(m, f, 256)
    assert L.cr_prm_build(C.byref(r), C.byref(sc), C.byref(w), C.byref(p), C.byref(m), dummy, 1 << 30,
                          None) == crlib.CR_EINVAL
    assert "sphere obstacles only" in crlib.last_error()
