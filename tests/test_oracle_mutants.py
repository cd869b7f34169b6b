"""The pins of tests/test_oracle_pins.py and tests/test_oracle_prims.py catch plausible mistakes in the
oracle.

Each case copies oracle/cr_oracle.cpp to a temporary directory, plants one mistake by a textual
substitution (the pattern must occur exactly once), builds that copy, and runs the pin that should
catch it in a child process pointed at the copy (CR_ORACLE_LIB). The pin must fail there; run
against the real oracle (in its own test module) it passes. Nothing here touches the oracle
the other tests load.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cr_oracle.cpp")

# (name, pattern, replacement, pin expected to fail[, the pin's test module])
MUTANTS = [
    ("pg_growth_x2", "      alpha *= 1.25;", "      alpha *= 2.0;", "pin_pg_interior"),
    ("pg_stale_gradient", "{ x[a] = x1[a]; g[a] = g1[a]; }", "{ x[a] = x1[a]; }", "pin_pg_projected"),
    ("pg_unnormalised_step", "const T scale = re(gn) > 0 ? alpha / gn : T(0);", "const T scale = alpha;",
     "pin_pg_interior"),
    ("pg_shrink_quarter", "    } else {\n      alpha *= 0.5;", "    } else {\n      alpha *= 0.25;",
     "pin_pg_stall_at_vertex"),
    ("lm_reject_nu_kept", "  st.lambda *= st.nu;\n  st.nu *= 2.0;\n  return 0;\n}\n\n// One LM iteration",
     "  st.lambda *= st.nu;\n  return 0;\n}\n\n// One LM iteration", "pin_lm_rejections"),
    ("lm_reject_lambda_x2", "  st.lambda *= st.nu;\n  st.nu *= 2.0;\n  return 0;\n}\n\n// One LM iteration",
     "  st.lambda *= 2.0;\n  st.nu *= 2.0;\n  return 0;\n}\n\n// One LM iteration", "pin_lm_rejections"),
    ("lm_accept_nu_not_reset", "    st.nu = 2.0;\n    for (int a = 0; a < nx; ++a) x[a] = xn[a];",
     "    for (int a = 0; a < nx; ++a) x[a] = xn[a];", "pin_lm_rejections"),
    ("lm_gain_cube_dropped", "st.lambda *= std::max(1.0 / 3.0, 1.0 - t * t * t);",
     "st.lambda *= std::max(1.0 / 3.0, 1.0 - t * t);", "pin_lm_gain_ratio_branch"),
    ("count_fma_twice", "static inline Cnt operator*(Cnt x, Cnt y) {\n  g_tally.f_flop++;",
     "static inline Cnt operator*(Cnt x, Cnt y) {\n  g_tally.f_flop += 2;", "pin_opcounts"),
    ("count_tangent_product_2", "  if (x.a && y.a) g_tally.t_flop += 3;\n  else if (x.a || y.a) g_tally.t_flop += 1;\n  return Cnt(x.v * y.v",
     "  if (x.a && y.a) g_tally.t_flop += 2;\n  else if (x.a || y.a) g_tally.t_flop += 1;\n  return Cnt(x.v * y.v",
     "pin_opcounts"),
    ("count_tangent_sum_either", "static inline Cnt operator+(Cnt x, Cnt y) {\n  g_tally.f_flop++;\n  if (x.a && y.a)",
     "static inline Cnt operator+(Cnt x, Cnt y) {\n  g_tally.f_flop++;\n  if (x.a || y.a)", "pin_opcount_ik_one_segment"),
    ("box_rotation_transposed", "T p = T(R[0][a]) * w[0] + T(R[1][a]) * w[1] + T(R[2][a]) * w[2];",
     "T p = T(R[a][0]) * w[0] + T(R[a][1]) * w[1] + T(R[a][2]) * w[2];", "test_box_distance_outside_vs_qp",
     "test_oracle_prims"),
    ("capsule_end_unclamped", "    if (re(t) > 1.0) t = T(1.0);\n", "", "test_capsule_end_caps_and_middle",
     "test_oracle_prims"),
    ("box_inside_nearest_face_min", "      if (re(q[a]) > re(m)) m = q[a];", "      if (re(q[a]) < re(m)) m = q[a];",
     "test_box_distance_inside_is_minus_nearest_face", "test_oracle_prims"),
    ("clearance_reach_without_body", "        const double reach = ob[1] + rb.rbody + W.delta;",
     "        const double reach = ob[1] + W.delta;", "test_clearance_cost_with_primitives", "test_oracle_prims"),
]


def _build(tmp, name, pat, rep):
    src = open(SRC).read()
    assert src.count(pat) == 1, (name, src.count(pat))
    mdir = os.path.join(tmp, name)
    os.makedirs(mdir)
    cpp = os.path.join(mdir, "cr_oracle.cpp")
    with open(cpp, "w") as f:
        f.write(src.replace(pat, rep))
    so = os.path.join(mdir, "libcr_oracle.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", cpp, "-o", so],
                   check=True, capture_output=True)
    return so


@pytest.fixture(scope="module")
def mutant_libs():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            futs = {m[0]: ex.submit(_build, tmp, m[0], m[1], m[2]) for m in MUTANTS}
            yield {k: f.result() for k, f in futs.items()}


def _module(m):
    return m[4] if len(m) > 4 else "test_oracle_pins"


def _run_pin(so, pin, module="test_oracle_pins"):
    code = ("import sys; sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r}); import oracle; "
            "import {module} as t; t.{pin}(oracle)").format(root=ROOT, tests=os.path.join(ROOT, "tests"), pin=pin,
                                                           module=module)
    env = dict(os.environ, CR_ORACLE_LIB=so)
    return subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)


@pytest.mark.parametrize("name,pin,module", [(m[0], m[3], _module(m)) for m in MUTANTS])
def test_pin_catches_mutant(mutant_libs, name, pin, module):
    res = _run_pin(mutant_libs[name], pin, module)
    assert res.returncode != 0, f"{pin} passed on the mutant {name}"
    assert "AssertionError" in res.stderr, res.stderr[-2000:]


def test_pins_pass_on_an_unmutated_copy(tmp_path):
    """Control: the same build recipe without a mutation passes every pin."""
    src = open(SRC).read()
    cpp = tmp_path / "cr_oracle.cpp"
    cpp.write_text(src)
    so = str(tmp_path / "libcr_oracle.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-pthread", str(cpp), "-o", so],
                   check=True, capture_output=True)
    for pin, module in sorted({(m[3], _module(m)) for m in MUTANTS}):
        res = _run_pin(so, pin, module)
        assert res.returncode == 0, (pin, res.stderr[-2000:])
