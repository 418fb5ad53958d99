"""The pins catch plausible mistakes in the oracle.

Each case copies the oracle's C source, plants one mistake (a changed
factor, a flipped comparison, a transposed operand), compiles the copy with
the oracle's own flags and runs the pin tests that should see it against
that build (loaded through ORC_LIB, in a child process).  Those tests must
fail; the unchanged oracle passes them in the ordinary test run.
"""
import os
import subprocess
import sys

import pytest

import oracle.build as ob

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REPRO = "tests/test_oracle_reprojection.py"
TILT = "tests/test_oracle_svgf.py::test_atrous_depth_weight_on_a_tilted_plane"

# (name, text in the source, planted replacement, tests that must fail)
MUTANTS = [
    ("slope term x10", "volatile float zsl = 2.0f * slope;", "volatile float zsl = 20.0f * slope;",
     [REPRO + "::test_depth_tolerance_is_two_slopes"]),
    ("slope term dropped", "volatile float zsl = 2.0f * slope;", "volatile float zsl = 0.0f * slope;",
     [REPRO + "::test_grazing_floor_keeps_one_pixel_taps"]),
    ("slope term x1", "volatile float zsl = 2.0f * slope;", "volatile float zsl = 1.0f * slope;",
     [REPRO + "::test_depth_tolerance_is_two_slopes"]),
    ("larger one-sided difference", "? ((fabsf(dm) < fabsf(dp)) ? dm : dp)", "? ((fabsf(dm) > fabsf(dp)) ? dm : dp)",
     [REPRO + "::test_depth_tolerance_is_two_slopes"]),
    ("slope without the sign test", "((dp > 0.0f && dm > 0.0f) || (dp < 0.0f && dm < 0.0f))", "1",
     [REPRO + "::test_ridge_slope_is_zero"]),
    ("a-trous slope without the sign test", "((dp > 0.0 && dm > 0.0) || (dp < 0.0 && dm < 0.0))", "1",
     ["tests/test_oracle_svgf.py::test_atrous_ridge_is_filtered_along_itself"]),
    ("depth weight offset without the step",
     "double wz = w_depth(zn[4 * p], zn[4 * q], g, -(double)i * step,\n"
     "                                                -(double)j * step, P);",
     "double wz = w_depth(zn[4 * p], zn[4 * q], g, -(double)i,\n"
     "                                                -(double)j, P);", [TILT]),
    ("depth weight gradient transposed", "double den = P->sigma_z * fabs(g[0] * ox + g[1] * oy) + P->eps_z;",
     "double den = P->sigma_z * fabs(g[1] * ox + g[0] * oy) + P->eps_z;", [TILT]),
    ("depth weight without sigma_z", "double den = P->sigma_z * fabs(g[0] * ox + g[1] * oy) + P->eps_z;",
     "double den = fabs(g[0] * ox + g[1] * oy) + P->eps_z;", [TILT]),
]


@pytest.mark.parametrize("name,old,new,tests", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, tests):
    src = open(ob.SRC).read()
    assert src.count(old) == 1, f"mutation site of '{name}' not found once in the oracle"
    mutant = tmp_path / "dhrs_oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libdhrs_oracle_mutant.so"
    subprocess.run(["gcc", *ob.CFLAGS, str(mutant), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, ORC_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *tests],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"'{name}' was not caught:\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}"
