"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a temporary copy of oracle/hf_oracle.c
(a dropped term, a flipped comparison, a wrong index, a transposed operand),
compiles it, and runs the whole pin suite (test_oracle_pins.py) against that
copy in a child process.  The suite has to fail for every planted mistake.
The committed oracle is never modified.
"""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hf_oracle.c")

MUTANTS = {
    "open floor interval": (
        "int in_floor = zsign(oz, dz, tin, h0 * OR_S) <= 0;",
        "int in_floor = zsign(oz, dz, tin, h0 * OR_S) < 0;"),
    "open slab top": (
        "zsign(oz, dz, tin, h2 * OR_S) <= 0;",
        "zsign(oz, dz, tin, h2 * OR_S) < 0;"),
    "corner steps one axis": (
        "tout = tx; step_x = step_y = 1;",
        "tout = tx; step_x = 1; step_y = 0;"),
    "no right-limit start cell": (
        "if (d[0] < 0 && cx * OR_S == o[0]) cx -= 1;", ""),
    "entry faces swapped": (
        "entry_face = d[0] > 0 ? OR_FACE_NX : OR_FACE_PX;",
        "entry_face = d[0] > 0 ? OR_FACE_PX : OR_FACE_NX;"),
    "slab top time uses h1": (
        "r->t = (rat){oz - h2 * OR_S, -dz};",
        "r->t = (rat){oz - h1 * OR_S, -dz};"),
    "depth drops dz": (
        "double dn = sqrt((double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2]);",
        "double dn = sqrt((double)d[0] * d[0] + (double)d[1] * d[1]);"),
    "underside crossing open": (
        "zsign(oz, dz, tout, h1 * OR_S) >= 0",
        "zsign(oz, dz, tout, h1 * OR_S) > 0"),
    "early miss one level low": (
        "255 * (int64_t)OR_S", "254 * (int64_t)OR_S"),
    "time comparison reversed": (
        "return (i128)a.num * b.den < (i128)b.num * a.den;",
        "return (i128)a.num * b.den > (i128)b.num * a.den;"),
    "z test operands transposed": (
        "i128 v = (i128)(oz - level) * t.den + (i128)t.num * dz;",
        "i128 v = (i128)(oz - level) * t.num + (i128)t.den * dz;"),
    "pyramid min becomes max": (
        "if (b < mn1) mn1 = b;", "if (b > mn1) mn1 = b;"),
    "shadow origin pushed inward": (
        "case OR_FACE_PZ: p[2] += 1; break;", "case OR_FACE_PZ: p[2] -= 1; break;"),
    "image rows flipped": (
        "int64_t a = 2 * px + 1 - w, b = h - 1 - 2 * py;",
        "int64_t a = 2 * px + 1 - w, b = 2 * py + 1 - h;"),
    "y exit boundary off by one": (
        "if (d[1] > 0) ty = (rat){(cy + 1) * OR_S - o[1], d[1]};",
        "if (d[1] > 0) ty = (rat){(cy + 2) * OR_S - o[1], d[1]};"),
}


def _run_pins(lib):
    env = dict(os.environ, HF_ORACLE_LIB=lib)
    return subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
         "-x", "-q", "-p", "no:cacheprovider"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           "-o", lib, str(mut), "-lm"])
    r = _run_pins(lib)
    assert r.returncode != 0, "planted mistake survived the pins: " + name
