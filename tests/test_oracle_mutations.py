"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a temporary copy of oracle/hf_oracle.c
(a dropped term, a flipped comparison, a wrong index, a transposed operand),
compiles it, and runs the whole pin suite (test_oracle_pins.py) against that
copy in a child process.  The suite has to fail for every planted mistake.
MARCH_MUTANTS does the same for the fixed-step march oracle (oracle/march.py)
against its pins (test_march_pins.py).  The committed oracles are never
modified.
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
    "diffuse sign flipped on the -X face": (
        "case OR_FACE_NX: ndl = -(double)L[0] / n; break;",
        "case OR_FACE_NX: ndl = (double)L[0] / n; break;"),
    "+Y face reads the x component": (
        "case OR_FACE_PY: ndl = (double)L[1] / n; break;",
        "case OR_FACE_PY: ndl = (double)L[0] / n; break;"),
    "-Z face takes the +Z normal": (
        "case OR_FACE_NZ: ndl = -(double)L[2] / n; break;",
        "case OR_FACE_NZ: ndl = (double)L[2] / n; break;"),
    "ambient and diffuse weights swapped": (
        "double k = OR_KA + OR_KD * ndl * (visible ? 1.0 : 0.0);",
        "double k = OR_KD + OR_KA * ndl * (visible ? 1.0 : 0.0);"),
    "shadow factor ignored": (
        "double k = OR_KA + OR_KD * ndl * (visible ? 1.0 : 0.0);",
        "double k = OR_KA + OR_KD * ndl;"),
    "colour rounded by truncation": (
        "uint32_t q = (uint32_t)floor(255.0 * v + 0.5);",
        "uint32_t q = (uint32_t)floor(255.0 * v);"),
    "albedo channels reversed": (
        "double v = a[ch] * k;", "double v = a[2 - ch] * k;"),
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


MARCH_SRC = os.path.join(ROOT, "oracle", "march.py")

MARCH_MUTANTS = {
    "spacing over steps instead of steps + 1": (
        "dt = (t_end / f32(steps + 1)).astype(f32)",
        "dt = (t_end / f32(steps)).astype(f32)"),
    "bisection keeps the empty end": (
        "b = np.where(found & s, m, b)\n        a = np.where(found & ~s, m, a)",
        "a = np.where(found & s, m, a)\n        b = np.where(found & ~s, m, b)"),
    "no clip at z = 0": (
        "t_end = np.where(down & (t_z < t_end), t_z, t_end).astype(f32)", ""),
    "one bisection fewer": (
        "for _ in range(bisections):", "for _ in range(max(bisections - 1, 0)):"),
    "samples start at t = 0": (
        "for i in range(1, steps + 1):", "for i in range(0, steps):"),
    "open floor interval": (
        "floor_ = z <= h0", "floor_ = z < h0"),
    "slab test ignores the underside": (
        "upper = slab & (z >= h1) & (z <= h2)", "upper = slab & (z <= h2)"),
    "depth without the direction length": (
        "depth = (b * length).astype(f32)", "depth = b"),
    "bracket start one sample late": (
        "a = np.where(new, (f32(i - 1) * dt).astype(f32), a)",
        "a = np.where(new, (f32(i) * dt).astype(f32), a)"),
}


@pytest.mark.parametrize("name", sorted(MARCH_MUTANTS))
def test_march_pins_catch_planted_mistake(name, tmp_path):
    old, new = MARCH_MUTANTS[name]
    src = open(MARCH_SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once: " + name
    mut = tmp_path / "march_mutant.py"
    mut.write_text(src.replace(old, new).replace("from . import ray_dirs", "from oracle import ray_dirs"))
    env = dict(os.environ, HF_MARCH_ORACLE=str(mut))
    r = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_march_pins.py"),
         "-x", "-q", "-p", "no:cacheprovider"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake survived the march pins: " + name


def test_march_pins_pass_on_the_unmodified_copy(tmp_path):
    """The loader path itself: an unmodified copy passes every march pin."""
    mut = tmp_path / "march_copy.py"
    mut.write_text(open(MARCH_SRC).read().replace("from . import ray_dirs",
                                                  "from oracle import ray_dirs"))
    env = dict(os.environ, HF_MARCH_ORACLE=str(mut))
    r = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_march_pins.py"),
         "-x", "-q", "-p", "no:cacheprovider"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
