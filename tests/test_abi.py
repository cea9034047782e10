"""The C-ABI library loads, exports every declared symbol, and its host-only
functions behave (no GPU needed: nothing here launches a kernel)."""

import ctypes
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hf():
    import __graft_entry__

    __graft_entry__.build_library()
    import paper_2608_17390_gb300 as m

    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hf_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(hf):
    names = _declared()
    assert len(names) >= 10
    lib = ctypes.CDLL(hf.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi(hf):
    for n in _declared():
        assert callable(getattr(hf, n)), n


def test_header_constants_match_the_binding(hf):
    """Every numeric #define HF_* in include/ has the same value in the binding."""
    seen = 0
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        for name, val in re.findall(r"#define\s+(HF_\w+)\s+\(?(-?(?:0x[0-9A-Fa-f]+|\d+))u?\)?", src):
            if hasattr(hf, name):
                assert getattr(hf, name) == int(val, 0), name
                seen += 1
    assert seen >= 15


def test_strerror(hf):
    for code in range(0, -7, -1):
        assert hf.hf_strerror(code) and hf.hf_strerror(code) != "unknown error"
    assert hf.hf_strerror(-99) == "unknown error"


POSES = [(128.5, 16.5, 140.0, 0.0, -35.0, 60.0, 320, 240),
         (1024.5, 1024.5, 107.0, 211.3, 0.0, 90.0, 1920, 1080),
         (3.25, 7.75, 2.0, 359.9, -89.0, 75.0, 641, 359),
         (2000.0, 16000.0, 250.5, 45.0, 30.0, 120.0, 1, 1)]


@pytest.mark.parametrize("pose", POSES)
def test_camera_from_pose_matches_the_input_generator(hf, pose):
    a = hf.hf_camera_from_pose(*pose)
    b = synth.pose_to_camera(*pose)
    assert tuple(a["o"]) == b[0] and tuple(a["f"]) == b[1]
    assert tuple(a["r"]) == b[2] and tuple(a["u"]) == b[3]
    assert (int(a["w"]), int(a["h"])) == (b[4], b[5])


def test_camera_from_pose_rejects(hf):
    with pytest.raises(hf.HFError):
        hf.hf_camera_from_pose(0, 0, 0, 0, 0, 180.0, 10, 10)
    with pytest.raises(hf.HFError):
        hf.hf_camera_from_pose(0, 0, 0, 0, 0, 60.0, 0, 10)
    with pytest.raises(hf.HFError):
        hf.hf_camera_from_pose(0, 0, 0, 0, 0, 60.0, 16385, 10)


def test_validate_camera(hf):
    ok = synth.camera_array([synth.pose_to_camera(10.5, 10.5, 50, 30, -20, 90, 1920, 1080)])[0]
    assert hf.hf_validate_camera(64, 64, ok) == hf.HF_OK
    bad = ok.copy()
    bad["o"][0] = 64 * 65536          # x on the far grid edge: outside [0, W)
    assert hf.hf_validate_camera(64, 64, bad) == hf.HF_E_INVALID_ARG
    bad = ok.copy()
    bad["o"][2] = 1 << 28             # z too high
    assert hf.hf_validate_camera(64, 64, bad) == hf.HF_E_INVALID_ARG
    bad = ok.copy()
    bad["o"][1] = -1
    assert hf.hf_validate_camera(64, 64, bad) == hf.HF_E_INVALID_ARG
    wide = synth.camera_array([synth.pose_to_camera(10.5, 10.5, 50, 30, -20, 150, 1920, 1080)])[0]
    assert hf.hf_validate_camera(64, 64, wide) == hf.HF_E_INVALID_ARG  # |d| reaches 2^21
    one = synth.camera_array([synth.ray_camera((5, 5, 5), ((1 << 21) - 1, 0, 0))])[0]
    assert hf.hf_validate_camera(64, 64, one) == hf.HF_OK
    one["f"][0] = 1 << 21
    assert hf.hf_validate_camera(64, 64, one) == hf.HF_E_INVALID_ARG


def test_validate_cells(hf):
    good = synth.pack_cells([5, 0, 7, 9], [0, 0, 9, 10], [0, 0, 9, 12], [1, 2, 3, 7])
    assert hf.hf_validate_cells(good) == (hf.HF_OK, None)
    for h0, h1, h2 in [(5, 3, 9), (5, 0, 4), (5, 9, 8), (5, 5, 5)]:
        cells = good.copy()
        cells[2] = synth.pack_cells(h0, h1, h2, 0)
        assert hf.hf_validate_cells(cells) == (hf.HF_E_INVALID_ARG, 2), (h0, h1, h2)


def test_create_rejects_before_touching_the_gpu(hf):
    with pytest.raises(hf.HFError) as e:
        hf.hf_create(np.zeros((0, 4), np.uint32))
    assert e.value.code == hf.HF_E_INVALID_ARG
    with pytest.raises(hf.HFError) as e:
        hf.hf_create(np.full((4, 4), synth.pack_cells(5, 3, 9, 0), np.uint32))
    assert e.value.code == hf.HF_E_INVALID_ARG
    with pytest.raises(hf.HFError) as e:
        hf.hf_create(np.zeros((4, 16385), np.uint32))
    assert e.value.code == hf.HF_E_INVALID_ARG


def test_camera_dtype_matches_c_layout(hf):
    assert hf.CAMERA_DTYPE.itemsize == ctypes.sizeof(hf.hf_camera) == 72
    assert synth.CAMERA_DTYPE == hf.CAMERA_DTYPE
    assert ctypes.sizeof(hf.hf_outputs) == 48
    assert ctypes.sizeof(hf.hf_render_opts) == 40


def test_struct_layouts_match_the_header(hf, tmp_path):
    """sizeof / offsetof of the ABI's structs as the C compiler lays them out,
    against the binding's ctypes mirrors."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    fields = {"hf_camera": ("origin", "w"), "hf_outputs": ("hit_cell", "shadow"),
              "hf_render_opts": ("tile_w", "cuda_stream"),
              "hf_request": ("arrival", "cam", "x0", "cells", "outs"),
              "hf_request_result": ("done", "batch"),
              "hf_serve_opts": ("output_budget", "mip_start")}
    lines = []
    for t, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (t, t))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (t, f, t, f))
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"hf.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for t, fs in fields.items():
        ct = getattr(hf, t)
        assert int(got[t]) == ctypes.sizeof(ct), t
        for f in fs:
            assert int(got["%s.%s" % (t, f)]) == getattr(ct, f).offset, (t, f)


def test_serve_replay_rejects_before_touching_the_gpu(hf):
    opts = hf.hf_serve_opts(8, 8, 1 << 30, 0, 0, 0, hf.HF_MIP_AUTO)
    assert hf.lib.hf_serve_replay(None, None, 0, ctypes.byref(opts), None) == hf.HF_E_INVALID_ARG
    with pytest.raises(ValueError):
        hf.hf_serve_replay(None, [{"kind": "render", "arrival": 0.0}], outputs=[])


def test_pair_validation_agrees_with_the_oracle(hf):
    """The library's paired-texel check and the oracle's decoder-side check
    accept and reject the same grids, at the same first bad pair."""
    import json

    from oracle import pairs as opairs

    g = json.load(open(os.path.join(ROOT, "tests", "golden", "pair_codec.json")))
    for case in g["valid"] + g["invalid"]:
        t = np.array(case["texels"], dtype=np.uint16)
        ok, bad = opairs.validate(t)
        rc, lbad = hf.hf_validate_pairs(t)
        assert (rc == hf.HF_OK) == ok and lbad == bad, case["name"]
    rng = np.random.default_rng(3)
    for _ in range(200):
        t = rng.integers(0, 1 << 16, (3, 4)).astype(np.uint16)
        t[:, 0::2] &= 0x87FF  # keep many pairs near the valid set
        t[:, 1::2] &= 0x87FF
        ok, bad = opairs.validate(t)
        rc, lbad = hf.hf_validate_pairs(t)
        assert (rc == hf.HF_OK) == ok and lbad == bad


def test_create_pairs_rejects_before_touching_the_gpu(hf):
    for t in (np.zeros((4, 3), np.uint16),                       # odd width
              np.array([[5 | (0x80 << 8), 100]], np.uint16),     # flag on one texel
              np.zeros((0, 4), np.uint16)):
        with pytest.raises(hf.HFError) as e:
            hf.hf_create_pairs(t)
        assert e.value.code == hf.HF_E_INVALID_ARG


def test_scatter_footprint_agrees_with_the_input_helper(hf):
    from synth.scatter import footprint_for

    cams = list(synth.config_c1()["cams"]) + [
        synth.camera_array([synth.pose_to_camera(50.0, 60.0, z, yaw, p, fov, 64, 40)])[0]
        for z, yaw, p, fov in ((10.0, 0.0, 0.0, 90.0), (200.0, 33.0, -90.0, 75.0),
                               (120.0, 250.0, -60.0, 60.0), (30.0, 100.0, 20.0, 80.0))]
    for cam in cams:
        a = np.array(hf.hf_scatter_footprint(cam))
        b = np.array(footprint_for(cam))
        assert np.allclose(a, b, rtol=1e-5, atol=1e-4), (a, b)
