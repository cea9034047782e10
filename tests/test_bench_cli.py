"""bench.py on the CPU: every workload builds, the reference arm's JSON line
has the contract's keys, and the traffic lookup follows the profile summary."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c4pair"])
def test_workloads_build(name):
    import bench

    wl = bench.workload(name, frames_per_step=7)
    assert wl["cells"].ndim == 2 and len(wl["cams"]) >= 1 and wl["name"]
    if name.startswith("c4"):
        assert "7 frames" in wl["name"] and len(wl["cams"]) == 1000
    if name == "c4pair":
        from oracle import pairs

        assert wl["texels"].nbytes == 64 << 20
        assert (pairs.decode(wl["texels"]) == wl["cells"]).all()


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
              "cpu_baseline", "e2e", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_traffic_lookup_tracks_the_kernel_source_and_launch():
    import bench

    f = bench._profile_fields("c3")
    path = os.path.join(ROOT, "profiles", "trace_batched_c3.md")
    text = open(path).read()
    if bench.trace_source_hash() not in text:
        assert f is None and bench._profiled_traffic("c3", 1000, "8x16", 5) is None
        return
    tile, mip = f["launch_tile"], int(f["launch_mip_start"])
    t = bench._profiled_traffic("c3", 1000, tile, mip)
    assert t is not None and t == pytest.approx(1000 * float(f["dram_bytes_per_ray"]))
    other = "4x8" if tile != "4x8" else "8x4"
    assert bench._profiled_traffic("c3", 1000, other, mip) is None
    assert bench._profiled_traffic("c3", 1000, tile, 2) is None
    assert bench._profiled_traffic("no_such_workload", 1000, tile, mip) is None
    for key, v in f.items():  # figures taken for other launch configurations
        if key.startswith("dram_bytes_per_ray@"):
            t2, m2 = key.split("@")[1].split("/")
            assert bench._profiled_traffic("c3", 1000, t2, int(m2)) == pytest.approx(1000 * float(v))


def test_alu_roofline_only_for_the_profiled_launch():
    import bench

    f = bench._profile_fields("c3")
    if f is None:
        assert bench._alu_roofline("c3", 188006400, 30.0, "8x16", 6, 152, 2070.0) is None
        return
    tile, mip = f["launch_tile"], int(f["launch_mip_start"])
    r = bench._alu_roofline("c3", 188006400, 30.0, tile, mip, 152, 2070.0)
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.5
    assert r["peak"] == pytest.approx(152 * 4 * 2070e6 / 1e12)
    other = "4x8" if tile != "4x8" else "8x4"
    assert bench._alu_roofline("c3", 188006400, 30.0, other, mip, 152, 2070.0) is None
    assert bench._alu_roofline("c3", 188006400, 30.0, tile, 2, 152, 2070.0) is None
    for key, v in f.items():
        if key.startswith("warp_instructions_per_primary_ray@"):
            t2, m2 = key.split("@")[1].split("/")
            r2 = bench._alu_roofline("c3", 188006400, 30.0, t2, int(m2), 152, 2070.0)
            assert r2["warp_instructions_per_primary_ray"] == pytest.approx(float(v))


def test_cpu_baseline_samples_every_camera_in_proportion():
    """The host-core oracle figure samples the same fraction of every
    camera's pixels (the workload's own mix), calls the oracle once per
    camera, and reports an all-core and a single-core rate with the CPU."""
    import bench

    wl = bench.workload("c3", scale=16)
    cams = wl["cams"]
    pix = bench._pixel_sample(cams, 0.05, seed=3)
    assert len(pix) == len(cams)
    for c, p in zip(cams, pix):
        n = int(c["w"]) * int(c["h"])
        assert (np.diff(p.astype(np.int64)) > 0).all() and p.max() < n
        assert abs(len(p) - 0.05 * n) <= 0.05 * 0.05 * n + 16
    wl1 = bench.workload("c1")
    b = bench.cpu_baseline(wl1, budget_s=0.3)
    assert b["kind"] == "oracle" and b["value"] > 0 and b["cores"] == os.cpu_count()
    assert b["single_core"]["value"] > 0 and b["nproc"] == os.cpu_count()
    assert "cpu_model" in b
