"""Host logic of bench.py's roofline inputs: figures are read from a committed
ncu summary only while its kernel-source hash matches the current sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, sha, body):
    p = tmp_path / "summary.md"
    p.write_text(f"# a kernel\n\n    kernel_source_sha: {sha}\n{body}\n")
    return str(p)


def test_profile_value_needs_the_current_source_hash(tmp_path):
    sha = bench.kernel_source_hash()
    good = _summary(tmp_path, sha, "    dram_bytes_per_launch: 449384448\n    fp32_flops_per_update: 1090.19")
    assert bench.profile_value(good, "dram_bytes_per_launch") == 449384448.0
    assert bench.profile_value(good, "fp32_flops_per_update") == 1090.19
    assert bench.profile_value(good, "missing_key") is None
    stale = _summary(tmp_path, "0" * 16, "    dram_bytes_per_launch: 1")
    assert bench.profile_value(stale, "dram_bytes_per_launch") is None
    assert bench.profile_value(str(tmp_path / "absent.md"), "dram_bytes_per_launch") is None


def test_fp64_figures_hash_only_the_fp64_kernel_body(tmp_path):
    sha = bench.kernel_source_hash(bench.FP64_KERNEL_SOURCES)
    assert sha != bench.kernel_source_hash()
    p = _summary(tmp_path, sha, "    fp64_flops_per_update: 1085")
    assert bench.profile_value(p, "fp64_flops_per_update", bench.FP64_KERNEL_SOURCES) == 1085.0
    assert bench.profile_value(p, "fp64_flops_per_update") is None


def test_step_traffic_of_other_workloads(tmp_path, monkeypatch):
    assert bench.step_traffic("sweep", "fp64") is None              # not profiled
    sha = bench.kernel_source_hash(bench.STEP_SOURCES["fp32"])
    p = _summary(tmp_path, sha, "    dram_bytes_per_step: 123456")
    monkeypatch.setattr(bench, "STEP_PROFILES", {("ellipsoid", "fp32"): p})
    assert bench.step_traffic("ellipsoid", "fp32") == 123456.0
    q = _summary(tmp_path, bench.kernel_source_hash(bench.STEP_SOURCES["bf16_shifted"]),
                 "    dram_bytes_per_step: 1")
    monkeypatch.setattr(bench, "STEP_PROFILES", {("ellipsoid", "fp32"): q})
    assert bench.step_traffic("ellipsoid", "fp32") is None          # another storage's sources


def test_work_list_launches_per_class():
    """gpu_launches of the tiled and batch steps: per metric kind the interior
    tiles and each non-empty wall-node class (r-layer, x3-layer, the rest)."""
    from oracle.geometry import Channel
    from paper_1411_3133_gb300.workloads import ellipsoid_cross_section, mixed_batch
    assert bench.work_lists([ellipsoid_cross_section(1.0)] * 24) == 4     # four walls: all classes
    assert bench.work_lists(mixed_batch(seed=20241111)) == 6              # cylinders 2 + double-curved 4
    cyl = Channel("cylindrical", 1.0, 1.1, 16, 4, 64)
    assert bench.work_lists([cyl, cyl]) == 2                               # periodic x3: r-layer only
    eq = Channel("ellipsoidal", 1.0, 1.1, 9, 4, 13, b=0.9, periodic3=False, wall="equilibrium")
    assert bench.work_lists([eq]) == 2                                     # every wall node general
    assert bench.work_lists([cyl, eq]) == 4
