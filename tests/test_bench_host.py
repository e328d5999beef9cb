"""Host-side logic of bench.py (no GPU): clock-sample parsing, the kernel
source hash that gates the committed DRAM traffic, and reading the traffic."""
import os
import shutil

import bench


def test_clock_summary_median_max_and_reasons(tmp_path):
    p = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not p.exists()  # the sample file is removed after reading


def test_clock_summary_flags_a_thermal_slowdown(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text("0, 1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown"]
    cs.path = str(tmp_path / "missing.csv")
    assert cs.summary()["sm_mhz"] is None


def _copy_sources(dst):
    src = os.path.join(bench.ROOT, "paper_1405_2728_gb300", "csrc")
    out = dst / "paper_1405_2728_gb300" / "csrc"
    out.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, name), out / name)
    return out


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    ref = bench.kernel_source_hash()
    out = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_hash() == ref
    f = out / "field_kernels.cuh"
    text = f.read_text()
    f.write_text("/* a new block\n   comment */\n" + text.replace("\n", "  // trailing note\n", 3) + "\n\n")
    assert bench.kernel_source_hash() == ref
    f.write_text(text.replace("__syncthreads();", "__syncwarp();", 1))
    assert bench.kernel_source_hash() != ref


def test_traffic_is_read_only_for_the_kernels_it_was_measured_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "ncu_film_8x8x1_fp32.md"
    prof.write_text("Kernel source hash: `0123456789abcdef`\n\n"
                    "    traffic_bytes_per_launch xfwd_step 1000\n"
                    "    traffic_bytes_per_launch xinv_local_bb 3000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    assert bench.load_traffic("xinv_local_bb", "film_8x8x1", "fp32") == 3000
    assert bench.load_traffic("yz_conv", "film_8x8x1", "fp32") is None
    assert bench.load_traffic("xinv_local_bb", "film_8x8x1", "fp64") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.load_traffic("xinv_local_bb", "film_8x8x1", "fp32") is None
