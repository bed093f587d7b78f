"""Host logic of bench.py that needs no GPU: the roofline's DRAM traffic is
read from a committed ncu summary only when that summary was taken on the
current kernel sources."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def write_profile(root, name, dram, src_hash):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", name), "w") as f:
        f.write("# a kernel\n\nsome text: with a colon\n\n")
        f.write(f"- dram_bytes_per_launch: {dram}\n- source_hash: {src_hash}\n")


def test_traffic_only_from_a_summary_of_the_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "00ff00ff00ff00ff")
    write_profile(str(tmp_path), "walk_kernel_case.md", 12345, "00ff00ff00ff00ff")
    assert bench.measured_traffic("walk_kernel") == 12345.0
    # another kernel's summary is not read
    assert bench.measured_traffic("other_kernel") is None
    # a summary of older sources gives no traffic
    write_profile(str(tmp_path), "walk_kernel_case.md", 12345, "1111222233334444")
    assert bench.measured_traffic("walk_kernel") is None


def test_source_hash_covers_the_compile_kernels():
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h)
    assert h == bench.kernel_source_hash()


def test_committed_stage1_summary_is_machine_readable():
    path = os.path.join(ROOT, "profiles", "stage1_split_kernel_surface_d25.md")
    if not os.path.exists(path):
        pytest.skip("no stage-1 summary")
    text = open(path).read()
    dram = re.search(r"^- dram_bytes_per_launch: (\d+)$", text, re.M)
    src = re.search(r"^- source_hash: ([0-9a-f]{16})$", text, re.M)
    assert dram and int(dram.group(1)) > 0
    assert src
