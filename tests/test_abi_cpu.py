"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every entry point include/gpdem.h and include/gpserve.h
declare, and the ctypes structures match the C layouts."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "gpdem.h"), os.path.join(ROOT, "include", "gpserve.h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(gp_[a-z_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2604_16613_gb300 import build, native
    build.build()
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_16613_gb300 import native
    names = declared_functions()
    assert len(names) >= 10
    assert set(names) == set(native.EXPORTED)
    for n in names:
        assert hasattr(lib, n), f"{n} missing from libgpdem.so"


def test_struct_layouts_match_header(tmp_path):
    from paper_2604_16613_gb300 import native
    src = tmp_path / "sz.c"
    src.write_text('#include "gpdem.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gp_bounds), sizeof(gp_circuit),'
                   ' sizeof(gp_dem_view), sizeof(gp_tuning), offsetof(gp_dem_view, det_offsets),'
                   ' offsetof(gp_bounds, max_det_entries));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(native.GpBounds), ctypes.sizeof(native.GpCircuit), ctypes.sizeof(native.GpDemView),
            ctypes.sizeof(native.GpTuning), native.GpDemView.det_offsets.offset,
            native.GpBounds.max_det_entries.offset]
    assert got == want


def test_server_struct_layouts_match_header(tmp_path):
    from paper_2604_16613_gb300 import native
    src = tmp_path / "sz2.c"
    src.write_text('#include "gpserve.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(gp_server_config),'
                   ' sizeof(gp_patch_spec), sizeof(gp_sealed_view), offsetof(gp_sealed_view, det_offsets),'
                   ' offsetof(gp_sealed_view, t_arrival_ns), offsetof(gp_patch_spec, logical_qubits));return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(native.GpServerConfig), ctypes.sizeof(native.GpPatchSpec),
            ctypes.sizeof(native.GpSealedView), native.GpSealedView.det_offsets.offset,
            native.GpSealedView.t_arrival_ns.offset, native.GpPatchSpec.logical_qubits.offset]
    assert got == want


def test_workspace_size_and_bound_validation(lib):
    from paper_2604_16613_gb300 import native
    from paper_2604_16613_gb300.dem import Bounds
    b = Bounds(max_circuits=1, max_qubits=17, max_ops=4096, max_recs=1024, max_layers=64,
               max_measurements=256, max_detectors=64, max_locations=4096, max_mechanisms=8192).to_c()
    size = ctypes.c_uint64()
    assert lib.gp_workspace_size(ctypes.byref(b), ctypes.byref(size)) == native.GP_OK
    assert size.value > 0 and size.value % 256 == 0
    bad = Bounds(max_qubits=100000).to_c()
    assert lib.gp_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == native.GP_ERR_INVALID
    assert b"8192" in lib.gp_last_error()


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2604_16613_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.h" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_2604_16613_gb300 import native
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        native._lib_backup = native._lib
        try:
            native._lib = None
            native.load(str(tmp_path / "absent.so"))
        finally:
            native._lib = native._lib_backup



def test_bench_reads_profile_traffic(tmp_path, monkeypatch):
    """bench.py takes roofline.traffic from a committed profile summary only
    when the summary's source hash matches the current kernel sources."""
    import bench
    current = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "demo_kernel_case.md").write_text(
        f"# x\n\n- dram_bytes_per_launch: 1234\n- source_hash: {current}\n")
    (prof / "stale_kernel_case.md").write_text("- dram_bytes_per_launch: 99\n- source_hash: 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: current)
    assert bench.measured_traffic("demo_kernel") == 1234.0
    assert bench.measured_traffic("stale_kernel") is None
    assert bench.measured_traffic("absent_kernel") is None
