"""CPU-side checks of the product library: it builds, loads, exports every
entry point that include/sar.h declares, and rejects bad arguments before
touching the GPU.  Also the reporting conventions against the paper's tables."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sar(built_lib):
    import paper_2604_03585_gb300 as sar
    return sar


def header_symbols():
    text = open(os.path.join(ROOT, "include", "sar.h")).read()
    return sorted(set(re.findall(r"SAR_API\s+[\w\s\*]+?\b(sar_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ("sar_plan_create", "sar_plan_destroy", "sar_range_compress", "sar_corner_turn",
                 "sar_azimuth_compress", "sar_rda_process"):
        assert name in syms


def test_library_exports_every_declared_symbol(sar):
    lib = sar.library()
    missing = [s for s in header_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(header_symbols()) == set(sar.EXPORTS)


def test_argument_errors_without_gpu(sar):
    lib = sar.library()
    import ctypes
    # NULL out-pointer
    assert lib.sar_plan_create(256, 256, None, None) == sar.SAR_ERR_INVALID_ARG
    f = sar.sar_filters(None, None, 0, 0)
    h = ctypes.c_void_p()
    # unsupported sizes are refused before any device call
    assert lib.sar_plan_create(10000, 256, ctypes.byref(f), ctypes.byref(h)) == sar.SAR_ERR_UNSUPPORTED
    assert lib.sar_plan_create(256, 262144, ctypes.byref(f), ctypes.byref(h)) == sar.SAR_ERR_UNSUPPORTED
    assert lib.sar_plan_create(0, 256, ctypes.byref(f), ctypes.byref(h)) == sar.SAR_ERR_INVALID_ARG
    assert "n_range" in sar.sar_last_error()
    f2 = sar.sar_filters(None, None, 0, 2)
    assert lib.sar_plan_create(256, 256, ctypes.byref(f2), ctypes.byref(h)) == sar.SAR_ERR_INVALID_ARG
    f3 = sar.sar_filters(None, None, 7, 0)          # unknown precision
    assert lib.sar_plan_create(256, 256, ctypes.byref(f3), ctypes.byref(h)) == sar.SAR_ERR_INVALID_ARG
    f4 = sar.sar_filters(None, None, sar.SAR_PREC_FP16X2, 0)   # split precision: 256 / 4096 only
    assert lib.sar_plan_create(1024, 256, ctypes.byref(f4), ctypes.byref(h)) == sar.SAR_ERR_UNSUPPORTED
    assert h.value is None
    assert lib.sar_fft_lines(10000, 1, None, None, 0, None) == sar.SAR_ERR_UNSUPPORTED   # above 8192, not 2^k
    assert lib.sar_fft_lines(100, 1, None, None, 0, None) == sar.SAR_ERR_INVALID_ARG     # any length: bad pointers
    assert lib.sar_fft_lines(256, -1, None, None, 0, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_fft_lines(256, 0, None, None, 0, None) == sar.SAR_OK   # nothing to do
    assert lib.sar_make_lfm_spectrum(256, 0, 1.0, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_make_lfm_spectrum(256, 64, -1.0, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_transpose(0, 4, None, None, None) == sar.SAR_ERR_INVALID_ARG
    for fn in ("sar_range_compress", "sar_azimuth_compress"):
        assert getattr(lib, fn)(None, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_rda_process(None, None, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_rda_process_host(None, None, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_rda_process_host_n(None, 2, None, None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_server_create(None, None) == sar.SAR_ERR_INVALID_ARG
    assert lib.sar_server_destroy(None) == sar.SAR_OK
    assert lib.sar_plan_destroy(None) == sar.SAR_OK
    assert "sm_103a" in sar.sar_version()


def _golden(name):
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_flop_convention_reproduces_table1(sar):
    from paper_2604_03585_gb300 import roofline
    for _, gflops, us in _golden("table1_fft_gflops.txt"):
        assert round(roofline.fft_gflops(4096, float(us) * 1e-6)) == int(gflops)


def test_traffic_convention_reproduces_range_step(sar):
    from paper_2604_03585_gb300 import roofline
    (n_lines, n, total_ms, us_line, gbs, min_ms), = _golden("table3_range_step.txt")
    n_lines, n = int(n_lines), int(n)
    assert abs(float(total_ms) * 1e3 / n_lines - float(us_line)) < 0.05
    t_min = roofline.fused_pass_bytes(n_lines, n) / (float(gbs) * 1e9) * 1e3
    assert abs(t_min - float(min_ms)) < 0.1
    assert roofline.rda_bytes(4096, 4096) == 805306368
    assert roofline.fused_line_flops(4096) == 516096


def test_binding_constants_match_the_header(sar):
    """Every #define of include/sar.h has the same value in the binding."""
    text = open(os.path.join(ROOT, "include", "sar.h")).read()
    defines = dict(re.findall(r"#define\s+(SAR_[A-Z0-9_]+)\s+(\d+)u?\b", text))
    assert defines, "no constants found"
    for name, value in defines.items():
        assert getattr(sar, name) == int(value), name


def test_bench_refuses_unknown_extras(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--extras", "no_such_section"])
    with pytest.raises(SystemExit):
        bench.parse()                      # refused before any GPU work
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    every = set(bench.parse().extras.split(","))
    assert {"passes", "scene_256", "pipelined", "az_major", "unfused", "precision", "rda_full", "long_lines",
            "any_length", "ragged_batch", "serving"} == every


def test_traffic_record_scope_and_hash(tmp_path):
    """The recorded ncu traffic is tied to the sources of the kernels it was
    taken from: the 4096-point schedule table and every csrc header it
    includes, followed through nested includes; a change to one of them
    changes the hash, a change elsewhere does not."""
    from paper_2604_03585_gb300 import roofline
    import os
    csrc = os.path.join(os.path.dirname(roofline.__file__), "csrc")
    seen = set()
    roofline._local_includes(os.path.join(csrc, "sched_4096.cu"), seen)
    names = {os.path.basename(f) for f in seen}
    assert {"sched_4096.cu", "launch.cuh", "streamed.cuh", "line_engine.cuh", "sar_common.cuh"} <= names
    assert "mixed_radix.cuh" not in names and "cluster_line.cu" not in names
    # nested includes on a scratch tree
    (tmp_path / "a.cu").write_text('#include "b.cuh"\n')
    (tmp_path / "b.cuh").write_text('#pragma once\n#include "c.h"\n')
    (tmp_path / "c.h").write_text("int x;\n")
    (tmp_path / "d.h").write_text("int y;\n")
    seen = set()
    roofline._local_includes(str(tmp_path / "a.cu"), seen)
    assert {os.path.basename(f) for f in seen} == {"a.cu", "b.cuh", "c.h"}
    h = roofline.kernel_source_hash()
    assert len(h) == 16 and h == roofline.kernel_source_hash()
    # the hash follows the code, not its comments or layout
    pkg = tmp_path / "pkg"
    (pkg / "csrc").mkdir(parents=True)
    (pkg / "csrc" / "sched_4096.cu").write_text('#include "k.cuh"\nint main_table = 1;\n')
    (pkg / "csrc" / "k.cuh").write_text('// a kernel\nint f(int a) { return a + 1; }  /* note */\nconst char* s = "// kept";\n')
    h0 = roofline.kernel_source_hash(str(pkg))
    (pkg / "csrc" / "k.cuh").write_text('// the kernel, reworded\nint f(int a)   {\n  return a + 1;\n}\nconst char* s = "// kept";\n')
    assert roofline.kernel_source_hash(str(pkg)) == h0
    (pkg / "csrc" / "k.cuh").write_text('// a kernel\nint f(int a) { return a + 2; }\nconst char* s = "// kept";\n')
    assert roofline.kernel_source_hash(str(pkg)) != h0
    (pkg / "csrc" / "k.cuh").write_text('// a kernel\nint f(int a) { return a + 1; }\nconst char* s = "// changed";\n')
    assert roofline.kernel_source_hash(str(pkg)) != h0
