"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/swadj.h declares; host-only logic (workspace sizing, descriptor
checks) works without a GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1605_05320_gb300 import build as B
from paper_1605_05320_gb300 import swadj as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "swadj.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(swa_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(S.EXPORTS) == decl


def test_library_targets_sm_103a():
    B.build()
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.NVCC_FLAGS)
    assert os.path.exists(B.LIB)


def test_workspace_sizes_and_descriptor_checks(lib):
    d = S.make_desc(2, 2048, 2048, 0.0, 0.0, 1000.0, 1000.0, precision=S.SWA_FP32)
    n = 2048 * 2048
    ws = S.swa_grid_workspace_bytes(d)
    # 2 x 3 state arrays + hbar (float) + FP64 staging + clock + partials
    assert 7 * 4 * n + 8 * n <= ws <= 7 * 4 * n + 8 * n + 1 << 20
    d64 = S.make_desc(2, 2048, 2048, 0.0, 0.0, 1000.0, 1000.0, precision=S.SWA_FP64)
    assert S.swa_grid_workspace_bytes(d64) >= 7 * 8 * n + 8 * n
    a = S.swa_adjoint_workspace_bytes(d)
    assert a >= 7 * 4 * n + 8 * n
    s = S.swa_snapstore_workspace_bytes(d, 101, S.SWA_FP32)
    # snapshots, tau, wet mask and the envelope (13 groups of 8, 3 x n/4 floats)
    assert s >= 101 * 3 * 4 * n + 101 * 8 + n + 13 * 3 * (n // 4) * 4
    s64 = S.swa_snapstore_workspace_bytes(d, 101, S.SWA_FP64)
    assert 101 * 3 * 8 * n + n <= s64 < 101 * 3 * 8 * n + n + 4096
    bad = S.make_desc(2, 2048, 2048, 0.0, 0.0, 1000.0, 1000.0, order=3)
    assert S.swa_grid_workspace_bytes(bad) == 0
    assert "order" in S.swa_last_error()
    bad1d = S.make_desc(1, 100, 2, 0.0, 0.0, 1.0, 1.0)
    assert S.swa_grid_workspace_bytes(bad1d) == 0
    assert "ny" in S.swa_last_error()


def test_create_rejects_small_or_misaligned_workspace(lib):
    import numpy as np
    d = S.make_desc(2, 64, 64, 0.0, 0.0, 1000.0, 1000.0)
    B0 = np.full(64 * 64, -100.0)
    need = S.swa_grid_workspace_bytes(d)
    out = ctypes.c_void_p()
    rc = lib.swa_create_grid(ctypes.byref(d), B0.ctypes.data, ctypes.c_void_p(256),
                             need - 1, None, ctypes.byref(out))
    assert rc == S.SWA_ENOMEM
    rc = lib.swa_create_grid(ctypes.byref(d), B0.ctypes.data, ctypes.c_void_p(257),
                             need, None, ctypes.byref(out))
    assert rc == S.SWA_EINVAL and "aligned" in S.swa_last_error()


def test_product_path_does_not_touch_oracle():
    """The library and its binding never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_1605_05320_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "swe_oracle" not in txt and "liboracle" not in txt, f


def test_launch_shape_and_gauge_calls_check_their_arguments(lib):
    """Argument checks that need no GPU: null handles and strip heights the
    kernels do not offer are rejected before anything is enqueued."""
    assert lib.swa_grid_set_strip_rows(None, 32) == S.SWA_EINVAL
    assert lib.swa_grid_set_scheme(None, S.SWA_SCHEME_CTU) == S.SWA_EINVAL
    assert lib.swa_amr_workspace_bytes(None, None, 1, 2) == 0
    out = ctypes.c_void_p()
    assert lib.swa_create_amr(None, None, 1, 2, None, 0, None, ctypes.byref(out)) == S.SWA_EINVAL
    assert lib.swa_amr_step(None, 0.0, 1.0, 1, None) == S.SWA_EINVAL
    assert lib.swa_patches_set_tile_rows(None, 1, 32) == S.SWA_EINVAL
    assert lib.swa_grid_record_gauges(None, 2, None, None, None, 10, None) == S.SWA_EINVAL
    rows = ctypes.c_longlong()
    assert lib.swa_grid_gauge_rows(None, ctypes.byref(rows), None) == S.SWA_EINVAL
    # the static step's scratch holds a 2048^2 FP64 step (64 x 512 tiles of
    # 32 x 4 cells, one reduction slot each)
    hdr = open(os.path.join(ROOT, "include", "swadj.h")).read()
    assert int(re.search(r"#define SWA_STATIC_MAX_BLOCKS (\d+)", hdr).group(1)) >= 64 * 512


def test_bench_arms_report_the_same_workload():
    """Both arms of bench.py name the same workload config."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a, b = bench.workload_config(2048, 1), bench.workload_config(2048, 1)
    assert a == b and a["cells"] == 2048 * 2048
    assert "flag pass every 10" in a["workload"]
    assert bench.whole_job_rate(100.0, 4, 2, 1000.0) == 800.0


def test_clock_summary_of_nvidia_smi_samples():
    """The bench's clock record: median SM clock, maximum, and the throttle
    reasons that were active in any sample (a run with hw_slowdown or a
    thermal slowdown is rejected; sw_power_cap is kept and noted)."""
    import bench
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.summarize_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    hot = lines[:1] + ["0, 1500, 2070, 800.0, 0x8, Active, Not Active, Active, Not Active"]
    assert bench.summarize_clocks(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarize_clocks([]) is None
