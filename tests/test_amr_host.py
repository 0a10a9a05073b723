"""Host logic of the AMR glue without a GPU: tests/native/amr_maps_check.cu
includes the library source, runs the map builder on random patch layouts
against a brute-force search, and checks that bad geometry is rejected."""
import os
import shutil
import subprocess

import pytest

from paper_1605_05320_gb300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which(B._nvcc()) is None and not os.path.exists(B._nvcc()),
                    reason="nvcc not available")
def test_amr_maps_match_a_brute_force_search(tmp_path):
    lib = B.build()
    exe = str(tmp_path / "amr_maps_check")
    cmd = [B._nvcc()] + B.ARCH + ["-O1", "-std=c++17", f"-I{B.INCLUDE}", f"-I{B.CSRC}",
                                  os.path.join(HERE, "native", "amr_maps_check.cu"), "-o", exe,
                                  f"-L{os.path.dirname(lib)}", "-lswadj",
                                  f"-Xlinker=-rpath={os.path.dirname(lib)}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
