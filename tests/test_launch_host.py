"""Host-side check of the launch splitter that issues one kernel
specialisation per run of equal kind (``csrc/launch.h``): merging of adjacent
entries, cut ranges, empty entries, the fallback to the dispatching kernel
beyond kMaxKindRuns runs, the kind order of mixed tables, and the compile-time
length maps. No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_09071_gb300", "csrc")
SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host", "launch_check.cpp")


def _cuda_include():
    nvcc = shutil.which("nvcc")
    for cand in ["/usr/local/cuda/include"] + ([os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")]
                                               if nvcc else []):
        if os.path.exists(os.path.join(cand, "cuda_runtime.h")):
            return cand
    return None


def test_kind_runs(tmp_path):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "launch_check")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I" + CSRC, "-I" + inc, SRC, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
