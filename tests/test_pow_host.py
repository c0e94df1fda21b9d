"""Host check of the double-word power of the parametric factors (no GPU).

csrc/dw_pow.cuh generates U(i) = u i^a in double-word FP32 (ln i from a
table, exp by Tang's table-driven method). Compiled for the CPU with the same
rounding (no contraction), it is compared with a long-double u i^a for every
size i <= 2^22: the error bound grows with |a ln i| (the double-word product
a ln i is good to about 2^-47 of itself), about 1e-13 for |a| <= 0.5 and 3e-13
for |a| = 2.5, the largest exponent a plan accepts.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_09071_gb300", "csrc")
SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host", "pow_check.cpp")


@pytest.fixture(scope="module")
def pow_check(tmp_path_factory):
    inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")) or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("pow") / "pow_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, "-I" + inc, SRC, "-o", exe],
                   check=True)
    return exe


def test_power_over_every_size_up_to_2_22(pow_check):
    exps = ["-0.5", "-0.3", "-0.1", "0", "0.3", "0.5", "-2.5", "2.5"]
    out = subprocess.run([pow_check, str(1 << 22), "0.7"] + exps, check=True, capture_output=True,
                         text=True).stdout.split("\n")
    rows = [ln.split() for ln in out if ln.strip()]
    assert len(rows) == len(exps)
    for a, err, _ in rows:
        a, err = float(a), float(err)
        bound = 1.2e-13 if abs(a) <= 0.5 else 4e-13
        assert err < bound, (a, err)
    # a = 0 is the constant u: only the rounding of u to a double-word remains
    assert float(rows[3][1]) < 1e-14
