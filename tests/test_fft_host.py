"""Host-side check of the library's FFT building blocks (no GPU).

The radix-2/3/4/5/8 butterflies, the Stockham pass indexing and the
double-word arithmetic of ``csrc/`` are compiled for the CPU and compared
with a long-double direct DFT: FP64 must reach ~1e-16 and double-word FP32
~1e-14 relative in max-norm at every length the library uses. The same holds
for the compile-time schedule run through its padded shared-memory index maps
(every load lands on a written slot, every store inside its transform).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_09071_gb300", "csrc")
SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host", "fft_check.cpp")
SIZES = [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 3, 6, 12, 96, 384, 1536, 3072,
         5, 10, 40, 320, 15, 60, 120, 1920]


def _cuda_include():
    for cand in ("/usr/local/cuda/include",):
        if os.path.exists(os.path.join(cand, "cuda_runtime.h")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def fft_check(tmp_path_factory):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC, "-I" + inc,
                    SRC, "-o", exe], check=True)
    return exe


def test_stockham_passes_match_direct_dft(fft_check):
    out = subprocess.run([fft_check] + [str(s) for s in SIZES], check=True, capture_output=True,
                         text=True).stdout.split("\n")
    rows = [ln.split() for ln in out if ln.strip()]
    assert len(rows) == len(SIZES)
    for P, e64, edw in rows:
        assert float(e64) < 1e-15, f"FP64 length {P}: {e64}"
        # radix 3 and 5 in double-word arithmetic, radix 2/4/8 grid-aligned
        assert float(edw) < 1e-12, f"double-word length {P}: {edw}"


CT_SIZES = [64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536]


def test_compile_time_passes_padded_layout(fft_check):
    out = subprocess.run([fft_check, "ct"] + [str(s) for s in CT_SIZES], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    rows = [ln.split() for ln in out if ln.startswith("ct ")]
    # the same passes in FP64 (the plain small DFTs, radix 6 included)
    rows64 = [ln.split() for ln in out if ln.startswith("ct64 ")]
    assert len(rows64) == len(CT_SIZES)
    for _, P, count, sin, err in rows64:
        assert float(err) < 1e-15, f"FP64 length {P}: {err}"
    # column layout for every length, row-chunk and inverse layouts for powers of two
    assert len(rows) == len(CT_SIZES) + 2 * 4
    # Double-word radix-2/4/8 butterflies of the compile-time passes round
    # their high words to a per-butterfly grid (low words at about 2^-43 of
    # the butterfly's largest input, against 2^-47 of each value for plain
    # double-word operations): about 2e-13 here, against 5e-15 before.
    for _, P, count, sin, err in rows:
        assert float(err) < 1e-12, f"length {P}, {count} transforms, natural input {sin}: {err}"
