"""The secondary CPU baseline of bench.py (the low-rank method with a library
FP64 FFT) computes the same right-hand side as the oracle. CPU only."""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import workloads as wl

bench = pytest.importorskip("bench")
pytest.importorskip("scipy")


@pytest.mark.parametrize("D,N,ranks,seed", [(2, 50, [3], 1), (3, 97, [2, 3], 2), (4, 200, [2, 0, 3], 3)])
def test_fft_method_matches_oracle(D, N, ranks, seed):
    s = wl.random_cp(D, N, ranks, seed=seed)
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
    got = bench.fft_method_rhs(s, s.n0, workers=1)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    assert np.max(np.abs(got - (p_ref + q_ref))) / scale < 1e-13
