"""sag_loss_noalloc: the loss term computed without any device allocation.

Some callers cannot let a library call cudaMalloc: code that runs under a
memory allocator it does not own (a framework's caching pool), inside a fixed
device-memory budget, or in a process that reserved all of its device memory up
front. For them the library offers sag_loss_noalloc, which keeps its partial
sums and loss weights in a static device array instead of a plan workspace.
This file checks, through the C ABI, that two consecutive calls give the CPU
oracle's loss term and the plan-based entry point's (sag_rhs_parts), that the
calls leave the device's free memory unchanged, and that oversized or
host-memory inputs are refused with a message. It is named to be collected
last.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    ("D4_N20000", lambda: wl.random_cp(4, 20000, [5, 4, 3], seed=1905)),  # ragged N, three size chunks
    ("D4_no_d3", lambda: wl.random_cp(4, 9000, [3, 0, 2], seed=1906)),     # a CP rank of 0: order left out
]


@pytest.mark.parametrize("sym", [1, 0])
@pytest.mark.parametrize("name,make", CASES)
def test_noalloc_loss_matches_oracle_and_plan_twice(name, make, sym):
    s = make()
    q_oracle = oracle.loss(s.n0, s.D, s.ranks, s.factors, sym=sym)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=sag.SAG_FP64, symmetrize_q=sym) as pl:
        n = torch.tensor(s.n0, device="cuda")
        q_plan = torch.empty_like(n)
        pl.rhs_parts(n, q=q_plan)
        torch.cuda.synchronize()
        q_plan = q_plan.cpu().numpy()
    f_dev = torch.tensor(s.factors, device="cuda")
    scale = np.abs(q_oracle).max()
    for _ in range(2):  # the static scratch is shared and reused by every call
        q = torch.full_like(n, float("nan"))
        sag.loss_noalloc(s.N, s.D, s.ranks, f_dev, n, q, symmetrize_q=sym)
        torch.cuda.synchronize()
        got = q.cpu().numpy()
        assert np.max(np.abs(got - q_oracle)) / scale < 1e-12
        assert np.max(np.abs(got - q_plan)) / scale < 1e-12


def test_noalloc_calls_allocate_no_device_memory():
    s = wl.random_cp(3, 30000, [4, 6], seed=1907)
    n = torch.tensor(s.n0, device="cuda")
    q = torch.empty_like(n)
    f_dev = torch.tensor(s.factors, device="cuda")
    sag.loss_noalloc(s.N, s.D, s.ranks, f_dev, n, q)  # first call: loads the kernels, finds the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for sym in (1, 0, 1, 0):
        sag.loss_noalloc(s.N, s.D, s.ranks, f_dev, n, q, symmetrize_q=sym)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == torch_bytes0


def test_noalloc_rejects_what_does_not_fit():
    # Sizes are checked before any buffer is touched, so small stand-in tensors
    # suffice for the oversized cases.
    tiny = torch.zeros(8, dtype=torch.float64, device="cuda")
    for N, D, ranks in ((64, 2, [1100]),          # sum_d d R_d = 2200 > 2048
                        (200000, 2, [1000])):     # 2000 vectors x 25 chunks > 32768
        with pytest.raises(sag.SagError) as ei:
            sag.loss_noalloc(N, D, ranks, tiny, tiny, tiny)
        assert ei.value.status == sag.SAG_EINVAL and "too large" in str(ei.value)
    with pytest.raises(sag.SagError) as ei:  # every order left out
        sag.loss_noalloc(8, 3, [0, 0], tiny, tiny, tiny)
    assert ei.value.status == sag.SAG_EINVAL
    # factors in host memory are refused too
    import ctypes
    s = wl.random_cp(3, 100, [2, 2], seed=3)
    n = torch.tensor(s.n0, device="cuda")
    q = torch.empty_like(n)
    r = np.asarray(s.ranks, dtype=np.int32)
    sysd = sag._System(s.N, s.D, sag.SAG_CP, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       s.factors.ctypes.data, 1)
    st = sag.load().sag_loss_noalloc(ctypes.byref(sysd), 1, n.data_ptr(), q.data_ptr(), None)
    assert st == sag.SAG_EINVAL
