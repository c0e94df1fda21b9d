"""Failure detection without a GPU fault: a device-side wait that runs out.

The row kernels wait on their own bulk copies with a clock-bounded wait. In
the plan's test mode every such wait targets a barrier that nothing completes
(a flag nothing sets), with a limit of 100,000 cycles (about 50 us): each
block latches SAG_ETIMEOUT, lets its real copies in flight land and ends. The
test reads the status on the host, checks that it is cleared once read,
restores the limit and checks that the next evaluation (and an RK2
integration) is correct, i.e. that the context stayed usable.
"""
import numpy as np
import pytest

import oracle
from paper_1905_09071_gb300 import sag, workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {sag.SAG_FP32_SPLIT: 1e-10, sag.SAG_FP32_SPLIT_EXACT: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("prec", [sag.SAG_FP32_SPLIT, sag.SAG_FP32_SPLIT_EXACT])
def test_wait_timeout_latches_status_and_context_stays_usable(prec):
    # D = 3, N = 4096: both orders take the pair-form row kernel (bulk copies
    # of 128-point rows behind an mbarrier)
    s = wl.random_cp(3, 4096, [2, 3], seed=71)
    p_ref, q_ref = oracle.rhs(s.n0, s.D, s.ranks, s.factors, mode=oracle.DIRECT)
    scale = np.abs(p_ref).max() + np.abs(q_ref).max()
    n1_ref, _ = oracle.integrate(s.n0, s.D, s.ranks, s.factors, 0.01, 2, diag=False)
    with sag.Plan(s.N, s.D, s.ranks, s.factors, prec=prec) as pl:
        assert pl.describe()["orders"][0]["pairs"] == 1
        n = dev(s.n0)
        out = torch.empty_like(n)
        pl.set_wait_limit(100000, unmet=True)
        pl.rhs(n, out)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_ETIMEOUT
        assert pl.sync_status() == sag.SAG_OK  # reading clears it
        x = dev(s.n0)
        pl.integrate(x, 0.01, 2)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_ETIMEOUT
        pl.set_wait_limit(0)  # back to the default
        pl.rhs(n, out)
        x = dev(s.n0)
        pl.integrate(x, 0.01, 2)
        torch.cuda.synchronize()
        assert pl.sync_status() == sag.SAG_OK
    assert np.max(np.abs(out.cpu().numpy() - (p_ref + q_ref))) / scale < TOL[prec]
    assert np.max(np.abs(x.cpu().numpy() - n1_ref)) / np.max(np.abs(n1_ref)) < TOL[prec]
