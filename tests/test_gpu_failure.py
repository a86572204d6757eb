"""Failure detection on the GPU without a fault: a bounded wait that gives up.

The streaming kernels wait on shared-memory barriers that their producer's
bulk copies complete.  If the copies never arrived, each wait would give up
after its poll limit, record the timeout in the device error word and
return; a solve then reports AMG_ERR_CUDA.  amg_check_wait_limit runs one
block of that pipeline on a barrier nothing completes (a short poll limit):
the wait must end by itself, the status must come back, and the device must
stay usable."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("_b", os.path.join(root, "paper_1811_05704_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_1811_05704_gb300 as m
    return m


def test_bounded_wait_gives_up_and_reports(amg):
    import torch
    dev = torch.device("cuda:0")
    st, sec = amg.amg_check_wait_limit()
    assert st == amg.AMG_ERR_CUDA
    assert "timed out" in amg.amg_last_error()
    assert 0.0 < sec < 5.0
    # the error word was cleared and the context works: an ordinary solve succeeds
    A = gen.poisson3d(12)
    f, _ = gen.rhs_from_solution(A, 4)
    with amg.Solver(A.n, A.row_ptr, A.col, A.val, coarse_enough=50) as S:
        x = torch.zeros(A.n, dtype=torch.float64, device=dev)
        s2, it, rr = S.solve(torch.from_numpy(f).to(dev), x, rtol=1e-8, maxiter=100)
    assert s2 == 0 and rr <= 1e-8 and np.isfinite(x.cpu().numpy()).all()
    # and the check repeats
    st, sec = amg.amg_check_wait_limit()
    assert st == amg.AMG_ERR_CUDA and 0.0 < sec < 5.0
