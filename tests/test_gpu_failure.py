"""Failure detection without a GPU fault.  The LSQR kernel's device-side
waits are bounded (timeout_ms); the RFM_OPT_LSQR_STALL test hook makes them
run out -- a grid barrier that no arrival releases, or forward tiles waiting
for a chunk of their block that never finishes -- and the test checks that
the kernel leaves with RFM_ETIMEOUT in the report, in about timeout_ms, and
that the context stays usable: the next solve is bitwise the one before."""
import time

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


@pytest.mark.parametrize("op", ["q32", "q64"])
def test_bounded_waits_time_out_and_leave_the_context_usable(rfm, op):
    from paper_2506_17626_gb300 import _native as N
    p = synth.poisson2d(S=4, K=48, n=40, delta=1.6)
    d = torch.from_numpy(synth.feature_params(p).ravel()).cuda()
    S = rfm.System([p], asm="fp32" if op == "q32" else "fp64", op=op, tol=1e-6)
    S.assemble(d)
    S.filter()
    a_ref, rep = S.solve(atol=0, btol=0, max_iter=20)
    torch.cuda.synchronize()
    assert rfm.report_dict(rep)["status"] == 0
    for mode in (1, 2):
        N.set_lsqr_stall(mode)
        try:
            t0 = time.time()
            a, rep = S.solve(atol=0, btol=0, max_iter=20, timeout_ms=100)
            torch.cuda.synchronize()
            dt = time.time() - t0
        finally:
            N.set_lsqr_stall(0)
        assert rfm.report_dict(rep)["status"] == N.RFM_ETIMEOUT, mode
        assert dt < 30.0, mode
    a2, rep = S.solve(atol=0, btol=0, max_iter=20)
    torch.cuda.synchronize()
    assert rfm.report_dict(rep)["status"] == 0
    assert torch.equal(a2, a_ref)
