"""Batched instances of uneven size in one launch (the batched 2D Poisson
family: per instance seeded S in [8, 24]^2 subdomains, K in [100, 400]
features, sources from four separable sine modes), here with few points per
subdomain edge so that the test runs in seconds.

* The QR clusters visit the blocks largest first (RFM_OPT_QR_ORDER): the
  kept sets, pivot orders and the LSQR iterate are bitwise the same as in
  block order (every block is factored by one cluster, whatever its place).
* Every instance of the batch gives what it gives alone (instances share
  launches, not arithmetic): FP64 path, 1e-12 relative.
"""
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


def _batch(n, p_range=(3, 5)):
    probs = [synth.batched_instance(i, p_range=p_range) for i in range(n)]
    prm = np.concatenate([synth.feature_params(p).ravel() for p in probs])
    return probs, torch.from_numpy(prm).cuda()


def test_batch_is_uneven():
    probs, _ = _batch(6)
    assert len({(p.S[0], p.K) for p in probs}) == 6


@pytest.mark.parametrize("asm,op", [("fp32", "q32"), ("fp64", "q64")])
def test_largest_first_order_gives_the_same_factors(rfm, asm, op):
    from paper_2506_17626_gb300 import _native as N
    probs, d = _batch(6)
    out = {}
    for order in (True, False):
        N.set_qr_order(order)
        try:
            S = rfm.System(probs, asm=asm, op=op, tol=1e-6)
            S.assemble(d)
            rank, perm = S.filter(want_perm=True)
            a, rep = S.solve(atol=0, btol=0, max_iter=40)
            torch.cuda.synchronize()
            out[order] = (rank.cpu(), perm.cpu(), a.cpu(), S.r11().cpu())
        finally:
            N.set_qr_order(True)
    for x, y in zip(out[True], out[False]):
        assert torch.equal(x, y)


def test_instances_of_a_batch_match_single_runs(rfm):
    probs, d = _batch(4)
    S = rfm.System(probs, asm="fp64", op="q64", tol=1e-8)
    S.assemble(d)
    S.filter()
    a, _ = S.solve(atol=0, btol=0, max_iter=30)
    a = a.cpu().numpy()
    off_c = off_p = 0
    for p in probs:
        n_prm = p.J * p.K * (p.dim + 1)
        S1 = rfm.System([p], asm="fp64", op="q64", tol=1e-8)
        S1.assemble(d[off_p:off_p + n_prm].contiguous())
        S1.filter()
        a1, _ = S1.solve(atol=0, btol=0, max_iter=30)
        a1 = a1.cpu().numpy()
        seg = a[off_c:off_c + p.J * p.K]
        assert np.linalg.norm(seg - a1) <= 1e-12 * np.linalg.norm(a1)
        off_c += p.J * p.K
        off_p += n_prm
