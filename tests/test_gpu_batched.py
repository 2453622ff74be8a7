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


def test_batch_matches_oracle_per_instance(rfm):
    """Four uneven instances of the batched family (S from 9 to 23 per side,
    K from 127 to 282) in one system, each against the oracle run on it
    alone: assembly of sampled blocks, kept sets of every block (FP64 QR on
    both sides: exact), the LSQR iterate after 20 steps (1e-8 relative, the
    FP64 path's tolerance), and the ansatz of the oracle's coefficients at
    sampled test points (1e-12)."""
    import oracle
    probs = [synth.batched_instance(i, p_range=(3, 5)) for i in (1, 2, 3, 4)]
    prms = [synth.feature_params(p) for p in probs]
    d = torch.from_numpy(np.concatenate([q.ravel() for q in prms])).cuda()
    tol, k = 1e-6, 20
    S = rfm.System(probs, asm="fp64", op="q64", tol=tol)
    S.assemble(d)
    rank, perm = S.filter(want_perm=True)
    a, rep, y = S.solve(atol=0, btol=0, max_iter=k, want_y=True)
    torch.cuda.synchronize()
    rank = rank.cpu().numpy()
    perm = perm.cpu().numpy()
    y = y.cpu().numpy()
    b0 = c0 = 0
    for i, (p, prm) in enumerate(zip(probs, prms)):
        B = oracle.assemble(p, prm)
        for j in (0, p.J // 2, p.J - 1):
            Mg = S.block_matrix(b0 + j).cpu().numpy()
            assert np.abs(Mg - B.M[j]).max() <= 1e-12 * np.abs(B.M[j]).max(), (i, j)
        F = oracle.filter_blocks(B, tol)
        for j, f in enumerate(F):
            assert rank[b0 + j] == f.rank, (i, j)
            pj = perm[c0 + j * p.K: c0 + j * p.K + f.rank]
            assert set(pj) == set(f.perm[:f.rank]), (i, j)
        So = oracle.build_system(B, F, mode=0)
        ref = So.lsqr(B.h, atol=0, btol=0, max_iter=k)
        yg = np.concatenate([y[c0 + j * p.K: c0 + j * p.K + f.rank] for j, f in enumerate(F)])
        assert np.linalg.norm(yg - ref["y"]) <= 1e-8 * np.linalg.norm(ref["y"]), i
        # the residual estimate phibar ~ ||h - A y_k||: a 1e-8 relative change
        # of the recurrence moves it by at most about 1e-8 ||h|| (it ranges from
        # rounding level, on instances whose blocks have fewer rows than
        # features, to 2e-7 ||h||)
        assert abs(rfm.report_dict(rep, i)["rnorm"] - ref["rnorm"]) <= 1e-8 * np.linalg.norm(B.h)
        # the ansatz of the oracle's coefficients, instance by instance in one call
        a_o = So.coefficients(ref["y"])
        X = oracle.test_grid(p, [13, 13])
        uo = oracle.evaluate(p, prm, a_o, X)
        a_all = torch.zeros(S.sizes["n_cols"], dtype=torch.float64, device="cuda")
        a_all[c0:c0 + p.J * p.K] = torch.from_numpy(a_o).cuda()
        Xs = [torch.from_numpy(X if q is p else X[:1]).cuda() for q in probs]
        u, _ = S.evaluate(d, a_all, Xs, with_error=False)
        un = u[i].cpu().numpy()
        assert np.abs(un - uo).max() <= 1e-12 * max(1.0, np.abs(uo).max(), np.abs(a_o).max())
        b0 += p.J
        c0 += p.J * p.K
