"""The benchmark's workload at full size (2D Poisson, 20 x 20 subdomains, 300
features, 360^2 interior + 1440 boundary rows), in the configuration the
benchmark times, against the oracle on sampled outputs and on properties
that hold at any size:

  * assembly of six sampled blocks (corners, edges, interior) element by
    element: FP32 within 3e-5 and FP64 within 1e-12 of the block's largest
    entry;
  * the kept columns of those blocks: exactly the oracle's QR with column
    pivoting of the same (FP32-rounded, for the mixed path) block, |R_11|
    to 1e-12, and the explicit Q_hat within the rounding bound of its
    storage precision;
  * LSQR after 50 iterations: its residual estimate against the residual of
    the downloaded operator recomputed on the host in FP64;
  * the ansatz at 404 sampled test points against the oracle's evaluation of
    the same coefficients.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

SAMPLED = [0, 19, 200, 210, 380, 399]


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


@pytest.mark.parametrize("asm,op", [("fp32", "q32"), ("fp64", "q64")])
def test_full_size_workload_against_oracle(rfm, asm, op):
    p = synth.poisson2d()
    assert p.J == 400 and p.K == 300
    prm = synth.feature_params(p)
    d = torch.from_numpy(prm.ravel()).cuda()
    S = rfm.System([p], asm=asm, op=op, tol=1e-6)
    S.assemble(d)
    rank, perm = S.filter(want_perm=True)
    a, rep, y = S.solve(atol=0, btol=0, max_iter=50, want_y=True)
    torch.cuda.synchronize()
    rank = rank.cpu().numpy()
    perm = perm.cpu().numpy()
    r11 = S.r11().cpu().numpy()
    eps = np.finfo(float).eps

    tol_asm = 3e-5 if asm == "fp32" else 1e-12
    for j in SAMPLED:
        Bo = oracle.assemble(p, prm, blocks=[j])
        assert np.array_equal(S.block_rows(j).cpu().numpy(), Bo.grow[0])
        Mg = S.block_matrix(j).double().cpu().numpy()
        scale = np.abs(Bo.M[0]).max()
        assert np.abs(Mg - Bo.M[0]).max() <= tol_asm * scale, j
        # the oracle's QRCP of the block the GPU factored (FP32-rounded for the mixed path)
        f = oracle.qrcp(np.asfortranarray(Mg), 1e-6)
        kept = perm[j * p.K: (j + 1) * p.K]
        assert f.rank == rank[j], j
        assert set(f.perm[: f.rank]) == set(kept[: f.rank]), j
        assert r11[j] == pytest.approx(f.r11, rel=1e-12)
        if list(f.perm[: f.rank]) == list(kept[: f.rank]):
            Qg = S.block_matrix(j, which=5)[:, : f.rank].double().cpu().numpy()
            bound = (0.0 if op == "q64" else 2e-7) + 100 * eps * f.r11 / np.abs(np.diag(f.R))
            assert np.all(np.abs(Qg - f.Q()).max(axis=0) <= bound), j

    # LSQR: residual estimate against the residual of the operator it applied
    from paper_2506_17626_gb300 import report_dict
    r = report_dict(rep)
    h = S.rhs().cpu().numpy()
    yv = y.cpu().numpy()
    Ay = np.zeros_like(h)
    for j in range(p.J):
        rj = int(rank[j])
        if rj == 0:
            continue
        Q = S.block_matrix(j, which=5)[:, :rj].double().cpu().numpy()
        rows = S.block_rows(j).cpu().numpy()
        np.add.at(Ay, rows, Q @ yv[j * p.K: j * p.K + rj])
    res = np.linalg.norm(h - Ay)
    assert r["itn"] == 50 and r["status"] == 0
    assert abs(r["rnorm"] - res) <= (1e-6 if op == "q64" else 1e-3) * res, (r["rnorm"], res)
    assert res < np.linalg.norm(h)

    # the ansatz at sampled test points
    Xt = oracle.test_grid(p)[::397]     # stride coprime with the 400-point raster
    u, _ = S.evaluate(d, a, [torch.from_numpy(Xt).cuda()], with_error=False)
    uo = oracle.evaluate(p, prm, a.cpu().numpy(), Xt)
    # each point sums at most a few subdomains' K terms |a_k omega phi_k| <= |a|_max
    an = a.cpu().numpy()
    assert np.abs(u[0].cpu().numpy() - uo).max() <= 1e-12 * max(1.0, np.abs(uo).max(), np.abs(an).max())
