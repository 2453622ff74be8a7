"""The benchmark's workloads at full size, in the configuration the benchmark
times, against the oracle on sampled outputs and on properties that hold at
any size:

  2D Poisson, 20 x 20 subdomains, 300 features, 360^2 interior + 1440
  boundary rows (blocks of up to 576 x 300: the cluster QR kernels);
  (2+1)D heat, 10 x 10 x 10 space-time subdomains, 500 features, 100^3
  interior + 50,000 boundary and initial rows (blocks of up to 2744 x 500:
  the global-memory QR kernel, FP64 arithmetic on both paths).

  * assembly of six sampled blocks (corners, edges, interior) element by
    element: FP32 within 3e-5 and FP64 within 1e-12 of the block's largest
    entry;
  * the kept columns of those blocks: a valid greedy pivot order with the
    threshold stop on the same (FP32-rounded, for the mixed path) block, the
    oracle's kept set on the FP64 path, |R_11| to 1e-12, and R and Q_hat
    against the Householder QR of the kept columns in the GPU's order, within
    the rounding bound of the arithmetic (FP64, or double-float for the
    mixed path's cluster kernel) and the storage precision;
  * LSQR after 50 iterations: its residual estimate against the residual of
    the downloaded operator recomputed on the host in FP64;
  * the ansatz at sampled test points against the oracle's evaluation of
    the same coefficients.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from qr_checks import check_pivoted_qr, signs

pytestmark = pytest.mark.gpu

WORKLOADS = {
    # workload, sampled blocks (corners, edges, interior), QR arithmetic of the mixed path
    "p2d": (synth.poisson2d, [0, 19, 200, 210, 380, 399], "df"),
    "heat": (synth.heat3d, [0, 9, 99, 555, 909, 999], "fp64"),
}


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("asm,op", [("fp32", "q32"), ("fp64", "q64")])
def test_full_size_workload_against_oracle(rfm, name, asm, op):
    make, SAMPLED, qr_mixed = WORKLOADS[name]
    p = make()
    assert (p.J, p.K) in ((400, 300), (1000, 500))
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
        # the block the GPU factored (FP32-rounded for the mixed path, whose
        # QR runs in double-float arithmetic: unit roundoff 2^-48)
        Mf = np.asfortranarray(Mg)
        kept = perm[j * p.K: (j + 1) * p.K]
        rk = rank[j]
        f = oracle.qrcp(Mf, 1e-6)
        # |R_11| is the first pivot's norm (the oracle's, unless a near-tie
        # of two column norms sent the GPU to the other one)
        assert r11[j] == pytest.approx(np.linalg.norm(Mf[:, kept[0]]), rel=1e-12)
        # a valid greedy pivot order with the threshold stop (a column within
        # 4e-12 |R_11| of the threshold may fall on either side) ...
        check_pivoted_qr(Mf, kept, rk, 1e-6, w=4e-6)
        # ... which is the oracle's own wherever no near-tie of two trailing
        # norms lets the orders part (always on the FP64 path's blocks here)
        if op == "q64":
            assert f.rank == rk and set(f.perm[:rk]) == set(kept[:rk]), j
        # R and Q_hat: the Householder QR of the kept columns in the GPU's order
        Qn, Rn = np.linalg.qr(Mf[:, kept[:rk]])
        Rg = np.triu(S.block_matrix(j, which=3).cpu().numpy()[:rk, :rk])
        sg = signs(Rg, Rn)
        assert np.abs(Rg - sg[:, None] * Rn).max() <= 1e-10 * f.r11, j
        Qg = S.block_matrix(j, which=5)[:, :rk].double().cpu().numpy()
        unit = eps if (op == "q64" or qr_mixed == "fp64") else 2.56 * 2.0 ** -48
        bound = (0.0 if op == "q64" else 2e-7) + 100 * unit * f.r11 / np.abs(np.diag(Rn))
        assert np.all(np.abs(Qg - Qn * sg).max(axis=0) <= bound), j

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
        del Q
    res = np.linalg.norm(h - Ay)
    assert r["itn"] == 50 and r["status"] == 0
    assert abs(r["rnorm"] - res) <= (1e-6 if op == "q64" else 1e-3) * res, (r["rnorm"], res)
    assert res < np.linalg.norm(h)

    # the ansatz at sampled test points
    Xt = oracle.test_grid(p)[::397]     # stride coprime with the 400- and 50-point rasters
    u, _ = S.evaluate(d, a, [torch.from_numpy(Xt).cuda()], with_error=False)
    uo = oracle.evaluate(p, prm, a.cpu().numpy(), Xt)
    # each point sums the K terms |a_k omega phi_k| <= |a|_max of at most 2^dim
    # covering subdomains: rounding within 4 eps per term
    an = a.cpu().numpy()
    n_terms = p.K * 2 ** p.dim
    bound = 4 * eps * n_terms * max(1.0, np.abs(uo).max(), np.abs(an).max())
    assert np.abs(u[0].cpu().numpy() - uo).max() <= bound
