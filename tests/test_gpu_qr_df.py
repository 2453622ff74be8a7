"""The double-float QR kernels (FP32-assembled blocks; the FP32 Q_hat or the
kept-column operator; the cluster kernel and the global-memory one) against
the oracle's QR with column pivoting of the same FP32-rounded blocks, and
against the FP64-arithmetic kernel.

A normalised double-float pair carries about 48 bits (unit roundoff
u = 2^-48), so a backward-stable Householder QR in it determines |R_kk| to
about m u |R_11| and column k of Q_hat to about u |R_11| / |R_kk|, where FP64
has 2^-53.  Tolerances:
  kept columns: a valid greedy pivot order with the threshold stop (a
    column within 4e-12 |R_11| of tol |R_11| may fall on either side), which
    is the oracle's own order wherever no near-tie of two trailing norms
    (within their rounding) lets the orders part;
  R where the pivot orders agree: 1e-10 |R_11| (as for the FP64 kernels);
  Q_hat per column: 2e-7 (FP32 storage) + 256 u |R_11| / |R_kk|.
Row k of R and column k of Q_hat are compared up to a common sign: beta_k
takes the sign opposite to the pivot column's leading entry, which for a
column that is nearly dependent on the earlier ones (|R_kk| near the
threshold) is rounding noise, so two correct factorisations may differ in
it.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from qr_checks import check_pivoted_qr, signs

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -48

CASES = {
    "p1d": lambda: synth.poisson1d(S=6, K=24, n=150),
    "p2d": lambda: synth.poisson2d(S=5, K=40, n=30),
    "heat": lambda: synth.heat3d(S=3, K=30, n=9),
    "p2d_d29": lambda: synth.poisson2d(S=4, K=20, n=17, delta=2.9),
    "p2d_wide": lambda: synth.poisson2d(S=3, K=120, n=36, delta=1.6),
    # fewer rows than features in every block (min(m, K) = m steps)
    "p2d_short": lambda: synth.poisson2d(S=4, K=60, n=16, delta=1.25),
}


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


def _system(rfm, p, prm, op, tol, kernel="cluster"):
    """kernel: "cluster" (the block in a cluster's shared memory) or "global"
    (the global-memory double-float kernel that takes blocks too tall for a
    cluster, forced here on small blocks)."""
    from paper_2506_17626_gb300 import _native as N
    S = rfm.System([p], asm="fp32", op=op, tol=tol)
    d = torch.from_numpy(np.ascontiguousarray(prm).ravel()).cuda()
    S.assemble(d)
    N.set_filter_kernel(kernel == "global")
    try:
        rank, perm = S.filter(want_perm=True)
        torch.cuda.synchronize()
    finally:
        N.set_filter_kernel(False)
    return S, rank.cpu().numpy(), perm.cpu().numpy().reshape(p.J, p.K)


def check_kept(Mg, tol, rank, kept):
    """Kept columns of one block: a valid greedy pivot order with the threshold
    stop; the oracle's kept set whenever the pivot orders agree up to the
    threshold window.  Returns the oracle factorisation at tol."""
    w = 4e-12 / tol
    check_pivoted_qr(Mg, kept, rank, tol, w=w)
    f = oracle.qrcp(Mg, tol)
    strict = oracle.qrcp(Mg, tol * (1 + w))
    loose = oracle.qrcp(Mg, tol * (1 - w))
    if list(kept[: strict.rank]) == list(strict.perm[: strict.rank]):
        assert strict.rank <= rank <= loose.rank, (strict.rank, rank, loose.rank)
        assert set(kept[:rank]) <= set(loose.perm[: loose.rank])
    return f


@pytest.mark.parametrize("kernel", ["cluster", "global"])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tol", [1e-10, 1e-6, 1e-2])
def test_double_float_filter_matches_oracle(rfm, name, tol, kernel):
    p = CASES[name]()
    prm = synth.feature_params(p)
    S, rank, perm = _system(rfm, p, prm, "q32", tol, kernel)
    r11 = S.r11().cpu().numpy()
    for j in range(p.J):
        Mg = np.asfortranarray(S.block_matrix(j).double().cpu().numpy())
        f = check_kept(Mg, tol, rank[j], perm[j])
        assert r11[j] == pytest.approx(np.linalg.norm(Mg[:, perm[j, 0]]), rel=1e-12)
        # whatever the pivot order: R and Q_hat are the Householder QR (no
        # pivoting, same sign convention) of the kept columns in that order
        rk = rank[j]
        if rk:
            Qn, Rn = np.linalg.qr(Mg[:, perm[j, :rk]])
            Rg = np.triu(S.block_matrix(j, which=3).cpu().numpy()[:rk, :rk])
            d = signs(Rg, Rn)
            assert np.abs(Rg - d[:, None] * Rn).max() <= 1e-10 * f.r11, j
            Qg = S.block_matrix(j, which=5)[:, :rk].double().cpu().numpy()
            bound = 2e-7 + 256 * U_DF * f.r11 / np.abs(np.diag(Rn))
            assert np.all(np.abs(Qg - Qn * d).max(axis=0) <= bound), j
        r = min(rank[j], f.rank)
        if r and list(perm[j, :r]) == list(f.perm[:r]):
            Rg = np.triu(S.block_matrix(j, which=3).cpu().numpy()[:r, :r])
            d = signs(Rg, f.R[:r, :r])
            assert np.abs(Rg - d[:, None] * f.R[:r, :r]).max() <= 1e-10 * f.r11, j
            if rank[j] == f.rank:
                Qg = S.block_matrix(j, which=5)[:, :r].double().cpu().numpy()
                bound = 2e-7 + 256 * U_DF * f.r11 / np.abs(np.diag(f.R))
                assert np.all(np.abs(Qg - f.Q() * d).max(axis=0) <= bound), j
                assert np.abs(Qg.T @ Qg - np.eye(r)).max() <= 1e-5


@pytest.mark.parametrize("name", ["p2d", "p2d_wide"])
def test_double_float_and_fp64_kernels_agree(rfm, name):
    """Same FP32 blocks through both kernels: same kept sets (threshold
    1e-6), and LSQR on the two FP32 Q_hat operators agrees to the FP32
    level over 12 iterations."""
    from paper_2506_17626_gb300 import _native as N
    p = CASES[name]()
    prm = synth.feature_params(p)
    res = {}
    for df in (True, False):
        N.set_qr_double_float(df)
        try:
            S, rank, perm = _system(rfm, p, prm, "q32", 1e-6)
            a, rep, y = S.solve(atol=0, btol=0, max_iter=12, want_y=True)
            torch.cuda.synchronize()
            res[df] = (rank, perm, y.cpu().numpy(), rfm.report_dict(rep))
        finally:
            N.set_qr_double_float(True)
    (r0, p0, y0, q0), (r1, p1, y1, q1) = res[True], res[False]
    assert np.array_equal(r0, r1)
    for j in range(p.J):
        assert set(p0[j, : r0[j]]) == set(p1[j, : r1[j]]), j
    assert q0["rnorm"] == pytest.approx(q1["rnorm"], rel=1e-5)
    if all(list(p0[j, : r0[j]]) == list(p1[j, : r1[j]]) for j in range(p.J)):
        assert np.linalg.norm(y0 - y1) <= 1e-5 * np.linalg.norm(y1)
    dropped = np.concatenate([np.arange(j * p.K + r0[j], (j + 1) * p.K) for j in range(p.J)])
    assert np.all(y0[dropped] == 0.0) and np.all(y1[dropped] == 0.0)


def test_double_float_kept_operator(rfm):
    """Kept-column operator (no Q_hat) from the double-float kernel: the
    gathered columns are the oracle's kept columns of the FP32 block."""
    p = CASES["p2d"]()
    prm = synth.feature_params(p)
    S, rank, perm = _system(rfm, p, prm, "ar64", 1e-6)
    for j in range(p.J):
        Mg = np.asfortranarray(S.block_matrix(j).double().cpu().numpy())
        check_kept(Mg, 1e-6, rank[j], perm[j])
        Op = S.block_matrix(j, which=5)[:, : rank[j]].cpu().numpy()
        assert np.array_equal(Op, Mg[:, perm[j, : rank[j]]]), j


@pytest.mark.parametrize("name", ["heat", "p2d_wide", "p2d", "p2d_short"])
@pytest.mark.parametrize("tol", [1e-6, 1e-2])
def test_double_float_panel_widths(rfm, name, tol):
    """The global double-float kernels with panels of 1, 2, 4 and 8 steps:
    the QR with column pivoting defers the trailing update over the panel
    (F = tau A^T v per step, one rank-nb update per panel) and Q_hat is
    formed from compact WY panels.  Every width is checked against the oracle
    as in test_double_float_filter_matches_oracle (a valid greedy pivot order
    with the threshold stop; R and Q_hat of the kept columns in that order);
    where two widths take the same pivot order, R agrees to 1e-10 |R_11| and
    Q_hat to 2e-7 (FP32 storage)."""
    from paper_2506_17626_gb300 import _native as N
    p = CASES[name]()
    prm = synth.feature_params(p)
    res = {}
    for pw in (1, 2, 4, 8):
        N.set_qr_panel(pw)
        try:
            S, rank, perm = _system(rfm, p, prm, "q32", tol, "global")
            r11 = S.r11().cpu().numpy()
            out = []
            for j in range(p.J):
                rk = rank[j]
                Mg = np.asfortranarray(S.block_matrix(j).double().cpu().numpy())
                Rg = np.triu(S.block_matrix(j, which=3).cpu().numpy()[:rk, :rk])
                Qg = S.block_matrix(j, which=5)[:, :rk].double().cpu().numpy()
                f = check_kept(Mg, tol, rk, perm[j])
                assert r11[j] == pytest.approx(np.linalg.norm(Mg[:, perm[j, 0]]), rel=1e-12)
                if rk:
                    Qn, Rn = np.linalg.qr(Mg[:, perm[j, :rk]])
                    d = signs(Rg, Rn)
                    assert np.abs(Rg - d[:, None] * Rn).max() <= 1e-10 * f.r11, (pw, j)
                    bound = 2e-7 + 256 * U_DF * f.r11 / np.abs(np.diag(Rn))
                    assert np.all(np.abs(Qg - Qn * d).max(axis=0) <= bound), (pw, j)
                out.append((list(perm[j, :rk]), Rg, Qg, f.r11))
            res[pw] = out
        finally:
            N.set_qr_panel(8)
    for pw in (2, 4, 8):
        for j in range(p.J):
            k1, R1, Q1, r11 = res[1][j]
            kp, Rp, Qp, _ = res[pw][j]
            if kp == k1 and k1:
                d = signs(Rp, R1)
                assert np.abs(Rp - d[:, None] * R1).max() <= 1e-10 * r11, (pw, j)
                assert np.abs(Qp - Q1 * d).max() <= 2e-7, (pw, j)
