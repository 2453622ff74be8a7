"""Mixed precision at convergence, iterative refinement and the warm start's
fallback, on the GPU through the C ABI, against the CPU oracle.

Refinement (rfm_lsqr_solve with refine_steps > 0): after the FP32-operator
solve, correction solves on the residual h - M a of the assembled system in
FP64.  The oracle's reference is its FP64 LSQR (Paige and Saunders 1982) on
the same filtered, preconditioned system run far past convergence; on the 1D
workload the kept columns are fewer than the rows and have full rank, so the
least-squares y is unique and is compared element by element (1e-5
relative for the mixed path).  The oracle assembles its own FP64
blocks from the same parameters.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


def _compact(y, ranks, K):
    y = y.cpu().numpy()
    return np.concatenate([y[j * K: j * K + r] for j, r in enumerate(ranks)])


def _oracle_reference(p, prm, tol, fp32=False):
    B = oracle.assemble(p, prm)
    F = oracle.filter_blocks(B, tol)
    S = oracle.build_system(B, F, mode=0)
    ref = S.lsqr(B.h, atol=1e-15, btol=1e-15, max_iter=60000)
    a = S.coefficients(ref["y"])
    # residual of the assembled system at the solution, in FP64
    res = B.h.copy()
    for j, g in enumerate(B.grow):
        res[g] -= B.M[j] @ a[j * p.K:(j + 1) * p.K]
    return B, F, ref, float(np.linalg.norm(res))


def test_refined_mixed_solution_matches_oracle_at_convergence(rfm):
    """The mixed path on FP64 blocks (double-float QR, FP32 Q_hat operator,
    FP32 products): y within 1e-5 (relative) of the oracle's converged
    y, refinement no worse than one solve, and the FP64 residuals of the
    assembled system non-increasing down to the oracle's."""
    from paper_2506_17626_gb300 import _native as N
    p = synth.poisson1d()
    prm = synth.feature_params(p)
    tol = 1e-6
    B, F, ref, res_ref = _oracle_reference(p, prm, tol, fp32=False)
    ranks_o = np.array([f.rank for f in F])
    assert ranks_o.sum() < B.N     # more rows than kept columns: y is unique
    N.set_qr_double_float(2)       # FP64 blocks factored in double-float too (the mixed path's QR)
    try:
        S = rfm.System([p], asm="fp64", op="q32", tol=tol)
        d = torch.from_numpy(prm.ravel()).cuda()
        S.assemble(d)
        rank, perm = S.filter(want_perm=True)
    finally:
        N.set_qr_double_float(1)
    rank = rank.cpu().numpy()
    perm = perm.cpu().numpy().reshape(p.J, p.K)
    for j, f in enumerate(F):
        assert rank[j] == f.rank and set(perm[j, :f.rank]) == set(f.perm[:f.rank]), j
    R_steps = 3
    rn = torch.zeros(R_steps + 1, dtype=torch.float64, device="cuda")
    _, rep0, y0 = S.solve(atol=0, btol=0, max_iter=4000, want_y=True)
    a, rep, y = S.solve(atol=0, btol=0, max_iter=4000, want_y=True, refine_steps=R_steps, refine_iters=2000,
                        rnorm64=rn)
    r = rfm.report_dict(rep)
    assert r["status"] == 0 and r["itn"] == 4000 + R_steps * 2000
    yr = ref["y"]
    e0 = np.linalg.norm(_compact(y0, rank, p.K) - yr) / np.linalg.norm(yr)
    e1 = np.linalg.norm(_compact(y, rank, p.K) - yr) / np.linalg.norm(yr)
    assert e1 <= 1e-5 and e1 <= 1.5 * e0, (e0, e1)
    rn = rn.cpu().numpy()
    assert np.all(np.diff(rn) <= 1e-12 * rn[0]), rn
    assert abs(rn[-1] - res_ref) <= 1e-6 * res_ref, (rn, res_ref)


def test_refinement_on_fp32_blocks_reduces_the_residual(rfm):
    """FP32 assembly (the blocks' values, not the rounding of the FP64
    values, so the oracle has no copy of this matrix): the FP64 residual of
    the stored system does not grow over the correction solves, and the
    refined solution's residual is no larger than one solve's."""
    p = synth.poisson1d()
    prm = synth.feature_params(p)
    S = rfm.System([p], asm="fp32", op="q32", tol=1e-6)
    S.assemble(torch.from_numpy(prm.ravel()).cuda())
    S.filter()
    rn = torch.zeros(4, dtype=torch.float64, device="cuda")
    a0, _ = S.solve(atol=0, btol=0, max_iter=4000)
    a, rep = S.solve(atol=0, btol=0, max_iter=4000, refine_steps=3, refine_iters=2000, rnorm64=rn)
    rn = rn.cpu().numpy()
    assert rfm.report_dict(rep)["status"] == 0
    assert np.all(np.diff(rn) <= 1e-12 * rn[0]), rn
    assert float(S.residual(a)[0]) == pytest.approx(rn[-1], rel=1e-12)
    assert float(S.residual(a0)[0]) >= rn[-1] * (1 - 1e-12)


def test_residual_history_without_refinement(rfm):
    """refine_steps = 0 with rnorm64 set: one FP64 residual, equal to the
    oracle's ||h - M a|| at the GPU's coefficients."""
    p = synth.poisson1d(S=6, K=24, n=150)
    prm = synth.feature_params(p)
    S = rfm.System([p], asm="fp64", op="q64", tol=1e-6)
    d = torch.from_numpy(prm.ravel()).cuda()
    S.assemble(d)
    S.filter()
    rn = torch.zeros(1, dtype=torch.float64, device="cuda")
    a, rep = S.solve(atol=0, btol=0, max_iter=40, rnorm64=rn)
    B = oracle.assemble(p, prm)
    an = a.cpu().numpy()
    res = B.h.copy()
    for j, g in enumerate(B.grow):
        res[g] -= B.M[j] @ an[j * p.K:(j + 1) * p.K]
    assert float(rn[0]) == pytest.approx(np.linalg.norm(res), rel=1e-10)
    assert rfm.report_dict(rep)["itn"] == 40


@pytest.mark.parametrize("op", ["q32", "ar64"])
def test_warm_start_fallback_per_instance(rfm, op):
    """Two instances side by side: a start far off (its residual above ||h||)
    is dropped for a zero start, and that instance then runs exactly as a zero
    start; a start at the solution is kept."""
    p = synth.poisson1d(S=6, K=24, n=150)
    prm = synth.feature_params(p)
    asm = "fp32" if op == "q32" else "fp64"
    S = rfm.System([p, p], asm=asm, op=op, tol=1e-6)
    d = torch.from_numpy(np.concatenate([prm.ravel(), prm.ravel()])).cuda()
    S.assemble(d)
    S.filter()
    nc = p.J * p.K
    _, _, ysol = S.solve(atol=1e-12, btol=1e-12, max_iter=3000, want_y=True)
    rng = np.random.default_rng(0)
    y0 = ysol.clone()
    y0[:nc] = torch.from_numpy(1e3 * rng.standard_normal(nc)).cuda()
    a, rep, y = S.solve(atol=0, btol=0, max_iter=30, y0=y0, want_y=True)
    az, repz, yz = S.solve(atol=0, btol=0, max_iter=30, want_y=True)
    r0, r1 = rfm.report_dict(rep, 0), rfm.report_dict(rep, 1)
    assert r0["start"] == 0 and r0["r0norm"] >= r0["bnorm"]
    assert r1["start"] == 1 and r1["r0norm"] < r1["bnorm"]
    assert rfm.report_dict(repz, 0)["start"] == 0
    # the fallen-back instance is the zero-start run, bit for bit
    assert torch.equal(y[:nc], yz[:nc]) and torch.equal(a[:nc], az[:nc])
    assert r0["rnorm"] == rfm.report_dict(repz, 0)["rnorm"]
