"""Why an accurate learned start does not speed LSQR up on the learned
start's workload, measured with the oracle (no GPU).

Setting: the source family with overlap ratio 2.9 on 4 x 4 subdomains, K =
60, threshold 1e-6 (a small version of the learned start's workload).  The
preconditioned unknowns y reach the residual through A S^-1 and the function
values through E S^-1 (E: the window-weighted features at a test grid).  The
least-squares y* is unique here (more rows than kept columns, full rank) and
is taken from numpy's dense least squares, not from the oracle's LSQR.

Checks:
  * cond(E S^-1) is more than three decades above cond(A S^-1): function
    values see some directions of y far less than the residual does;
  * a start exact in function values but carrying a residual (y* plus a
    combination of the directions E S^-1 sees least) loses that accuracy in
    the first LSQR iterations: LSQR's iterates approach y* monotonically in
    the 2-norm (a property of LSQR/CGLS, Paige and Saunders 1982) while the
    function error rises by orders of magnitude.
"""
import numpy as np

import oracle
import synth


def _system():
    p = synth.param5(*synth.param5_draw(0), S=4, K=60, n=40, delta=2.9)
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    F = oracle.filter_blocks(B, 1e-6)
    S = oracle.build_system(B, F, mode=0, K=p.K)
    n = S.n
    AS = np.zeros((B.N, n))
    Cm = np.zeros((p.J * p.K, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0.0
        e[i] = 1.0
        AS[:, i] = S.matvec(e)
        Cm[:, i] = S.coefficients(e)
    X = oracle.test_grid(p, [30, 30])
    E = np.zeros((len(X), p.J * p.K))
    for j in range(p.J):
        w = np.array([oracle.window(p, j, x)[0] for x in X])
        E[:, j * p.K:(j + 1) * p.K] = w[:, None] * oracle.feature_values(p, prm, j, X)
    ES = E @ Cm
    # E S^-1 y is the ansatz at X: the same values as the oracle's evaluation
    a = S.coefficients(np.linspace(-1.0, 1.0, n))
    u = oracle.evaluate(p, prm, a, X)
    assert np.abs(ES @ np.linspace(-1.0, 1.0, n) - u).max() <= 1e-6 * np.abs(u).max()
    return B, S, AS, ES


def test_function_values_are_far_worse_conditioned_than_the_residual():
    B, S, AS, ES = _system()
    sA = np.linalg.svd(AS, compute_uv=False)
    sE = np.linalg.svd(ES, compute_uv=False)
    cA, cE = sA[0] / sA[-1], sE[0] / sE[-1]
    print(f"\ncond(A S^-1) = {cA:.2e}, cond(E S^-1) = {cE:.2e}")
    assert cE > 1e3 * cA


def test_lsqr_from_a_function_exact_start_loses_its_accuracy():
    B, S, AS, ES = _system()
    y = np.linalg.lstsq(AS, B.h, rcond=None)[0]
    u = ES @ y
    # twenty directions E S^-1 sees least, combined to carry a residual of 0.3 ||h||
    V = np.linalg.svd(ES, full_matrices=True)[2].T[:, -20:]
    c = np.linalg.lstsq(AS @ V, -B.h, rcond=None)[0]
    delta = V @ c
    delta *= 0.3 * np.linalg.norm(B.h) / np.linalg.norm(AS @ delta)
    y0 = y + delta
    f0 = np.linalg.norm(ES @ delta) / np.linalg.norm(u)
    e_prev = np.linalg.norm(delta)
    errs = []
    for it in (10, 30, 100):
        r = S.lsqr(B.h, y0=y0, atol=0, btol=0, max_iter=it)
        e = np.linalg.norm(r["y"] - y)
        assert e <= e_prev * (1 + 1e-9), (it, e, e_prev)      # monotone in y
        e_prev = e
        errs.append(np.linalg.norm(ES @ r["y"] - u) / np.linalg.norm(u))
    print(f"\nstart: function error {f0:.1e}, residual 0.3 ||h||; after 10 / 30 / 100 LSQR iterations: "
          + " / ".join(f"{v:.2f}" for v in errs))
    assert f0 < 1e-3
    assert errs[0] > 100 * f0
