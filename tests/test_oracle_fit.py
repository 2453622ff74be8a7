"""Pins of the oracle's local fit (learned warm start): predictions that the
kept features represent exactly are recovered exactly; a full-rank fit equals
numpy's least squares; the partition of unity turns exact local predictions
into a global approximation of the solution; and LSQR started from the fit
needs fewer iterations than from zero."""
import numpy as np
import pytest

import oracle
import synth


def _setup(p, tol=1e-10):
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    F = oracle.filter_blocks(B, tol)
    return prm, B, F


def test_feature_values_are_the_features():
    p = synth.poisson2d(S=3, K=5, n=9)
    prm = synth.feature_params(p)
    j = 4
    mu, sig = oracle.subdomain(p, j)
    X = np.array([[0.3, 0.6], [0.45, 0.5]])
    Phi = oracle.feature_values(p, prm, j, X)
    P = prm.reshape(-1, p.K, p.dim + 1)[j]
    for i, x in enumerate(X):
        z = P[:, :2] @ ((x - mu) / sig) + P[:, 2]
        assert Phi[i] == pytest.approx(np.tanh(z), rel=1e-14)


def test_representable_predictions_are_recovered():
    p = synth.poisson1d(S=3, K=6, n=30)
    prm, B, F = _setup(p)
    rng = np.random.default_rng(0)
    uh, ctrue, kap = [], [], []
    for j, (g, f) in enumerate(zip(B.grow, F)):
        X, _ = oracle.row_points(p, g)
        Phi = oracle.feature_values(p, prm, j, X)[:, f.perm[: f.rank]]
        c = rng.standard_normal(f.rank)
        ctrue.append(c)
        uh.append(Phi @ c)
        kap.append(np.linalg.cond(Phi))
    ys, cs = oracle.local_fit(p, prm, B, F, uh, tol_fit=1e-13)
    for c, ct, y, f, k in zip(cs, ctrue, ys, F, kap):
        tol = 1e-13 * max(1.0, k)
        assert c == pytest.approx(ct, rel=tol, abs=tol)
        assert y == pytest.approx(f.R @ ct, rel=tol, abs=tol * np.abs(f.R @ ct).max())


def test_full_rank_fit_is_numpy_least_squares():
    p = synth.poisson1d(S=4, K=5, n=40)
    prm, B, F = _setup(p)
    rng = np.random.default_rng(1)
    uh = [rng.standard_normal(len(g)) for g in B.grow]
    ys, cs = oracle.local_fit(p, prm, B, F, uh, tol_fit=1e-14)
    for j, (g, f) in enumerate(zip(B.grow, F)):
        X, _ = oracle.row_points(p, g)
        Phi = oracle.feature_values(p, prm, j, X)[:, f.perm[: f.rank]]
        assert np.linalg.matrix_rank(Phi) == f.rank
        ref = np.linalg.lstsq(Phi, uh[j], rcond=None)[0]
        kappa = np.linalg.cond(Phi)
        assert cs[j] == pytest.approx(ref, rel=1e-13 * kappa, abs=1e-13 * kappa * np.abs(ref).max())


def test_exact_local_predictions_give_the_solution_by_partition_of_unity():
    # predictions equal to the exact solution at every block's rows: the
    # warm-start coefficients evaluate to that solution (up to how well each
    # block's features represent it) and the system residual is small
    # (with 8 subdomains of 60 features the converged solve's error is 1.0e-3)
    p = synth.poisson1d(S=8, K=60, n=400)
    prm, B, F = _setup(p)
    uh = []
    for g in B.grow:
        X, _ = oracle.row_points(p, g)
        uh.append(oracle.exact(p, X))
    ys, cs = oracle.local_fit(p, prm, B, F, uh, tol_fit=1e-10)
    S = oracle.build_system(B, F)
    y0 = np.concatenate(ys)
    a0 = S.coefficients(y0)
    Xt = oracle.test_grid(p, [1000])
    err = oracle.errors(oracle.evaluate(p, prm, a0, Xt), oracle.exact(p, Xt))["rel_l2"]
    assert err < 1e-3
    # a zero start has relative residual 1
    r0 = np.linalg.norm(S.matvec(y0) - B.h) / np.linalg.norm(B.h)
    assert r0 < 0.05


def test_warm_start_needs_fewer_lsqr_iterations():
    p = synth.poisson1d(S=8, K=60, n=400)
    prm, B, F = _setup(p)
    uh = []
    for g in B.grow:
        X, _ = oracle.row_points(p, g)
        uh.append(oracle.exact(p, X))
    ys, _ = oracle.local_fit(p, prm, B, F, uh, tol_fit=1e-10)
    S = oracle.build_system(B, F)
    cold = S.lsqr(B.h, atol=1e-9, btol=1e-9, max_iter=20000)
    warm = S.lsqr(B.h, y0=np.concatenate(ys), atol=1e-9, btol=1e-9, max_iter=20000)
    assert warm["istop"] in (1, 2) and cold["istop"] in (1, 2)
    assert warm["itn"] < cold["itn"]
