"""Pins of the oracle's fits of predicted values (learned warm start): the
local fit recovers predictions that the kept features represent exactly and
equals numpy's weighted least squares at full rank; the partition of unity
turns exact local predictions into the solution; LSQR started from a fit
needs fewer iterations than from zero; the blend of identical per-block
predictions is the prediction itself; and the global fit run to convergence
equals numpy's least squares on the assembled window-weighted value matrix."""
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
        w = np.array([oracle.window(p, j, x)[0] for x in X])
        Phi = w[:, None] * oracle.feature_values(p, prm, j, X)[:, f.perm[: f.rank]]
        assert np.linalg.matrix_rank(Phi) == f.rank
        ref = np.linalg.lstsq(Phi, w * uh[j], rcond=None)[0]
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


def test_blend_of_identical_predictions_is_the_prediction():
    p = synth.poisson2d(S=4, K=6, n=20, delta=2.0)
    prm, B, F = _setup(p)
    f = lambda X: np.sin(2 * X[:, 0]) * np.cos(X[:, 1])
    uh = [f(oracle.row_points(p, g)[0]) for g in B.grow]
    ub = oracle.blend(p, B, uh)
    Xr, _ = oracle.row_points(p, np.arange(B.N))
    assert ub == pytest.approx(f(Xr), rel=1e-13, abs=1e-14)


def test_global_fit_converges_to_least_squares_on_the_value_matrix():
    p = synth.poisson1d(S=4, K=6, n=40)
    prm, B, F = _setup(p)
    rng = np.random.default_rng(3)
    uh = [rng.standard_normal(len(g)) for g in B.grow]
    ys, cs, res = oracle.global_fit(p, prm, B, F, uh, tol_fit=1e-14, iters=5000)
    # the assembled N x (sum r_j) matrix of window-weighted kept features
    cols = sum(f.rank for f in F)
    A = np.zeros((B.N, cols))
    c0 = 0
    for j, (g, f) in enumerate(zip(B.grow, F)):
        X, _ = oracle.row_points(p, g)
        w = np.array([oracle.window(p, j, x)[0] for x in X])
        A[g, c0:c0 + f.rank] = w[:, None] * oracle.feature_values(p, prm, j, X)[:, f.perm[: f.rank]]
        c0 += f.rank
    ub = oracle.blend(p, B, uh)
    assert np.linalg.matrix_rank(A) == cols
    ref = np.linalg.lstsq(A, ub, rcond=None)[0]
    got = np.concatenate(cs)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(A @ got - ub) <= np.linalg.norm(A @ ref - ub) * (1 + 1e-8) + 1e-12
    assert got == pytest.approx(ref, rel=1e-12 * kappa, abs=1e-12 * kappa * np.abs(ref).max())
