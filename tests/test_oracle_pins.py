"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to a published value, a closed form, a
library routine or an invariant of the mathematics, chosen so that a plausible
mistake (a dropped term, a sign, a transposed operand, a wrong index) fails.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------

def test_splitmix64_known_answers():
    lines = [l.strip() for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    want = [int(x, 16) for x in lines[1:]]
    got = [int(v) for v in synth.splitmix64_u64(seed, len(want))]
    assert got == want


def test_splitmix64_offset_and_unit_range():
    a = synth.splitmix64_u64(7, 10)
    b = synth.splitmix64_u64(7, 4, offset=6)
    assert list(a[6:]) == list(b)
    u = synth.splitmix64_unit(3, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


# --------------------------------------------------------------------------
# decomposition and windows (Sec. 4.2)
# --------------------------------------------------------------------------

def _prob(dim, S, delta, pde=synth.PDE_POISSON, n=8, K=4):
    fam = synth.FAM_SINPROD if pde == synth.PDE_POISSON else synth.FAM_HEAT_SINPROD
    return synth.Problem(dim=dim, pde=pde, S=[S] * dim, delta=delta, K=K, n=[n] * dim, family=fam,
                         coef=[1.0], waves=[[1.0] * (dim if pde == 0 else dim - 1)], kappa=0.1)


def test_subdomain_boxes_follow_decomposition_formula():
    # S = 5 on [0, 1], delta = 1.5: spacing 1/4, centres 0, .25, .5, .75, 1, half-width .1875
    p = _prob(1, 5, 1.5)
    for j in range(5):
        mu, sg = oracle.subdomain(p, j)
        assert mu[0] == pytest.approx(0.25 * j, abs=1e-15)
        assert sg[0] == pytest.approx(0.1875, abs=1e-15)


def test_window_closed_form_values_1d():
    # S = 2 on [0,1], delta = 1.5: mu = 0, 1, sigma = 0.75.
    # x = 0.5: both hats equal (1 + cos(2 pi/3))^2 = 1/4 -> w_0 = 1/2.
    # x = 0.25: the second box excludes the point (|0.25 - 1| = 0.75 is not < 0.75) -> w_0 = 1.
    # x = 0.4: hats (1 + cos(pi 0.4/0.75))^2 and (1 + cos(pi 0.6/0.75))^2.
    p = _prob(1, 2, 1.5)
    assert oracle.window(p, 0, [0.5])[0] == pytest.approx(0.5, abs=1e-15)
    assert oracle.window(p, 0, [0.25])[0] == pytest.approx(1.0, abs=1e-15)
    assert oracle.window(p, 1, [0.25])[0] == 0.0
    h0 = (1 + np.cos(np.pi * 0.4 / 0.75)) ** 2
    h1 = (1 + np.cos(np.pi * 0.6 / 0.75)) ** 2
    assert oracle.window(p, 0, [0.4])[0] == pytest.approx(h0 / (h0 + h1), rel=1e-14)
    assert oracle.window(p, 0, [0.4], normalised=False)[0] == pytest.approx(h0, rel=1e-14)


@pytest.mark.parametrize("dim,S,delta", [(1, 7, 1.3), (2, 4, 1.25), (3, 3, 1.2), (2, 5, 2.9)])
def test_partition_of_unity_and_derivative_sums(dim, S, delta):
    p = _prob(dim, S, delta)
    rng = np.random.default_rng(1)
    J = p.J
    for _ in range(20):
        x = rng.uniform(0, 1, dim)
        w = np.zeros(J)
        dw = np.zeros((J, dim))
        d2w = np.zeros((J, dim))
        for j in range(J):
            w[j], dw[j], d2w[j] = oracle.window(p, j, x)
        sig = oracle.subdomain(p, 0)[1]
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.all(w >= 0)
        assert np.abs(dw.sum(0)).max() * sig.min() < 1e-12
        assert np.abs(d2w.sum(0)).max() * sig.min() ** 2 < 1e-10


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_window_derivatives_match_finite_differences(dim):
    p = _prob(dim, 4, 1.4)
    rng = np.random.default_rng(2)
    sig = oracle.subdomain(p, 0)[1][0]
    e = 1e-5 * sig
    checked = 0
    for _ in range(40):
        x = rng.uniform(0, 1, dim)
        for j in range(p.J):
            w, dw, d2w = oracle.window(p, j, x)
            if w == 0.0:
                continue
            for i in range(dim):
                xp, xm = x.copy(), x.copy()
                xp[i] += e
                xm[i] -= e
                wp, wm = oracle.window(p, j, xp)[0], oracle.window(p, j, xm)[0]
                if wp == 0.0 or wm == 0.0:
                    continue
                assert dw[i] * sig == pytest.approx((wp - wm) / (2 * e) * sig, abs=1e-6)
                assert d2w[i] * sig ** 2 == pytest.approx((wp - 2 * w + wm) / e ** 2 * sig ** 2, abs=1e-3)
                checked += 1
    assert checked > 20


def test_normalised_window_factorises_over_dimensions():
    # On a tensor-product decomposition the sum of hats factorises, so the
    # normalised window is the product of 1D normalised windows.
    p2 = _prob(2, 4, 1.3)
    p1 = _prob(1, 4, 1.3)
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.uniform(0, 1, 2)
        for j in range(p2.J):
            j0, j1 = j % 4, j // 4
            w2 = oracle.window(p2, j, x)[0]
            assert w2 == pytest.approx(oracle.window(p1, j0, [x[0]])[0] * oracle.window(p1, j1, [x[1]])[0],
                                       abs=1e-15)


# --------------------------------------------------------------------------
# collocation rows and assembly (Sec. 2.1, Eqs. (4)-(6))
# --------------------------------------------------------------------------

def test_row_counts_and_points():
    p = synth.poisson2d(S=4, K=5, n=10)
    z = oracle.sizes(p)
    assert z["N_I"] == 100 and z["N_B"] == 40
    X, kinds = oracle.row_points(p)
    assert np.all(kinds[:100] == -1) and np.all(kinds[100:] == 0)
    assert X[0] == pytest.approx([0.05, 0.05]) and X[1] == pytest.approx([0.15, 0.05])
    assert X[100] == pytest.approx([0.0, 0.05]) and X[110] == pytest.approx([1.0, 0.05])
    assert X[120] == pytest.approx([0.05, 0.0]) and X[139] == pytest.approx([0.95, 1.0])
    h = synth.heat3d(S=3, K=4, n=5)
    zh = oracle.sizes(h)
    assert zh["N_I"] == 125 and zh["N_B"] == 5 * 25
    Xh, kh = oracle.row_points(h)
    assert np.all(kh[125:225] == 0) and np.all(kh[225:] == 1)
    assert np.all(Xh[225:, 2] == 0.0)


def _unit_eval(p, prm, j, k, X):
    a = np.zeros(p.J * p.K)
    a[j * p.K + k] = 1.0
    return oracle.evaluate(p, prm, a, X)


@pytest.mark.parametrize("which", ["poisson1d", "poisson2d", "heat3d"])
def test_operator_rows_match_finite_differences(which):
    """N[w_j phi_jk](x)/sqrt(N_I) against central differences of the evaluated
    basis function w_j phi_jk (Eq. (1) with one unit coefficient)."""
    if which == "poisson1d":
        p = synth.poisson1d(S=4, K=6, n=40)
    elif which == "poisson2d":
        p = synth.poisson2d(S=3, K=5, n=12)
    else:
        p = synth.heat3d(S=3, K=4, n=6)
    prm = synth.feature_params(p)
    M, _ = oracle.assemble_dense(p, prm)
    z = oracle.sizes(p)
    X, kinds = oracle.row_points(p)
    rng = np.random.default_rng(4)
    sig = oracle.subdomain(p, 0)[1]
    e = 1e-4 * sig.min()
    for r in rng.choice(z["N_I"], 6, replace=False):
        for j in range(p.J):
            for k in range(min(p.K, 3)):
                x = X[r]

                def f(dx):
                    return _unit_eval(p, prm, j, k, (x + dx)[None, :])[0]

                lap = 0.0
                nsp = p.dim if p.pde == synth.PDE_POISSON else p.dim - 1
                for i in range(nsp):
                    d = np.zeros(p.dim)
                    d[i] = e
                    lap += (f(d) - 2 * f(0 * d) + f(-d)) / e ** 2
                if p.pde == synth.PDE_POISSON:
                    want = -lap
                else:
                    d = np.zeros(p.dim)
                    d[-1] = e
                    want = (f(d) - f(-d)) / (2 * e) - p.kappa * lap
                want /= np.sqrt(z["N_I"])
                got = M[r, j * p.K + k]
                scale = np.abs(M[:, j * p.K + k]).max() + 1e-30
                assert abs(got - want) <= 2e-5 * scale, (r, j, k, got, want)


def test_boundary_rows_are_scaled_traces():
    p = synth.heat3d(S=3, K=4, n=5)
    prm = synth.feature_params(p)
    M, h = oracle.assemble_dense(p, prm)
    z = oracle.sizes(p)
    X, kinds = oracle.row_points(p)
    NB = [np.sum(kinds == 0), np.sum(kinds == 1)]
    for r in [z["N_I"], z["N_I"] + 30, z["N"] - 1]:
        l = kinds[r]
        for col in [0, 7, p.J * p.K - 1]:
            j, k = divmod(col, p.K)
            v = _unit_eval(p, prm, j, k, X[r][None, :])[0]
            assert M[r, col] == pytest.approx(np.sqrt(1.0 / NB[l]) * v, abs=1e-14)
        assert h[r] == pytest.approx(np.sqrt(1.0 / NB[l]) * oracle.exact(p, X[r][None, :])[0], abs=1e-14)


@pytest.mark.parametrize("which", ["poisson2d", "heat3d"])
def test_source_matches_finite_difference_of_exact_solution(which):
    p = synth.poisson2d() if which == "poisson2d" else synth.heat3d()
    rng = np.random.default_rng(5)
    e = 1e-4
    for _ in range(5):
        x = rng.uniform(0.1, 0.9, p.dim)
        u = lambda y: oracle.exact(p, y[None, :])[0]
        lap = 0.0
        nsp = p.dim if p.pde == 0 else p.dim - 1
        for i in range(nsp):
            d = np.zeros(p.dim)
            d[i] = e
            lap += (u(x + d) - 2 * u(x) + u(x - d)) / e ** 2
        if p.pde == 0:
            want = -lap
        else:
            d = np.zeros(p.dim)
            d[-1] = e
            want = (u(x + d) - u(x - d)) / (2 * e) - p.kappa * lap
        got = oracle.source(p, x)
        assert got == pytest.approx(want, abs=1e-4 * max(1.0, abs(want)))


def test_block_decomposition_identity():
    """M = sum_j V_j^T M_j W_j (Eq. (6)): blocks are the nonzero pattern of M."""
    p = synth.poisson2d(S=4, K=3, n=10)
    prm = synth.feature_params(p)
    M, h = oracle.assemble_dense(p, prm)
    B = oracle.assemble(p, prm)
    R = np.zeros_like(M)
    for j, (g, Mj) in enumerate(zip(B.grow, B.M)):
        R[np.ix_(g, np.arange(j * p.K, (j + 1) * p.K))] += Mj
    assert np.array_equal(R, M)
    assert np.array_equal(B.h, h)


def test_manufactured_solution_is_recovered_by_dense_least_squares():
    """Pins signs and terms of the whole assembly: a wrong sign or a dropped
    chain-rule term leaves a large error against the exact u."""
    p = synth.poisson1d(S=8, K=40, n=400)
    p.coef, p.waves = [1.0, 0.3], [[2.0], [5.0]]
    prm = synth.feature_params(p)
    M, h = oracle.assemble_dense(p, prm)
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    k = int((s > 1e-12 * s[0]).sum())
    a = Vt[:k].T @ ((U[:, :k].T @ h) / s[:k])
    X = oracle.test_grid(p, [500])
    e = oracle.errors(oracle.evaluate(p, prm, a, X), oracle.exact(p, X))
    assert e["rel_l2"] < 1e-7


def test_manufactured_solution_2d_and_heat():
    p2 = synth.poisson2d(S=3, K=64, n=36, R=2.0)
    p2.coef, p2.waves = [1.0], [[1.0, 2.0]]
    p3 = synth.heat3d(S=2, K=100, n=12, k=1.0, R=2.0)
    for p, lim in [(p2, 3e-4), (p3, 3e-3)]:
        prm = synth.feature_params(p)
        M, h = oracle.assemble_dense(p, prm)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        k = int((s > 1e-10 * s[0]).sum())
        a = Vt[:k].T @ ((U[:, :k].T @ h) / s[:k])
        X = oracle.test_grid(p, [12] * p.dim)
        e = oracle.errors(oracle.evaluate(p, prm, a, X), oracle.exact(p, X))
        assert e["rel_l2"] < lim, e


# --------------------------------------------------------------------------
# sigma-RRQR filtering (Algorithm 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,n", [(30, 20), (20, 30), (25, 25), (1, 4), (5, 1)])
def test_qrcp_reconstructs_and_is_orthonormal(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n)) * np.logspace(0, -3, n)[None, :]
    f = oracle.qrcp(A, 0.0)
    r = f.rank
    assert r == min(m, n)
    Q = f.Q()
    R = np.triu(f.QR[:r, :])
    eps = np.finfo(float).eps
    assert np.linalg.norm(A[:, f.perm] - Q @ R) <= 50 * eps * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(r)) <= 50 * eps
    d = np.abs(np.diag(R))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))
    assert sorted(f.perm) == list(range(n))


def test_qrcp_diagonal_matrix_closed_form():
    """On a permuted diagonal the pivots come out in decreasing order, |R_kk|
    are the sorted magnitudes, and the kept count is #{|d| >= tol max|d|}.
    Powers of two make every threshold exact: an entry equal to tol |R_11|
    is kept (the drop test is strict)."""
    d = np.array([4.0, -2.0 ** -10, 8.0, 2.0 ** -20, 1.0, -2.0 ** -14, 2.0 ** -30])
    A = np.zeros((9, 7))
    A[np.arange(7), np.arange(7)] = d
    A = A[np.random.default_rng(0).permutation(9)]
    order = np.argsort(-np.abs(d), kind="stable")
    f = oracle.qrcp(A, 0.0)
    assert list(f.perm) == list(order)
    assert np.abs(np.diag(f.QR[:7, :7])) == pytest.approx(np.abs(d[order]), rel=1e-15)
    for tol in [2.0 ** -2, 2.0 ** -12, 2.0 ** -16, 2.0 ** -25, 2.0 ** -40]:
        assert oracle.qrcp(A, tol).rank == int((np.abs(d) >= tol * 8.0).sum())
    assert oracle.qrcp(A, 2.0 ** -23).rank == 6      # 2^-20 == tol * 8: kept
    assert oracle.qrcp(A, 2.0 ** -23 * (1 + 2.0 ** -50)).rank == 5


def test_qrcp_rank_equals_numerical_rank_with_spectral_gap():
    rng = np.random.default_rng(7)
    for trial in range(10):
        m, n = rng.integers(20, 60), rng.integers(20, 60)
        k = int(rng.integers(1, min(m, n)))
        U = np.linalg.qr(rng.standard_normal((m, m)))[0]
        V = np.linalg.qr(rng.standard_normal((n, n)))[0]
        s = np.concatenate([np.logspace(0, -2, k), np.logspace(-12, -14, min(m, n) - k)])
        A = (U[:, : len(s)] * s) @ V[:, : len(s)].T
        f = oracle.qrcp(A, 1e-7)
        sv = np.linalg.svd(A, compute_uv=False)
        assert f.rank == int((sv > 1e-7 * sv[0]).sum()) == k


def test_qrcp_pivots_match_lapack():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(8)
    for trial in range(5):
        A = rng.standard_normal((40, 30)) @ np.diag(rng.uniform(0.1, 10, 30))
        f = oracle.qrcp(A, 0.0)
        _, Rs, piv = scipy_linalg.qr(A, pivoting=True, mode="economic")
        assert list(f.perm) == list(piv)
        assert np.abs(np.diag(f.QR[:30, :30])) == pytest.approx(np.abs(np.diag(Rs)), rel=1e-10)


def test_qrcp_zero_matrix_and_zero_columns():
    assert oracle.qrcp(np.zeros((5, 4)), 1e-10).rank == 0
    A = np.zeros((6, 4))
    A[:, 2] = np.arange(6)
    f = oracle.qrcp(A, 1e-10)
    assert f.rank == 1 and f.perm[0] == 2


def test_trsv_matches_library_solve():
    rng = np.random.default_rng(9)
    R = np.triu(rng.standard_normal((12, 12))) + 5 * np.eye(12)
    x = rng.standard_normal(12)
    assert oracle.trsv(R, x) == pytest.approx(np.linalg.solve(R, x), rel=1e-12)
    assert oracle.trsv(R, x, trans=True) == pytest.approx(np.linalg.solve(R.T, x), rel=1e-12)


# --------------------------------------------------------------------------
# preconditioner (Sec. 3.2, Proposition 3.1, Theorem 3.2, the J = 2 remark)
# --------------------------------------------------------------------------

def _small_1d(S=6, K=20, n=120, delta=1.3, tol=1e-8):
    p = synth.poisson1d(S=S, K=K, n=n, delta=delta)
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    F = oracle.filter_blocks(B, tol)
    return p, prm, B, F


def test_proposition_3_1_and_orthonormal_blocks():
    p, prm, B, F = _small_1d()
    eps = np.finfo(float).eps
    for M, f in zip(B.M, F):
        Q = f.Q()
        Ahat = M[:, f.perm[: f.rank]]
        X = np.linalg.solve(f.R.T, Ahat.T).T   # Ahat R^-1
        kappa = np.linalg.cond(f.R)
        assert np.linalg.norm(X - Q) <= 10 * kappa * eps * np.sqrt(f.rank)
        assert np.linalg.norm(Q.T @ Q - np.eye(f.rank)) <= 100 * eps


def test_preconditioned_operator_equals_explicit_q():
    p, prm, B, F = _small_1d()
    S0 = oracle.build_system(B, F, mode=0)
    S1 = oracle.build_system(B, F, mode=1)
    rng = np.random.default_rng(10)
    x = rng.standard_normal(S0.n)
    y = rng.standard_normal(S0.N)
    # A_hat R^-1 by substitution and Q_hat agree up to rounding amplified by kappa(R_hat)
    kap = max(np.linalg.cond(f.R) for f in F)
    tol = 100 * np.finfo(float).eps * kap
    assert np.linalg.norm(S0.matvec(x) - S1.matvec(x)) <= tol * np.linalg.norm(x)
    assert np.linalg.norm(S0.rmatvec(y) - S1.rmatvec(y)) <= tol * np.linalg.norm(y)
    # adjointness of the forward and transposed applications
    assert abs(np.dot(S0.matvec(x), y) - np.dot(x, S0.rmatvec(y))) <= tol * np.linalg.norm(x) * np.linalg.norm(y)


def _global_q(B, F):
    n = sum(f.rank for f in F)
    Q = np.zeros((B.N, n))
    c = 0
    for g, f in zip(B.grow, F):
        Q[g, c:c + f.rank] = f.Q()
        c += f.rank
    return Q


def test_two_block_condition_number_is_exact():
    """J = 2: kappa(Q) = sqrt((1 + ||A_1||) / (1 - ||A_1||)), A_1 the overlap coupling."""
    p, prm, B, F = _small_1d(S=2, K=12, n=60, delta=1.6, tol=1e-6)
    Q = _global_q(B, F)
    r0 = F[0].rank
    A1 = Q[:, :r0].T @ Q[:, r0:]
    a = np.linalg.norm(A1, 2)
    assert a < 1
    sv = np.linalg.svd(Q, compute_uv=False)
    assert sv[0] / sv[-1] == pytest.approx(np.sqrt((1 + a) / (1 - a)), rel=1e-8)


def test_theorem_3_2_bound_holds_on_a_1d_strip():
    p, prm, B, F = _small_1d(S=5, K=10, n=200, delta=1.1, tol=1e-3)
    Q = _global_q(B, F)
    offs = np.concatenate([[0], np.cumsum([f.rank for f in F])])
    alpha = max(np.linalg.norm(Q[:, offs[j]:offs[j + 1]].T @ Q[:, offs[j + 1]:offs[j + 2]], 2)
                for j in range(len(F) - 1))
    sv = np.linalg.svd(Q, compute_uv=False)
    if 2 * alpha < 1:
        assert sv[0] / sv[-1] <= np.sqrt((1 + 2 * alpha) / (1 - 2 * alpha)) * (1 + 1e-12)
    else:
        pytest.skip("coupling too strong for the bound on this draw")


# --------------------------------------------------------------------------
# LSQR (Paige and Saunders 1982) on the block operator
# --------------------------------------------------------------------------

def _dense_system(A, mode=1):
    """A dense matrix packed as one block so the oracle LSQR runs on it."""
    m, n = A.shape
    return oracle.FilteredSystem(m, [np.arange(m)], [np.asfortranarray(A)], None, mode=1,
                                 perms=[np.arange(n, dtype=np.int32)], K=n)


def test_lsqr_full_rank_matches_lstsq():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 15))
    b = rng.standard_normal(40)
    S = _dense_system(A)
    res = S.lsqr(b, atol=1e-14, btol=1e-14, max_iter=500)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    assert res["y"] == pytest.approx(x, rel=1e-10, abs=1e-12)
    assert res["istop"] in (1, 2)
    assert res["rnorm"] == pytest.approx(np.linalg.norm(b - A @ res["y"]), rel=1e-8)


def test_lsqr_underdetermined_gives_min_norm_solution():
    rng = np.random.default_rng(12)
    A = rng.standard_normal((12, 30))
    b = rng.standard_normal(12)
    res = _dense_system(A).lsqr(b, atol=1e-14, btol=1e-14, max_iter=500)
    assert res["y"] == pytest.approx(np.linalg.pinv(A) @ b, rel=1e-9, abs=1e-12)


def test_lsqr_iterates_are_krylov_minimisers():
    rng = np.random.default_rng(13)
    A = rng.standard_normal((30, 20))
    b = rng.standard_normal(30)
    S = _dense_system(A)
    K = [A.T @ b]
    for k in range(1, 7):
        res = S.lsqr(b, atol=0, btol=0, max_iter=k)
        V = np.linalg.qr(np.array(K).T)[0]
        c = np.linalg.lstsq(A @ V, b, rcond=None)[0]
        assert res["y"] == pytest.approx(V @ c, rel=1e-8, abs=1e-10)
        K.append(A.T @ (A @ K[-1]))


def _krylov_basis(Op, b, k):
    """Orthonormal basis of span{Op^T b, (Op^T Op) Op^T b, ...} (k vectors),
    each new direction orthogonalised twice against the previous ones."""
    v = Op.T @ b
    V = [v / np.linalg.norm(v)]
    for _ in range(1, k):
        w = Op.T @ (Op @ V[-1])
        for _rep in range(2):
            for q in V:
                w = w - (q @ w) * q
        V.append(w / np.linalg.norm(w))
    return np.array(V).T


def test_lsqr_iterates_are_krylov_minimisers_on_the_preconditioned_operator():
    """Iterate k (k <= 10) of the oracle's LSQR on A S^-1 (Algorithm 2's
    operator, triangular substitution with the filter's R_j) minimises
    ||h - A S^-1 y|| over the k-th Krylov space of (A S^-1)^T (A S^-1) and
    (A S^-1)^T h (Paige and Saunders 1982); the dense A S^-1 is formed column
    by column from the oracle's own products on a small 1D problem, and its
    transpose product is checked against the oracle's too.  The products
    apply R_j^-1 by substitution, so two mathematically equal ways of forming
    them differ by rounding of order eps kappa(R_j) (measured: 1e-8 relative
    at kappa 1.2e8, 1e-10 at 3e6); the tolerance is 10 eps max kappa(R_j)."""
    p = synth.poisson1d(S=4, K=10, n=48)
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    for tol in (1e-8, 1e-6):
        F = oracle.filter_blocks(B, tol)
        rtol = 10 * np.finfo(float).eps * max(np.linalg.cond(f.R) for f in F)
        Sy = oracle.build_system(B, F, mode=0)
        Op = np.stack([Sy.matvec(e) for e in np.eye(Sy.n)], axis=1)
        z = np.random.default_rng(21).standard_normal(B.N)
        ref = Op.T @ z
        assert np.abs(Sy.rmatvec(z) - ref).max() <= rtol * np.abs(ref).max()
        h = B.h
        for k in range(1, 11):
            res = Sy.lsqr(h, atol=0, btol=0, max_iter=k)
            V = _krylov_basis(Op, h, k)
            c = np.linalg.lstsq(Op @ V, h, rcond=None)[0]
            y = V @ c
            assert np.abs(res["y"] - y).max() <= rtol * np.abs(y).max(), (tol, k)
            # and its residual is the smallest over that space
            assert np.linalg.norm(h - Op @ res["y"]) <= np.linalg.norm(h - Op @ y) * (1 + rtol)


def test_lsqr_residual_estimates_are_monotone_and_exact():
    rng = np.random.default_rng(14)
    A = rng.standard_normal((50, 30)) @ np.diag(np.logspace(0, -4, 30))
    b = rng.standard_normal(50)
    S = _dense_system(A)
    res = S.lsqr(b, atol=0, btol=0, max_iter=25, history=True)
    h = res["rhist"]
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-14))
    assert res["rnorm"] == pytest.approx(np.linalg.norm(b - A @ res["y"]), rel=1e-9)


def test_lsqr_warm_start_and_exact_start():
    rng = np.random.default_rng(15)
    A = rng.standard_normal((25, 10))
    x = rng.standard_normal(10)
    b = A @ x
    S = _dense_system(A)
    res = S.lsqr(b, y0=x, atol=1e-12, btol=1e-12)
    assert res["itn"] <= 1 and res["y"] == pytest.approx(x, rel=1e-10)
    res2 = S.lsqr(b, y0=x + 1e-3 * rng.standard_normal(10), atol=1e-13, btol=1e-13)
    assert res2["y"] == pytest.approx(x, rel=1e-9)


def test_lsqr_stops_by_stated_rules():
    rng = np.random.default_rng(16)
    A = rng.standard_normal((30, 10))
    b = rng.standard_normal(30)
    res = _dense_system(A).lsqr(b, atol=1e-6, btol=1e-6, max_iter=100)
    assert res["istop"] == 2 and res["arnorm"] <= 1e-6 * res["anorm"] * res["rnorm"]
    res = _dense_system(A).lsqr(A @ np.ones(10), atol=1e-6, btol=1e-6, max_iter=100)
    assert res["istop"] in (1, 2)
    res = _dense_system(A).lsqr(b, atol=0, btol=0, max_iter=3)
    assert res["istop"] == 7 and res["itn"] == 3


# --------------------------------------------------------------------------
# Algorithm 2 end to end
# --------------------------------------------------------------------------

def test_algorithm2_output_layout_and_least_squares_optimality():
    p, prm, B, F = _small_1d(S=4, K=16, n=80, tol=1e-6)
    S = oracle.build_system(B, F, mode=0)
    res = S.lsqr(B.h, atol=1e-13, btol=1e-13, max_iter=20000)
    a = S.coefficients(res["y"])
    for j, f in enumerate(F):
        dropped = sorted(set(range(p.K)) - set(f.perm[: f.rank]))
        assert np.all(a[j * p.K + np.array(dropped, dtype=int)] == 0.0) if dropped else True
    # a minimises ||M a - h|| over the kept columns: compare with lstsq on Mhat
    M, h = oracle.assemble_dense(p, prm)
    kept = np.concatenate([j * p.K + f.perm[: f.rank] for j, f in enumerate(F)])
    ak = np.linalg.lstsq(M[:, kept], h, rcond=None)[0]
    assert np.linalg.norm(M @ a - h) == pytest.approx(np.linalg.norm(M[:, kept] @ ak - h), rel=1e-6)


def test_error_metrics_definitions():
    u = np.array([1.0, 2.0, 3.0, 4.0])
    uh = u + np.array([0.1, -0.1, 0.0, 0.2])
    e = oracle.errors(uh, u)
    assert e["rel_l2"] == pytest.approx(np.sqrt(0.06) / np.sqrt(30.0))
    assert e["e_l1"] == pytest.approx(0.1 / np.std(u))
