"""Pins of the oracle's extensions to the paper's own problems and networks
(Sec. 4.1 problems, Eq. (2) networks of depth h, the activation ablations of
Tables 1 and 2), against facts that do not come from the oracle itself:

  * the oscillator's closed-form solution solves m u'' + mu u' + k u = 0 with
    u(0) = 1, u'(0) = 0 (finite differences);
  * the network features equal a plain numpy forward pass of Eq. (2) from the
    parameter layout (depth 1, 3, 5; tanh, sigmoid, sine);
  * every row of M is the row operator applied to the evaluated basis
    function g w_j phi_jk, by central differences of the oracle's evaluation
    with one unit coefficient: the oscillator's operator and its value and
    derivative rows, the hard-constraint Laplace rows, deep networks and the
    other activations;
  * the hard-constraint ansatz vanishes on the boundary;
  * dense least squares over the assembled system recovers the manufactured
    solutions (a dropped or mis-signed term would not).
"""
import numpy as np
import pytest

import oracle
import synth


def _unit_eval(p, prm, j, k, X):
    a = np.zeros(p.J * p.K)
    a[j * p.K + k] = 1.0
    return oracle.evaluate(p, prm, a, X)


def _act(act, s):
    if act == synth.ACT_SIGMOID:
        return 1.0 / (1.0 + np.exp(-s))
    if act == synth.ACT_SIN:
        return np.sin(s)
    return np.tanh(s)


def _numpy_features(p, prm, j, X):
    """Eq. (2) restated with numpy: hidden layers of K units, then the
    features, on the normalised input (x - mu)/sig."""
    mu, sig = oracle.subdomain(p, j)
    z = (X - mu[: p.dim]) / sig[: p.dim]
    v = np.asarray(prm).reshape(p.J, -1)[j]
    n_last = p.dim if p.depth <= 1 else p.K
    out = v[: p.K * (n_last + 1)].reshape(p.K, n_last + 1)
    o, nin = p.K * (n_last + 1), p.dim
    for _ in range(1, max(1, p.depth)):
        W = v[o: o + p.K * nin].reshape(p.K, nin)
        b = v[o + p.K * nin: o + p.K * (nin + 1)]
        z = _act(p.act, z @ W.T + b)
        o += p.K * (nin + 1)
        nin = p.K
    return _act(p.act, z @ out[:, :-1].T + out[:, -1])


def test_oscillator_exact_solution_solves_the_problem():
    p = synth.oscillator()
    m, mu, k = p.fparams
    u = lambda t: oracle.exact(p, np.array([[t]]))[0]
    e = 1e-5
    for t in (0.05, 0.3, 0.77):
        u2 = (u(t + e) - 2 * u(t) + u(t - e)) / e ** 2
        u1 = (u(t + e) - u(t - e)) / (2 * e)
        assert abs(m * u2 + mu * u1 + k * u(t)) <= 1e-4 * k
    assert u(0.0) == pytest.approx(1.0, abs=1e-15)
    assert (u(e) - u(-e)) / (2 * e) == pytest.approx(0.0, abs=1e-6 * np.sqrt(k))
    # the derivative row's data is u'
    x = np.array([0.37])
    dt = oracle.lib().orc_bdata_set(oracle.problem_struct(p), x.ctypes.data_as(oracle.C.c_void_p), 1)
    assert dt == pytest.approx((u(0.37 + e) - u(0.37 - e)) / (2 * e), rel=1e-6)


@pytest.mark.parametrize("depth", [1, 3, 5])
@pytest.mark.parametrize("act", [synth.ACT_TANH, synth.ACT_SIGMOID, synth.ACT_SIN])
def test_features_are_the_network_of_eq2(depth, act):
    p = synth.laplace_multiscale(S=3, K=6, depth=depth, act=act)
    prm = synth.feature_params(p)
    assert prm.size == p.J * p.params_per_subdomain
    assert prm.size == p.J * oracle.lib().orc_params_per_subdomain(oracle.problem_struct(p))
    rng = np.random.default_rng(1)
    for j in (0, 4, 8):
        X = rng.uniform(0, 1, (7, 2))
        Phi = oracle.feature_values(p, prm, j, X)
        assert np.allclose(Phi, _numpy_features(p, prm, j, X), rtol=0, atol=1e-14)


def _rows_match_fd(p, rows, cols, tol=2e-5):
    prm = synth.feature_params(p)
    M, h = oracle.assemble_dense(p, prm)
    z = oracle.sizes(p)
    X, kinds = oracle.row_points(p)
    sig = oracle.subdomain(p, 0)[1][: p.dim]
    e = 1e-4 * sig.min()
    checked = 0
    for r in rows:
        x = X[r]
        for col in cols:
            j, k = divmod(col, p.K)

            def f(dx):
                return _unit_eval(p, prm, j, k, (x + dx)[None, :])[0]

            d = [np.eye(p.dim)[i] * e for i in range(p.dim)]
            if kinds[r] < 0:
                if p.pde == synth.PDE_OSC:
                    m, mu, kk = p.fparams
                    v2 = (f(d[0]) - 2 * f(0 * d[0]) + f(-d[0])) / e ** 2
                    v1 = (f(d[0]) - f(-d[0])) / (2 * e)
                    want = (m * v2 + mu * v1 + kk * f(0 * d[0])) / np.sqrt(z["N_I"])
                else:
                    lap = sum((f(di) - 2 * f(0 * di) + f(-di)) / e ** 2 for di in d)
                    want = -lap / np.sqrt(z["N_I"])
            else:
                nb = np.sum(kinds == kinds[r])
                if p.pde == synth.PDE_OSC and kinds[r] == 1:
                    want = (f(d[0]) - f(-d[0])) / (2 * e) / np.sqrt(nb)
                else:
                    want = f(0 * d[0]) / np.sqrt(nb)
            scale = np.abs(M[:, col]).max() + 1e-30
            assert abs(M[r, col] - want) <= tol * scale, (r, col, M[r, col], want)
            checked += 1
    return checked, M, h


def test_oscillator_rows_match_finite_differences():
    p = synth.oscillator(S=5, K=4, omega0=12.0)
    z = oracle.sizes(p)
    assert z["N_I"] == 20 and z["N_B"] == 2
    X, kinds = oracle.row_points(p)
    assert list(kinds[-2:]) == [0, 1] and X[-1][0] == 0.0 and X[-2][0] == 0.0
    rows = [0, 3, 9, 14, 19, z["N"] - 2, z["N"] - 1]
    n, M, h = _rows_match_fd(p, rows, range(p.J * p.K))
    assert n == len(rows) * p.J * p.K
    assert h[-2] == pytest.approx(1.0) and h[-1] == 0.0 and np.all(h[:-2] == 0.0)


@pytest.mark.parametrize("depth,act", [(1, synth.ACT_TANH), (3, synth.ACT_TANH), (1, synth.ACT_SIGMOID),
                                       (1, synth.ACT_SIN), (5, synth.ACT_SIN)])
def test_hard_constraint_laplace_rows_match_finite_differences(depth, act):
    p = synth.laplace_multiscale(S=3, K=4, depth=depth, act=act)
    z = oracle.sizes(p)
    assert z["N_B"] == 0 and z["N_I"] == 36
    n, M, h = _rows_match_fd(p, [0, 7, 20, 35], range(0, p.J * p.K, 3))
    assert n > 0


def test_hard_constraint_vanishes_on_the_boundary():
    p = synth.laplace_multiscale(S=3, K=5)
    prm = synth.feature_params(p)
    a = np.random.default_rng(0).standard_normal(p.J * p.K)
    t = np.linspace(0, 1, 9)
    B = np.concatenate([np.stack([t, 0 * t], 1), np.stack([t, 0 * t + 1], 1), np.stack([0 * t, t], 1),
                        np.stack([0 * t + 1, t], 1)])
    assert np.all(oracle.evaluate(p, prm, a, B) == 0.0)
    assert np.abs(oracle.evaluate(p, prm, a, np.array([[0.4, 0.6]]))).max() > 0


@pytest.mark.parametrize("which", ["oscillator", "laplace"])
def test_paper_problems_are_recovered_by_dense_least_squares(which):
    if which == "oscillator":
        p = synth.oscillator(S=10, K=16, omega0=20.0)
        lim = 1e-4
    else:
        p = synth.laplace_multiscale(n_scales=2, S=4, K=36)
        lim = 2e-3
    prm = synth.feature_params(p)
    M, h = oracle.assemble_dense(p, prm)
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    k = int((s > 1e-12 * s[0]).sum())
    a = Vt[:k].T @ ((U[:, :k].T @ h) / s[:k])
    X = oracle.test_grid(p, [400] if p.dim == 1 else [30, 30])
    e = oracle.errors(oracle.evaluate(p, prm, a, X), oracle.exact(p, X))
    assert e["rel_l2"] < lim, e
