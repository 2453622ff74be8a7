"""Host-side pieces of the threshold sweep (no GPU): the test grid and the
errors it derives from the evaluation's sums, against the oracle's own test
grid and its error definitions (relative L2, and e_L1 of Sec. 4.2)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("p", [synth.poisson1d(S=4, K=5, n=20, n_test=37), synth.poisson2d(S=3, K=4, n=9, n_test=11),
                               synth.heat3d(S=2, K=3, n=4, n_test=5)])
def test_grid_is_the_oracles(p):
    from paper_2506_17626_gb300.sweep import grid_points
    np.testing.assert_array_equal(grid_points(p), oracle.test_grid(p))


def test_errors_from_sums_match_the_definitions():
    from paper_2506_17626_gb300.sweep import errors_from_sums
    rng = np.random.default_rng(3)
    u = rng.standard_normal(500) + 0.7          # nonzero mean: the std must subtract it
    u_hat = u + 1e-3 * rng.standard_normal(500)
    d = u_hat - u
    sums = np.array([np.sum(d * d), np.sum(u * u), np.sum(np.abs(d)), np.sum(u)])
    got = errors_from_sums(sums, len(u))
    ref = oracle.errors(u_hat, u)
    assert got["rel_l2"] == pytest.approx(ref["rel_l2"], rel=1e-12)
    assert got["e_l1"] == pytest.approx(ref["e_l1"], rel=1e-12)
