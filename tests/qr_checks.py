"""Checks of a QR with column pivoting and relative-threshold drop (Algorithm
1) that hold for every valid pivot sequence.  Where two columns' trailing
norms tie to within the norms' rounding, correct implementations may take
different pivots from there on and keep different (equally valid) column
sets; these checks then replace the comparison with the oracle's kept set.

For a full column order perm (kept columns first) let R be the Householder R
factor of M[:, perm] without pivoting (numpy, LAPACK's sign convention).
After k steps the trailing norm of column j is ||R[k:, j]||, so:
  greedy    every kept pivot k is the largest remaining column up to a
            relative slack: |R_kk| >= (1 - slack) max_{j >= k} ||R[k:, j]||;
  threshold every kept pivot passes, |R_kk| >= tol |R_11| (1 - w), and
            after the last one no remaining column does,
            max_{j >= r} ||R[r:, j]|| < tol |R_11| (1 + w) (1 + slack).
"""
import numpy as np


def trailing_norms(R):
    """T[k, j] = ||R[k:, j]|| for the n x n (or min(m, n) x n) factor R."""
    sq = np.cumsum((R * R)[::-1], axis=0)[::-1]
    return np.sqrt(sq)


def check_pivoted_qr(M, perm, rank, tol, slack=1e-5, w=0.0):
    """Assert the greedy and threshold properties of the pivot order perm
    (all columns, kept first) with rank kept columns; returns R of M[:, perm]."""
    m, n = M.shape
    perm = np.asarray(perm, dtype=np.int64)
    R = np.linalg.qr(M[:, perm], mode="r")
    T = trailing_norms(R)
    r11 = abs(R[0, 0])
    steps = min(m, n)
    for k in range(rank):
        best = T[k, k:].max()
        assert abs(R[k, k]) >= (1 - slack) * best, (k, abs(R[k, k]), best)
        assert abs(R[k, k]) >= tol * r11 * (1 - w), (k, abs(R[k, k]) / r11)
    if rank < steps:
        assert T[rank, rank:].max() < tol * r11 * (1 + w) * (1 + slack), (rank, T[rank, rank:].max() / r11)
    return R


def signs(Rg, Rref):
    """Per-row sign that aligns the diagonal of Rg with that of Rref (beta_k
    takes the sign opposite to the pivot column's leading entry, rounding
    noise for a column near the threshold)."""
    d = np.sign(np.diag(Rg)) * np.sign(np.diag(Rref))
    d[d == 0] = 1.0
    return d
