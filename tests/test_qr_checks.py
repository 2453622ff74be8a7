"""The pivot-order checks used by the GPU QR tests, pinned on the CPU: the
oracle's own factorisations pass them, and orders with a planted mistake
(the smallest column taken first, one column too many or too few kept) fail."""
import numpy as np
import pytest

import oracle
import synth
from qr_checks import check_pivoted_qr

CASES = [lambda: synth.poisson2d(S=5, K=40, n=30), lambda: synth.poisson1d(S=6, K=24, n=150),
         lambda: synth.heat3d(S=3, K=30, n=9)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_checks_accept_the_oracle_and_reject_planted_mistakes(case):
    p = CASES[case]()
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    for j in range(p.J):
        M = B.M[j]
        f = oracle.qrcp(M, 1e-6)
        kept = set(f.perm[: f.rank])
        full = np.array(list(f.perm[: f.rank]) + [c for c in range(p.K) if c not in kept], dtype=np.int64)
        check_pivoted_qr(M, full, f.rank, 1e-6)
        smallest = int(np.argmin(np.linalg.norm(M, axis=0)))
        bad = full.copy()
        at = list(full).index(smallest)
        bad[[0, at]] = bad[[at, 0]]
        planted = [(bad, f.rank), (full, f.rank - 1)]
        if f.rank < min(M.shape):
            planted.append((full, f.rank + 1))
        for order, rank in planted:
            if rank < 0:
                continue
            with pytest.raises(AssertionError):
                check_pivoted_qr(M, order, rank, 1e-6)
