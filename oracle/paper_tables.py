"""The condition numbers and drop shares of Tables 1 and 2 (Sec. 4.3-4.4),
recomputed with the oracle on the paper's own problems: the damped
oscillator (omega0 = 60, J = 20, delta = 2.9, K = 8) and the multi-scale
Laplace problem (n = 3, S = 16, delta = 2.9, K = 16, hard constraint).

TEST INFRASTRUCTURE: computes with oracle/ only (dense SVDs of the oracle's
assembled matrices, the oracle's filter and LSQR), and writes
tests/golden/paper_tables.json, which the CPU tests and the design notes
read.  The paper's seeds are not published, so its numbers pin orders of
magnitude and trends, not values.

    python -m oracle.paper_tables [--out tests/golden/paper_tables.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SIGMAS = (1e-10, 1e-8, 1e-6, 1e-4, 1e-2)


def kappa(A: np.ndarray) -> float:
    s = np.linalg.svd(A, compute_uv=False)
    return float(s[0] / s[-1])


def table(p, sigmas=SIGMAS, iters=10000, every=100):
    """kappa(M), and per threshold the drop share, kappa(M_hat),
    kappa(M_hat S^-1) (= kappa of the explicit Q_hat blocks, Prop. 3.1) and
    the smallest e_L1 and relative L2 errors over LSQR iterations recorded
    every `every` (the paper reports the minimum over its 10,000)."""
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    M, _ = oracle.assemble_dense(p, prm)
    X = oracle.test_grid(p)
    ue = oracle.exact(p, X)
    out = {"problem": p.name, "rows": int(M.shape[0]), "columns": int(M.shape[1]), "kappa_M": kappa(M), "runs": []}
    for sg in sigmas:
        F = oracle.filter_blocks(B, sg)
        cols, c = [], 0
        Q = np.zeros((B.N, sum(f.rank for f in F)))
        for j, f in enumerate(F):
            cols += [j * p.K + int(q) for q in f.perm[:f.rank]]
            Q[B.grow[j], c:c + f.rank] = f.Q()
            c += f.rank
        S = oracle.build_system(B, F, mode=0)
        best = {"e_l1": np.inf, "rel_l2": np.inf}
        # LSQR from zero run to each checkpoint (the iterate after k steps)
        for k in range(every, iters + 1, every):
            r = S.lsqr(B.h, atol=0, btol=0, max_iter=k)
            e = oracle.errors(oracle.evaluate(p, prm, S.coefficients(r["y"]), X), ue)
            for key in best:
                best[key] = min(best[key], e[key])
        out["runs"].append({"sigma": sg, "drop_pct": 100.0 * (1 - len(cols) / M.shape[1]),
                            "kappa_Mhat": kappa(M[:, cols]), "kappa_MhatSinv": kappa(Q),
                            "min_e_l1": float(best["e_l1"]), "min_rel_l2": float(best["rel_l2"])})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "paper_tables.json"))
    ap.add_argument("--iters", type=int, default=10000)
    ap.add_argument("--every", type=int, default=500)
    a = ap.parse_args(argv)
    res = {"oscillator": table(synth.oscillator(), iters=a.iters, every=a.every),
           "laplace": table(synth.laplace_multiscale(), iters=a.iters, every=a.every)}
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
