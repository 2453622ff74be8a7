"""Threshold sweep of the local filter against plain LSQR, on the GPU through
the C ABI (the comparison of Sec. 4.3 and Table 1: share of columns dropped,
error, convergence of LSQR with and without the filter and preconditioner).

    python -m paper_2506_17626_gb300.sweep [--case p1d|p2d|osc|laplace] [--iters 10000] [--every 100]

Runs, on one problem instance, zero-start LSQR for a fixed number of
iterations with no stopping rule (as the paper runs its solvers), once on the
unfiltered, unpreconditioned system M (plain LSQR) and once per threshold
sigma of Algorithm 1 on M_hat S^-1.  The iterate is recorded every `every`
iterations and evaluated on the test grid.  Per run it reports the share of
columns dropped, the smallest relative L2 and e_L1 errors over the recorded
iterates (the paper reports the minimum over all iterations) and where they
occur, the first recorded iteration within twice the run's smallest relative
L2 error ("converged"), the first recorded iteration at or below each of a
few fixed errors, and the device time of the filter and of the LSQR run
(CUDA events; the LSQR time includes the iterate copies).  One JSON line.

Workloads: p1d is 1D Poisson -u'' = f on [0,1], u = sin 2 pi x + 0.1 sin 50 pi
x, 20 subdomains, overlap ratio 1.3, 100 features, 1600 interior points,
FP64 throughout; p2d is the 2D Poisson workload of the benchmark (20 x 20
subdomains, overlap ratio 1.25, 300 features, 360^2 interior points), FP64
assembly with the explicit FP64 Q_hat operator; osc and laplace are the
paper's own baselines (Sec. 4.3 and 4.4: the damped oscillator with omega0 =
60, J = 20, overlap ratio 2.9, K = 8; the multi-scale Laplace problem with
n = 3, 16 x 16 subdomains, overlap ratio 2.9, K = 16 and the hard-constraint
ansatz), FP64 with the paper's operator form (R_hat^-1 substitution), with
--depth and --act for the network ablations of Tables 1 and 2.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from .api import System

SIGMAS = (1e-10, 1e-8, 1e-6, 1e-4, 1e-2)
LADDER = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)


def grid_points(p) -> np.ndarray:
    """Cell-centred grid of p.n_test points per dimension (dimension 0
    fastest), n x dim."""
    axes = [p.lo[i] + (np.arange(p.n_test[i]) + 0.5) * (p.hi[i] - p.lo[i]) / p.n_test[i] for i in range(p.dim)]
    g = np.meshgrid(*axes[::-1], indexing="ij")
    return np.ascontiguousarray(np.stack([a.ravel() for a in g[::-1]], axis=1))


def errors_from_sums(e: np.ndarray, n_pts: int) -> Dict[str, float]:
    """Relative L2 and the normalised L1 error e_L1 of Sec. 4.2 (mean |u_hat -
    u| over the standard deviation of u) from the evaluation's four sums
    (sum (u_hat-u)^2, sum u^2, sum |u_hat-u|, sum u)."""
    mean = e[3] / n_pts
    std = math.sqrt(max(e[1] / n_pts - mean * mean, 0.0))
    return {"rel_l2": math.sqrt(e[0] / e[1]), "e_l1": (e[2] / n_pts) / std}


def run_one(p, params: torch.Tensor, X: torch.Tensor, asm: str, op: str, sigma: float, iters: int, every: int,
            device) -> dict:
    """One zero-start LSQR run of `iters` iterations; errors of the iterate
    every `every` iterations."""
    S = System([p], asm=asm, op=op, tol=sigma, device=str(device))
    S.assemble(params)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    rank = S.filter()
    ev[1].record()
    cap = iters // every
    snap = torch.zeros((cap, S.sizes["n_cols"]), dtype=torch.float64, device=device)
    S.solve(atol=0.0, btol=0.0, max_iter=iters, snap=snap, snap_every=every)
    ev[2].record()
    torch.cuda.synchronize()
    n_cols = S.sizes["n_cols"]
    kept = n_cols if rank is None else int(rank.sum().item())
    rel, el1 = [], []
    for s in range(cap):
        a = S.coefficients(snap[s])
        _, err = S.evaluate(params, a, [X])
        e = errors_from_sums(err.cpu().numpy(), X.shape[0])
        rel.append(e["rel_l2"])
        el1.append(e["e_l1"])
    rel, el1 = np.array(rel), np.array(el1)
    at = [every * (s + 1) for s in range(cap)]
    best = int(np.argmin(rel))
    conv = int(np.argmax(rel <= 2.0 * rel[best]))
    reach = {f"{t:g}": (at[int(np.argmax(rel <= t))] if (rel <= t).any() else None) for t in LADDER}
    return {"op": op, "sigma": None if op == "plain" else sigma, "columns": n_cols, "kept": kept,
            "dropped_pct": 100.0 * (n_cols - kept) / n_cols,
            "min_rel_l2": float(rel[best]), "min_rel_l2_at": at[best],
            "min_e_l1": float(el1.min()), "min_e_l1_at": at[int(np.argmin(el1))],
            "converged_at": at[conv], "iterations_to": reach,
            "rel_l2_at_end": float(rel[-1]),
            "filter_ms": ev[0].elapsed_time(ev[1]), "lsqr_ms": ev[1].elapsed_time(ev[2])}


def sweep(p, params: torch.Tensor, X: torch.Tensor, asm: str = "fp64", op: str = "ar64",
          sigmas: Sequence[float] = SIGMAS, iters: int = 10000, every: int = 100, device="cuda:0") -> List[dict]:
    """Plain LSQR, then one run per threshold."""
    runs = [run_one(p, params, X, asm, "plain", 0.0, iters, every, device)]
    for s in sigmas:
        runs.append(run_one(p, params, X, asm, op, s, iters, every, device))
    return runs


def main(argv: Optional[Sequence[str]] = None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="p1d", choices=["p1d", "p2d", "osc", "laplace"])
    ap.add_argument("--depth", type=int, default=1, help="osc, laplace: depth h of the subdomain networks")
    ap.add_argument("--act", default="tanh", choices=["tanh", "sigmoid", "sin"],
                    help="osc, laplace: activation of the subdomain networks")
    ap.add_argument("--iters", type=int, default=10000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--op", default=None, choices=["ar64", "q64"],
                    help="operator of the filtered runs (default: ar64 for p1d, q64 for p2d)")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth
    dev = torch.device("cuda:0")
    act = {"tanh": synth.ACT_TANH, "sigmoid": synth.ACT_SIGMOID, "sin": synth.ACT_SIN}[args.act]
    if args.case == "p1d":
        p = synth.poisson1d()
        op = args.op or "ar64"
    elif args.case == "osc":
        p = synth.oscillator(act=act, depth=args.depth)
        op = args.op or "ar64"
    elif args.case == "laplace":
        p = synth.laplace_multiscale(act=act, depth=args.depth)
        op = args.op or "ar64"
    else:
        p = synth.poisson2d()
        op = args.op or "q64"
    prm = torch.from_numpy(synth.feature_params(p).ravel()).to(dev)
    X = torch.from_numpy(grid_points(p)).to(dev)
    runs = sweep(p, prm, X, asm="fp64", op=op, iters=args.iters, every=args.every, device=dev)
    print(json.dumps({"workload": p.name, "iterations": args.iters, "record_every": args.every,
                      "test_points": int(X.shape[0]), "runs": runs}), flush=True)


if __name__ == "__main__":
    main()
