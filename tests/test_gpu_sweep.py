"""Threshold sweep on the GPU (plain LSQR and the filtered, preconditioned
solver at several thresholds) against the oracle on a small 1D problem: the
share of columns each threshold drops, and the errors of the iterate after a
fixed number of iterations."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_sweep_matches_oracle():
    import torch
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300.sweep import grid_points, sweep

    p = synth.poisson1d(S=6, K=24, n=240, n_test=300)
    prm = synth.feature_params(p)
    dev = torch.device("cuda:0")
    X = grid_points(p)
    sigmas = (1e-8, 1e-4, 1e-2)
    iters, every = 400, 100
    runs = sweep(p, torch.from_numpy(prm.ravel()).to(dev), torch.from_numpy(X).to(dev), op="ar64",
                 sigmas=sigmas, iters=iters, every=every, device=dev)
    assert [r["op"] for r in runs] == ["plain", "ar64", "ar64", "ar64"]
    assert runs[0]["dropped_pct"] == 0.0 and runs[0]["kept"] == p.J * p.K
    B = oracle.assemble(p, prm)
    u = oracle.exact(p, X)
    drops = []
    for r, s in zip(runs[1:], sigmas):
        F = oracle.filter_blocks(B, s)
        assert r["kept"] == sum(f.rank for f in F), s
        drops.append(r["dropped_pct"])
        if s >= 1e-4:
            # the iterate after `iters` steps, on the oracle
            ref = oracle.solve(p, prm, tol=s, atol=0.0, btol=0.0, max_iter=iters)
            e = oracle.errors(oracle.evaluate(p, prm, ref["a"], X), u)
            assert r["rel_l2_at_end"] == pytest.approx(e["rel_l2"], rel=1e-2), s
        assert np.isfinite(r["min_rel_l2"]) and np.isfinite(r["min_e_l1"])
        assert r["min_rel_l2"] <= r["rel_l2_at_end"]
        assert r["filter_ms"] > 0 and r["lsqr_ms"] > 0
    assert drops == sorted(drops)                 # a larger threshold drops at least as much
