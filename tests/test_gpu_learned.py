"""The learned warm start end to end on the GPU: solutions of a parametric
source family generated by the solver, the network trained on them by the
library's kernels (targets brought to a common scale by the family's
amplitude pi^2 (a^2 + b^2)), and LSQR started from the fitted prediction.

What the test asserts: the training lowers the loss; the fitted prediction
for solved instances starts far inside the zero start's error (which is 1 by
definition); the solver keeps that start (its residual is below ||h||, the
rule that otherwise falls back to zero) and LSQR from it runs.  What it reports: the error trajectories
from both starts.  On these 2D systems the measured gain does not survive
the first LSQR iterations (the preconditioned unknowns map to function values
through a badly conditioned evaluation, so the residual-driven iterations
move the iterate in function space from either start); the benchmark records
the same measurement on held-out instances.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rfm():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    return R


BASE = dict(S=10, K=120, delta=2.9, n=110)


def _family(seeds):
    return [synth.param5(*synth.param5_draw(s), **BASE) for s in seeds]


def _ctx(problems):
    return torch.from_numpy(np.stack([synth.param5_context(p.fparams) for p in problems])).cuda()


def _scale(problems):
    return [synth.param5_amplitude_scale(p.fparams) for p in problems]


def _params(problems):
    prm = synth.feature_params(problems[0])        # same decomposition and features for the family
    return torch.from_numpy(np.tile(prm.ravel(), len(problems))).cuda()


def _grid(nt=60):
    ax = (np.arange(nt) + 0.5) / nt
    X, Y = np.meshgrid(ax, ax, indexing="xy")
    return torch.from_numpy(np.stack([X.ravel(), Y.ravel()], 1)).cuda()


def _rel(u, r):
    return max(float(torch.linalg.norm(ui - ri) / torch.linalg.norm(ri)) for ui, ri in zip(u, r))


def test_learned_warm_start_end_to_end(rfm):
    from paper_2506_17626_gb300.warm import LearnedWarmStart
    train = _family(range(32))
    Xs, Ts = [], []
    first = None
    for i in range(0, len(train), 16):
        ps = train[i:i + 16]
        S = rfm.System(ps, asm="fp32", op="q32", tol=1e-6)
        d = _params(ps)
        S.assemble(d)
        S.filter()
        a, _ = S.solve(atol=0, btol=0, max_iter=3000)
        X, T = LearnedWarmStart.samples(S, d, a, _ctx(ps), inst_scale=_scale(ps))
        Xs.append(X)
        Ts.append(T)
        if first is None:
            first = (S, d, a)
    X, T = torch.cat(Xs), torch.cat(Ts)
    assert X.shape[1] == 9 and X.shape[0] == T.shape[0]
    W = LearnedWarmStart([9, 128, 128, 128, 128, 1], seed=0)
    scale = float(T.abs().max())
    hist = W.train(X, T / scale, epochs=60, batch=4096, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < 0.2 * hist[0]
    W.theta[-129:] *= scale      # output layer (W_L, b_L) in the targets' units

    # two of the solved instances; the reference is their own 3000-iteration solve
    S16, d16, a16 = first
    u16, _ = S16.evaluate(d16, a16, [_grid() for _ in range(16)], with_error=False)
    u_ref = u16[:2]
    ps = train[:2]
    d = _params(ps)
    S = rfm.System(ps, asm="fp32", op="q32", tol=1e-6)
    S.assemble(d)
    S.filter()
    S.fit_prepare(d, tol_fit=1e-8)
    Xt = [_grid() for _ in ps]
    inv = torch.tensor([1.0 / v for v in _scale(ps)], dtype=torch.float32, device="cuda")
    y0 = W.warm_start(S, _ctx(ps), fit_iters=300, inst_scale=inv)
    u0, _ = S.evaluate(d, S.coefficients(y0), Xt, with_error=False)
    e0 = _rel(u0, u_ref)

    def errs(y0=None, every=100, iters=1000):
        snap = torch.zeros((iters // every, S.sizes["n_cols"]), dtype=torch.float64, device="cuda")
        _, rep = S.solve(atol=0, btol=0, max_iter=iters, snap=snap, snap_every=every, y0=y0)
        e = np.array([_rel(S.evaluate(d, S.coefficients(snap[k]), Xt, with_error=False)[0], u_ref)
                      for k in range(snap.shape[0])])
        return e, [rfm.report_dict(rep, i) for i in range(len(ps))]

    (cold, rc), (warm, rw) = errs(None), errs(y0)
    print(f"\nlearned warm start: error at the start {e0:.3e} (zero start 1); after 100/500/1000 LSQR "
          f"iterations: zero start {cold[0]:.2e}/{cold[4]:.2e}/{cold[-1]:.2e}, "
          f"learned start {warm[0]:.2e}/{warm[4]:.2e}/{warm[-1]:.2e}")
    assert e0 < 0.5
    assert np.all(np.isfinite(warm))
    # the solver keeps the fitted start (its residual is below ||h||) and
    # reports it; the zero start reports no start
    assert all(r["start"] == 1 and r["r0norm"] < r["bnorm"] for r in rw)
    assert all(r["start"] == 0 and r["r0norm"] == r["bnorm"] for r in rc)
