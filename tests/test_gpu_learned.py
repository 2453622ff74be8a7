"""The learned warm start end to end on the GPU: solutions of a parametric
source family generated by the solver, the network trained on them by the
library's kernels, and LSQR on held-out instances started from the fitted
prediction against the same LSQR from zero.

The gain is measured, not pinned: the test asserts that the warm start begins
well inside the zero start's error (which is 1 by definition) and stays ahead
of it for a fixed iteration budget, with errors taken against a long zero-start
reference solve of the same system on the test grid.
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


BASE = dict(S=5, K=60, delta=2.9, n=40)


def _family(seeds):
    return [synth.param5(*synth.param5_draw(s), **BASE) for s in seeds]


def _ctx(problems):
    return torch.from_numpy(np.stack([synth.param5_context(p.fparams) for p in problems])).cuda()


def _scale(problems):
    return [synth.param5_amplitude_scale(p.fparams) for p in problems]


def _params(problems):
    prm = synth.feature_params(problems[0])        # same decomposition and features for the family
    return torch.from_numpy(np.tile(prm.ravel(), len(problems))).cuda()


def _grid(p, nt=40):
    ax = (np.arange(nt) + 0.5) / nt
    X, Y = np.meshgrid(ax, ax, indexing="xy")
    return torch.from_numpy(np.stack([X.ravel(), Y.ravel()], 1)).cuda()


def test_learned_warm_start_beats_zero_start(rfm):
    from paper_2506_17626_gb300.warm import LearnedWarmStart
    train = _family(range(128))
    Xs, Ts = [], []
    for i in range(0, len(train), 32):
        ps = train[i:i + 32]
        S = rfm.System(ps, asm="fp32", op="q32", tol=1e-6)
        d = _params(ps)
        S.assemble(d)
        S.filter()
        a, _ = S.solve(atol=0, btol=0, max_iter=3000)
        X, T = LearnedWarmStart.samples(S, d, a, _ctx(ps), inst_scale=_scale(ps))
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    assert X.shape[1] == 9 and X.shape[0] == T.shape[0]
    W = LearnedWarmStart([9, 128, 128, 128, 128, 1], seed=0)
    scale = float(T.abs().max())
    hist = W.train(X, T / scale, epochs=20, batch=4096, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < 0.2 * hist[0]
    W.theta[-129:] *= scale      # output layer (W_L, b_L) in the targets' units

    held = _family([10000, 10001])
    S = rfm.System(held, asm="fp32", op="q32", tol=1e-6)
    d = _params(held)
    S.assemble(d)
    S.filter()
    S.fit_prepare(d, tol_fit=1e-8)
    inv = torch.tensor([1.0 / v for v in _scale(held)], dtype=torch.float32, device="cuda")
    y0 = W.warm_start(S, _ctx(held), fit_iters=100, inst_scale=inv)
    Xt = [_grid(p) for p in held]
    # reference: a long zero-start FP64 solve of the same discretisation
    R64 = rfm.System(held, asm="fp64", op="q64", tol=1e-6)
    R64.assemble(d)
    R64.filter()
    a_ref, _ = R64.solve(atol=0, btol=0, max_iter=8000)
    u_ref, _ = R64.evaluate(d, a_ref, Xt, with_error=False)

    def errs(y0=None, every=50, iters=2000):
        snap = torch.zeros((iters // every, S.sizes["n_cols"]), dtype=torch.float64, device="cuda")
        S.solve(atol=0, btol=0, max_iter=iters, snap=snap, snap_every=every, y0=y0)
        out = []
        for k in range(snap.shape[0]):
            u, _ = S.evaluate(d, S.coefficients(snap[k]), Xt, with_error=False)
            out.append(max(float(torch.linalg.norm(ui - ri) / torch.linalg.norm(ri)) for ui, ri in zip(u, u_ref)))
        return np.array(out)

    u0, _ = S.evaluate(d, S.coefficients(y0), Xt, with_error=False)
    e0 = max(float(torch.linalg.norm(ui - ri) / torch.linalg.norm(ri)) for ui, ri in zip(u0, u_ref))
    cold, warm = errs(None), errs(y0)
    print(f"warm start error {e0:.3e}; error after 50/500/2000 iterations: cold "
          f"{cold[0]:.2e}/{cold[9]:.2e}/{cold[-1]:.2e} warm {warm[0]:.2e}/{warm[9]:.2e}/{warm[-1]:.2e}")
    # the fitted prediction starts inside the zero start's error (1) and
    # reaches the zero start's error after 500 iterations sooner
    assert e0 < 1.0
    k_cold = 9
    k_warm = int(np.argmax(warm <= cold[k_cold])) if (warm <= cold[k_cold]).any() else len(warm)
    assert k_warm < k_cold
