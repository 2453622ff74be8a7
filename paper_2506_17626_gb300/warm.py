"""Learned warm start: training data from solves, network training, and the
prediction turned into an LSQR starting point.

The network, its gradient and Adam, the network inputs at the block rows, the
local fit and the solves all run in the library's kernels (include/rfm.h);
this module strings the calls together and does the bookkeeping of sample
selection and minibatch order with torch index operations.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from .api import Mlp, System


def block_row_mask(S: System) -> torch.Tensor:
    """Indices of the live rows (not padding) of the block-row layout."""
    m, ld, _, roff = S.block_table()
    idx = [np.arange(r, r + k, dtype=np.int64) for k, r in zip(m, roff)]
    return torch.from_numpy(np.concatenate(idx)).to(S.device)


def instance_row_ranges(S: System) -> List[tuple]:
    """(first, end) of each instance's rows in the block-row layout."""
    _, ld, _, roff = S.block_table()
    out = []
    b0 = 0
    for p in S.problems:
        J = int(np.prod([int(x) for x in p.S[: p.dim]]))
        out.append((int(roff[b0]), int(roff[b0 + J - 1] + ld[b0 + J - 1])))
        b0 += J
    return out


class LearnedWarmStart:
    """Network over [instance context, block centre, local coordinates] that
    predicts the solution at every block row; its predictions become y0 through
    System.warm_start (the local fit through each block's kept features)."""

    def __init__(self, widths: Sequence[int], seed: int = 0, device: str = "cuda"):
        self.net = Mlp(widths, device=device)
        self.widths = list(widths)
        self.device = torch.device(device)
        # LeCun-uniform weights, zero biases (drawn on the host from a seeded
        # generator, then moved to the device)
        g = np.random.default_rng(seed)
        parts = []
        for l in range(1, len(widths)):
            fan_in, fan_out = widths[l - 1], widths[l]
            lim = math.sqrt(3.0 / fan_in)
            parts.append(g.uniform(-lim, lim, fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        self.theta = torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(self.device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.step = 0

    # -- data ------------------------------------------------------------------------
    @staticmethod
    def samples(S: System, params: torch.Tensor, a: torch.Tensor, ctx: torch.Tensor,
                inst_scale: Optional[Sequence[float]] = None):
        """Training pairs from a solved system: network inputs at every live
        block row and the solution u_hat(a) at the row's point, multiplied by
        the instance's scale when given (targets on a common scale)."""
        X, pts = S.block_inputs(ctx)
        ranges = instance_row_ranges(S)
        dim = S.problems[0].dim
        P = [pts[r0:r1, :dim].contiguous() for r0, r1 in ranges]
        u, _ = S.evaluate(params, a, P, with_error=False)
        if inst_scale is not None:
            u = [ui * float(s) for ui, s in zip(u, inst_scale)]
        T = torch.cat(u).to(torch.float32)
        live = block_row_mask(S)
        return X.index_select(0, live).contiguous(), T.index_select(0, live).contiguous()

    # -- training ----------------------------------------------------------------------
    def train(self, X: torch.Tensor, T: torch.Tensor, epochs: int = 1, batch: int = 4096, lr: float = 1e-3,
              seed: int = 0, lr_final: Optional[float] = None) -> List[float]:
        """Adam on minibatches (reshuffled every epoch); returns the mean loss
        of every epoch.  With lr_final the rate decays geometrically to it."""
        n = X.shape[0]
        batch = min(batch, n)
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        hist = []
        nb = max(1, n // batch)
        total = epochs * nb
        losses = torch.zeros(nb, dtype=torch.float32, device=self.device)
        for e in range(epochs):
            perm = torch.randperm(n, generator=gen, device=self.device)
            rates = [lr if lr_final is None else lr * (lr_final / lr) ** ((e * nb + b) / max(1, total - 1))
                     for b in range(nb)]
            # one library call per epoch: gather, gradient and Adam for every batch
            self.net.train_steps(self.theta, self.m, self.v, X, T, perm, batch, self.step + 1, rates, loss=losses)
            self.step += nb
            hist.append(float(losses.sum().item()) / nb)
        return hist

    # -- use -----------------------------------------------------------------------------
    def predict(self, S: System, ctx: torch.Tensor) -> torch.Tensor:
        """Predictions at every block row (padding rows included, ignored by the fit)."""
        X, _ = S.block_inputs(ctx, want_points=False)
        return self.net.forward(self.theta, X)

    def warm_start(self, S: System, ctx: torch.Tensor, fit_iters: int = 100,
                   inst_scale: Optional[torch.Tensor] = None) -> torch.Tensor:
        """y0 for S.solve (needs S.filter() and S.fit_prepare() first); the
        predictions are multiplied by inst_scale per instance (the inverse of
        the scale the training targets were brought to)."""
        return S.warm_start(self.predict(S, ctx), fit_iters=fit_iters, inst_scale=inst_scale)
