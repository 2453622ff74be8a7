"""Slab partition of one system over several processes, and LSQR (Paige and
Saunders 1982) on the partitioned operator of Algorithm 2.

Rank q owns the subdomains whose slowest index (the last dimension) lies in
its contiguous range, with their blocks (assembly and the local filter of
Algorithm 1 need nothing else) and the columns of those blocks.  A global row
is touched by every rank that owns a block covering it (the overlap of Eq. (6)
makes the rows near a slab boundary shared); its owner is the lowest such rank.
One LSQR iteration on rank q:

  t = sum over its blocks of Op_b v_b        partial row sums on its touched rows
  halo exchange 1: partial sums of shared rows go to their owners, who add them
  u~ = t - alpha u on the owned rows;  beta^2 = all-reduce of ||u~||^2
  halo exchange 2: owners send u = u~ / beta of shared rows to the other ranks
  z = sum over its blocks of Op_b^T u_b on its columns
  v~ = z - beta v;  alpha^2 = all-reduce of ||v~||^2
  the plane rotation on (alpha, beta) (the same on every rank), y and w updates

The two scalar all-reduces and the two exchanges are the only communication.
The rank-local products are supplied by the caller (`apply` and `apply_t` on
the rank's blocks), so the recurrence and the exchange pattern are the same
whatever computes them.  The row sets come from the library's host-only
rfm_block_rows.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Sequence

import numpy as np

from . import _native as N


def block_rows(problems: Sequence, asm: str = "fp64", op: str = "ar64", tol: float = 1e-10) -> List[np.ndarray]:
    """Global rows of every block (host-only library call per block)."""
    arr = (N.RfmProblem * len(problems))(*[N.problem_struct(p) for p in problems])
    cfg = N.RfmConfig(N.ASM[asm], N.OPS[op], float(tol))
    lib = N.load()
    tab = [np.zeros(0, dtype=np.int64)]
    m = np.zeros(sum(int(np.prod([int(s) for s in p.S[:p.dim]])) for p in problems), dtype=np.int64)
    N.check("rfm_block_table", lib.rfm_block_table(arr, len(problems), C.byref(cfg), m.ctypes.data_as(C.c_void_p),
                                                   None, None, None))
    out = []
    for b, mb in enumerate(m):
        rows = np.zeros(int(mb), dtype=np.int64)
        N.check("rfm_block_rows", lib.rfm_block_rows(arr, len(problems), C.byref(cfg), b,
                                                     rows.ctypes.data_as(C.c_void_p)))
        out.append(rows)
    del tab
    return out


@dataclass
class RankPlan:
    rank: int
    blocks: np.ndarray                    # global block indices owned by this rank
    touched: np.ndarray                   # sorted global rows touched by its blocks
    owned: np.ndarray                     # rows it owns (subset of touched)
    owned_pos: np.ndarray                 # positions of the owned rows within touched
    send: Dict[int, np.ndarray] = field(default_factory=dict)   # rank -> positions (in touched) of rows it owns
    recv: Dict[int, np.ndarray] = field(default_factory=dict)   # rank -> positions (in touched) of my owned rows it touches


def plan_slabs(problem, rows_of_block: Sequence[np.ndarray], world: int) -> List[RankPlan]:
    """Contiguous slabs of the slowest subdomain index, one per rank (sizes
    differ by at most one subdomain layer)."""
    S = [int(s) for s in problem.S[:problem.dim]]
    inner = int(np.prod(S[:-1])) if len(S) > 1 else 1
    J = int(np.prod(S))
    layer = np.arange(J) // inner
    rank_of_block = layer * world // S[-1]
    toucher = {}
    for b in range(J):
        for r in rows_of_block[b]:
            toucher.setdefault(int(r), set()).add(int(rank_of_block[b]))
    owner = {r: min(qs) for r, qs in toucher.items()}
    plans = []
    for q in range(world):
        blocks = np.nonzero(rank_of_block == q)[0]
        touched = np.unique(np.concatenate([rows_of_block[b] for b in blocks])) if len(blocks) else np.zeros(0, np.int64)
        pos = {int(r): i for i, r in enumerate(touched)}
        owned = np.array([r for r in touched if owner[int(r)] == q], dtype=np.int64)
        plan = RankPlan(q, blocks, touched, owned, np.array([pos[int(r)] for r in owned], dtype=np.int64))
        for p in range(world):
            if p == q:
                continue
            plan.send[p] = np.array([pos[int(r)] for r in touched if owner[int(r)] == p], dtype=np.int64)
            plan.recv[p] = np.array([pos[int(r)] for r in owned if p in toucher[int(r)]], dtype=np.int64)
        plans.append(plan)
    return plans


class SlabLsqr:
    """LSQR on one rank of the slab partition.  apply(v) returns the rank's
    partial row sums on plan.touched for its column vector v; apply_t(u)
    returns its column vector for u given on plan.touched.  Vectors are
    torch tensors (FP64) on the rank's device; the process group carries the
    exchanges and the all-reduces."""

    def __init__(self, plan: RankPlan, apply: Callable, apply_t: Callable, n_local_cols: int, group=None,
                 device="cpu"):
        import torch
        self.plan, self.apply, self.apply_t = plan, apply, apply_t
        self.n, self.group, self.device = n_local_cols, group, torch.device(device)
        self.owned_pos = torch.as_tensor(plan.owned_pos, device=self.device)
        self.send = {p: torch.as_tensor(v, device=self.device) for p, v in plan.send.items()}
        self.recv = {p: torch.as_tensor(v, device=self.device) for p, v in plan.recv.items()}

    def _allreduce(self, x: float) -> float:
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, group=self.group)
        return float(t.item())

    def _exchange(self, buf, outgoing, incoming, add: bool):
        """Send buf[outgoing[p]] to every rank p and receive into
        buf[incoming[p]] (added, or written), in rank order (no cycles)."""
        import torch
        import torch.distributed as dist
        reqs, got = [], {}
        for p, idx in outgoing.items():
            if len(idx):
                reqs.append(dist.isend(buf[idx].contiguous(), p, group=self.group))
        for p, idx in incoming.items():
            if len(idx):
                got[p] = torch.empty(len(idx), dtype=buf.dtype, device=buf.device)
                reqs.append(dist.irecv(got[p], p, group=self.group))
        for r in reqs:
            r.wait()
        for p in sorted(got):
            if add:
                buf[incoming[p]] += got[p]
            else:
                buf[incoming[p]] = got[p]

    def solve(self, h_touched, iters: int):
        """LSQR from zero for `iters` iterations; h on plan.touched (only the
        owned entries are used).  Returns the rank's y and the estimates."""
        import torch
        mask = torch.zeros(len(self.plan.touched), dtype=torch.bool, device=self.device)
        mask[self.owned_pos] = True
        u = torch.where(mask, h_touched, torch.zeros_like(h_touched))
        beta = np.sqrt(self._allreduce(float((u * u).sum())))
        u = u / beta if beta > 0 else u
        self._exchange(u, self.recv, self.send, add=False)        # owners -> touchers
        v = self.apply_t(u)
        alpha = np.sqrt(self._allreduce(float((v * v).sum())))
        v = v / alpha if alpha > 0 else v
        w = v.clone()
        y = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        phibar, rhobar = beta, alpha
        for _ in range(iters):
            t = self.apply(v)
            self._exchange(t, self.send, self.recv, add=True)     # partial sums -> owners
            u = torch.where(mask, t - alpha * u, torch.zeros_like(t))
            beta = np.sqrt(self._allreduce(float((u * u).sum())))
            if beta > 0:
                u = u / beta
            self._exchange(u, self.recv, self.send, add=False)
            v = self.apply_t(u) - beta * v
            alpha = np.sqrt(self._allreduce(float((v * v).sum())))
            if alpha > 0:
                v = v / alpha
            rho = np.sqrt(rhobar * rhobar + beta * beta)
            c, s = rhobar / rho, beta / rho
            theta = s * alpha
            rhobar = -c * alpha
            phi = c * phibar
            phibar = s * phibar
            y = y + (phi / rho) * w
            w = v - (theta / rho) * w
        return y, {"rnorm": phibar}
