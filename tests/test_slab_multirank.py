"""The slab-partitioned LSQR (paper_2506_17626_gb300.slab) on two and three
gloo ranks on CPU, against the single-process oracle.

The partition comes from the library's host-only row sets (rfm_block_rows,
checked here against the oracle's I_j of Eq. (6)); every rank owns a slab of
subdomains, and its local products are the oracle's operator A S^-1
(Sec. 3.2) restricted to the rank's blocks.  After k iterations the ranks'
y, gathered, equals the oracle's single-process LSQR iterate, and every rank
holds the same residual estimate: the halo exchanges (partial row sums to the
owners, u back to the other ranks) and the two scalar all-reduces per
iteration reproduce the undistributed recurrence up to the order of the sums.

That order is the only difference, and LSQR amplifies it by the conditioning
of the filtered operator: the first update u~ = A v - alpha u cancels to the
scale of 1/kappa.  With the loose threshold (1e-2, kappa of a few tens) the
distributed and single-process iterates agree to 1e-12; with 1e-6 they agree
to 1e-8 (measured 1e-10 on one rank, where only the sums' order differs),
the FP64 parity bound used for LSQR iterates elsewhere.  A wrong exchange or
a missing halo row moves y by O(1).
"""
from __future__ import annotations

import os
import pickle
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K_ITERS = 10
BOUND = {1e-2: 1e-12, 1e-6: 1e-8}       # relative y bound per filter threshold


def _problem():
    import synth
    return synth.poisson2d(S=5, K=12, n=30, delta=1.6)


def _rank_main(rank, world, tol, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_2506_17626_gb300 import slab

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem()
        prm = synth.feature_params(p)
        rows = slab.block_rows([p])
        plan = slab.plan_slabs(p, rows, world)[rank]
        B = oracle.assemble(p, prm, blocks=list(plan.blocks))
        F = oracle.filter_blocks(B, tol)
        So = oracle.build_system(B, F, mode=0)            # A S^-1 on the rank's blocks, rows global

        def apply(v):
            full = So.matvec(v.numpy())
            return torch.from_numpy(full[plan.touched])

        def apply_t(u):
            full = np.zeros(B.N)
            full[plan.touched] = u.numpy()
            return torch.from_numpy(So.rmatvec(full))

        solver = slab.SlabLsqr(plan, apply, apply_t, So.n)
        h = torch.from_numpy(B.h[plan.touched])
        y, est = solver.solve(h, K_ITERS)
        got = [None] * world
        dist.all_gather_object(got, {"rank": rank, "blocks": plan.blocks, "ranks": [f.rank for f in F],
                                     "y": y.numpy(), "rnorm": est["rnorm"], "owned": plan.owned})
        if rank == 0:
            with open(out_path, "wb") as f:
                pickle.dump(got, f)
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_block_rows_are_the_oracles_row_sets():
    import oracle
    import synth
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import slab
    for p in (_problem(), synth.heat3d(S=3, K=4, n=7), synth.oscillator(S=5, K=4)):
        rows = slab.block_rows([p])
        for j in range(p.J):
            assert np.array_equal(rows[j], oracle.block_rows(p, j)), (p.name, j)


def test_slab_plan_covers_rows_once():
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import slab
    p = _problem()
    rows = slab.block_rows([p])
    for world in (2, 3):
        plans = slab.plan_slabs(p, rows, world)
        owned = np.sort(np.concatenate([q.owned for q in plans]))
        assert np.array_equal(owned, np.unique(np.concatenate(rows)))     # every row owned exactly once
        assert sorted(np.concatenate([q.blocks for q in plans]).tolist()) == list(range(p.J))
        for q in plans:
            for r in q.send:
                # what q sends to r is exactly what r expects from q, row for row
                assert np.array_equal(q.touched[q.send[r]], plans[r].touched[plans[r].recv[q.rank]])


@pytest.mark.parametrize("tol", sorted(BOUND))
@pytest.mark.parametrize("world", [2, 3])
def test_slab_lsqr_matches_single_process_oracle(tmp_path, world, tol):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    import synth
    from paper_2506_17626_gb300 import build
    build.build()
    oracle.build()
    out = str(tmp_path / "slab.pkl")
    mp.spawn(_rank_main, args=(world, tol, _free_port(), out), nprocs=world, join=True)
    with open(out, "rb") as f:
        got = pickle.load(f)
    p = _problem()
    prm = synth.feature_params(p)
    B = oracle.assemble(p, prm)
    F = oracle.filter_blocks(B, tol)
    ref = oracle.build_system(B, F, mode=0).lsqr(B.h, atol=0, btol=0, max_iter=K_ITERS)
    # the ranks' columns in block order give the single-process y layout
    y = np.zeros(sum(f.rank for f in F))
    off = np.concatenate([[0], np.cumsum([f.rank for f in F])])
    for g in got:
        c = 0
        for b, r in zip(g["blocks"], g["ranks"]):
            assert r == F[b].rank
            y[off[b]:off[b] + r] = g["y"][c:c + r]
            c += r
    assert np.linalg.norm(y - ref["y"]) <= BOUND[tol] * np.linalg.norm(ref["y"])
    for g in got:
        assert g["rnorm"] == pytest.approx(ref["rnorm"], rel=BOUND[tol])
