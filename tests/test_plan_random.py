"""Randomised host-side checks of the library's layout logic (no GPU): for
seeded random problem descriptions (1D, 2D, (2+1)D heat; boxes other than the
unit cube; overlap ratios that put grid points exactly on window edges), the
library's row counts per block, system sizes and QR launch order against the
oracle's row sets I_j = {r : w_j(x_r) > 0}, and rejection (not a crash) where
a subdomain has no collocation point."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def native():
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import _native
    return _native


def _random_problem(rng):
    dim = int(rng.integers(1, 4))
    heat = dim >= 2 and rng.random() < 0.4
    S = [int(rng.integers(2, 7)) for _ in range(dim)]
    # "nice" overlap ratios and grids put points exactly on window edges
    delta = float(rng.choice([1.0, 1.5, 2.0, 2.9])) if rng.random() < 0.5 else float(rng.uniform(1.0, 3.0))
    n = [int(rng.integers(1, 5)) * (s - 1) if rng.random() < 0.5 else int(rng.integers(s, 7 * s)) for s in S]
    lo = [float(rng.choice([0.0, -1.0, float(rng.uniform(-1, 1))])) for _ in range(3)]
    hi = [l + float(rng.choice([1.0, 2.0, float(rng.uniform(0.3, 2.0))])) for l in lo]
    K = int(rng.integers(1, 40))
    if heat:
        return synth.Problem(dim=dim, pde=synth.PDE_HEAT, S=S, delta=delta, K=K, n=n,
                             family=synth.FAM_HEAT_SINPROD, coef=[1.0], waves=[[1.0] * (dim - 1)], kappa=0.01,
                             lo=lo, hi=hi)
    return synth.Problem(dim=dim, pde=synth.PDE_POISSON, S=S, delta=delta, K=K, n=n, family=synth.FAM_SINPROD,
                         coef=[1.0], waves=[[1.0] * dim], lo=lo, hi=hi)


def _sizes(native, probs):
    arr = (native.RfmProblem * len(probs))(*[native.problem_struct(p) for p in probs])
    cfg = native.RfmConfig(native.ASM["fp64"], native.OPS["ar64"], 1e-10)
    sz = native.RfmSizes()
    rc = native.load().rfm_problem_size(arr, len(probs), C.byref(cfg), C.byref(sz))
    return rc, sz, arr, cfg


@pytest.mark.parametrize("seed", range(6))
def test_random_layouts_match_oracle_row_sets(native, seed):
    rng = np.random.default_rng(1000 + seed)
    L = native.load()
    checked = rejected = 0
    for _ in range(12):
        p = _random_problem(rng)
        rows = [len(oracle.block_rows(p, j)) for j in range(p.J)]
        rc, sz, arr, cfg = _sizes(native, [p])
        if min(rows) == 0:
            # a subdomain without collocation points is an invalid description
            assert rc == native.RFM_EINVAL and len(L.rfm_last_error()) > 0
            rejected += 1
            continue
        assert rc == native.RFM_OK, L.rfm_last_error()
        z = oracle.sizes(p)
        assert (sz.n_rows, sz.n_blocks, sz.n_cols) == (z["N"], p.J, p.J * p.K)
        assert sz.max_block_rows == max(rows)
        assert sz.block_rows == sum((r + 31) // 32 * 32 for r in rows)
        m, ld, moff, roff = (np.zeros(p.J, dtype=np.int64) for _ in range(4))
        assert L.rfm_block_table(arr, 1, C.byref(cfg), *[a.ctypes.data_as(C.c_void_p) for a in (m, ld, moff, roff)]) \
            == native.RFM_OK
        assert m.tolist() == rows
        assert np.all(ld % 32 == 0) and np.all(ld >= m)
        assert np.array_equal(roff, np.concatenate([[0], np.cumsum(ld)[:-1]]))
        assert np.array_equal(moff, roff * p.K)
        checked += 1
    assert checked > 0


def test_random_batches_order_and_sum(native):
    """Several random instances in one system: sizes add up and the QR launch
    order is the largest-first permutation of all blocks."""
    rng = np.random.default_rng(7)
    probs = []
    while len(probs) < 5:
        p = _random_problem(rng)
        if min(len(oracle.block_rows(p, j)) for j in range(p.J)) > 0:
            probs.append(p)
    rc, sz, arr, cfg = _sizes(native, probs)
    assert rc == native.RFM_OK
    assert sz.n_blocks == sum(p.J for p in probs)
    assert sz.n_rows == sum(oracle.sizes(p)["N"] for p in probs)
    order = np.zeros(sz.n_blocks, dtype=np.int32)
    assert native.load().rfm_qr_order(arr, len(probs), C.byref(cfg), order.ctypes.data_as(C.c_void_p)) == 0
    work = np.array([len(oracle.block_rows(p, j)) * p.K * min(len(oracle.block_rows(p, j)), p.K)
                     for p in probs for j in range(p.J)], dtype=np.float64)
    assert order.tolist() == sorted(range(len(work)), key=lambda b: (-work[b], b))
