"""Host-side checks of the CUDA library (no GPU needed): it loads, exports every
symbol include/rfm.h declares, and its host-only layout logic agrees with the
oracle's row sets.  No compute call runs here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import _native
    return _native


def test_library_exports_every_declared_symbol(native):
    hdr = open(os.path.join(ROOT, "include", "rfm.h")).read()
    declared = set(re.findall(r"^\s*(?:rfm_status|const char \*|int)\s*(rfm_\w+)\s*\(", hdr, re.M))
    assert {"rfm_assemble", "rfm_rrqr_filter", "rfm_lsqr_solve", "rfm_eval"} <= declared
    lib = C.CDLL(native.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    L = native.load()
    assert L.rfm_abi_version() == 2


def _sizes(native, probs, asm="fp64", op="ar64", tol=1e-10):
    arr = (native.RfmProblem * len(probs))(*[native.problem_struct(p) for p in probs])
    cfg = native.RfmConfig(native.ASM[asm], native.OPS[op], tol)
    sz = native.RfmSizes()
    rc = native.load().rfm_problem_size(arr, len(probs), C.byref(cfg), C.byref(sz))
    return rc, sz, arr, cfg


@pytest.mark.parametrize("p", [synth.poisson1d(S=5, K=7, n=50), synth.poisson2d(S=4, K=5, n=13),
                               synth.heat3d(S=3, K=4, n=7), synth.poisson2d(S=5, K=3, n=11, delta=2.9),
                               synth.oscillator(S=5, K=4), synth.laplace_multiscale(S=3, K=4),
                               synth.laplace_multiscale(S=3, K=9, depth=3, act=synth.ACT_SIN)])
def test_block_row_counts_match_oracle(native, p):
    rc, sz, arr, cfg = _sizes(native, [p])
    assert rc == 0
    z = oracle.sizes(p)
    assert sz.n_rows == z["N"] and sz.n_blocks == z["J"] and sz.n_cols == z["J"] * p.K
    rows = [len(oracle.block_rows(p, j)) for j in range(p.J)]
    padded = [(r + 31) // 32 * 32 for r in rows]
    assert sz.block_rows == sum(padded) and sz.max_block_rows == max(rows)
    L = native.load()
    for j in range(p.J):
        m, ld, moff, roff = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        assert L.rfm_block_info(arr, 1, C.byref(cfg), j, C.byref(m), C.byref(ld), C.byref(moff), C.byref(roff)) == 0
        assert m.value == rows[j] and ld.value == padded[j]
        assert roff.value == sum(padded[:j])


def test_multi_instance_sizes_add_up(native):
    ps = [synth.poisson2d(S=4, K=5, n=13), synth.poisson1d(S=3, K=6, n=20)]
    rc, sz, _, _ = _sizes(native, ps)
    assert rc == 0
    one = [_sizes(native, [p])[1] for p in ps]
    for f in ("n_rows", "n_cols", "n_blocks", "block_rows"):
        assert getattr(sz, f) == sum(getattr(o, f) for o in one)


@pytest.mark.parametrize("field,value", [("dim", 4), ("K", 0), ("K", 5000), ("delta", -1.0), ("S", [1, 4, 1]),
                                         ("n", [0, 5, 1])])
def test_invalid_problems_are_rejected(native, field, value):
    p = synth.poisson2d(S=4, K=5, n=13)
    setattr(p, field, value)
    rc, sz, _, _ = _sizes(native, [p])
    assert rc == native.RFM_EINVAL
    assert len(native.load().rfm_last_error()) > 0


def test_invalid_config_is_rejected(native):
    p = synth.poisson2d(S=4, K=5, n=13)
    rc, *_ = _sizes(native, [p], tol=2.0)
    assert rc == native.RFM_EINVAL
    rc, *_ = _sizes(native, [p], tol=float("nan"))
    assert rc == native.RFM_EINVAL


def test_subdomain_without_points_is_rejected(native):
    # a grid too coarse for the decomposition leaves subdomains without rows
    p = synth.poisson1d(S=20, K=4, n=3)
    rc, *_ = _sizes(native, [p])
    assert rc == native.RFM_EINVAL


def test_qr_launch_order_is_largest_first(native):
    """The filter's QR launch order over an uneven batch: a permutation of the
    blocks, by decreasing m K min(m, K) with ties in block order, where m are
    the oracle's block row counts."""
    ps = [synth.batched_instance(i, p_range=(3, 5)) for i in range(3)] + [synth.poisson1d(S=5, K=7, n=50)]
    rc, sz, arr, cfg = _sizes(native, ps)
    assert rc == 0
    order = np.zeros(sz.n_blocks, dtype=np.int32)
    assert native.load().rfm_qr_order(arr, len(ps), C.byref(cfg), order.ctypes.data_as(C.c_void_p)) == 0
    assert np.array_equal(np.sort(order), np.arange(sz.n_blocks))
    work = []
    for p in ps:
        for j in range(p.J):
            m = len(oracle.block_rows(p, j))
            work.append(m * p.K * min(m, p.K))
    work = np.array(work, dtype=np.float64)
    expect = sorted(range(len(work)), key=lambda b: (-work[b], b))
    assert order.tolist() == expect
    assert len(set(work.tolist())) > 3           # the batch is uneven


def test_full_size_heat_workload_plans_on_the_host(native):
    """The (2+1)D heat workload at its full size (10^3 subdomains, K = 500,
    100^3 interior points plus the lateral and initial faces): the plan builds
    and its sizes agree with the oracle's row count."""
    p = synth.heat3d()
    rc, sz, _, _ = _sizes(native, [p], asm="fp32", op="q32", tol=1e-6)
    assert rc == 0, native.load().rfm_last_error()
    z = oracle.sizes(p)
    assert sz.n_rows == z["N"] == 100 ** 3 + 5 * 100 ** 2
    assert sz.n_blocks == 1000 and sz.n_cols == 1000 * 500 and sz.max_K == 500
    assert sz.max_block_rows == 2744
    assert sz.workspace_bytes < 32 * 2 ** 30
