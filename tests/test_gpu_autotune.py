"""The QR cluster-size autotuner: with RFM_OPT_AUTOTUNE the first filter
call of a block shape times every feasible cluster size; the kept factors it
leaves (ranks, the pivot order of the kept columns, Q_hat) and those of
later calls with the cached choice are bitwise equal to the default choice's
(the per-column arithmetic does not depend on how the columns are spread
over the CTAs of a cluster; the order of the dropped columns does)."""
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


@pytest.mark.parametrize("asm,op", [("fp32", "q32"), ("fp64", "q64")])
def test_autotuned_filter_is_bitwise_the_default(rfm, asm, op):
    from paper_2506_17626_gb300 import _native as N
    p = synth.poisson2d(S=4, K=48, n=40, delta=1.6)
    prm = synth.feature_params(p)
    d = torch.from_numpy(prm.ravel()).cuda()

    def run():
        S = rfm.System([p], asm=asm, op=op, tol=1e-6)
        S.assemble(d)
        r, perm = S.filter(want_perm=True)
        rk = r.cpu().numpy()
        perm = perm.cpu().numpy()
        kept = np.concatenate([perm[j * p.K: j * p.K + rk[j]] for j in range(p.J)])
        Q = torch.cat([S.block_matrix(j, which=5)[:, : int(rk[j])].flatten() for j in range(p.J)])
        torch.cuda.synchronize()
        return rk, kept, Q.cpu().numpy()

    base = run()
    try:
        N.set_autotune(True)
        first = run()      # times the cluster sizes
        second = run()     # uses the cached choice
    finally:
        N.set_autotune(False)
    for got in (first, second):
        assert np.array_equal(got[0], base[0])
        assert np.array_equal(got[1], base[1])
        assert np.array_equal(got[2], base[2])


@pytest.mark.parametrize("asm,op", [("fp32", "q32"), ("fp64", "q64")])
def test_autotuned_global_kernels(rfm, asm, op):
    """Blocks on the global-memory kernels (forced): the tuner times 8, 16 and
    32 warps per block on the first call and leaves the chosen variant's
    factors, which later calls with the cached choice reproduce bitwise; the
    variants agree with the default (32 warps) to rounding (the pivot
    column's norm is summed over the CTA in another order): the same kept
    columns, Q_hat within 1e-12 (FP64) or 2e-7 (FP32 storage)."""
    from paper_2506_17626_gb300 import _native as N
    p = synth.poisson2d(S=4, K=48, n=40, delta=1.6)
    prm = synth.feature_params(p)
    d = torch.from_numpy(prm.ravel()).cuda()

    def run():
        S = rfm.System([p], asm=asm, op=op, tol=1e-6)
        S.assemble(d)
        r, perm = S.filter(want_perm=True)
        rk = r.cpu().numpy()
        perm = perm.cpu().numpy()
        kept = [perm[j * p.K: j * p.K + rk[j]].tolist() for j in range(p.J)]
        Q = torch.cat([S.block_matrix(j, which=5)[:, : int(rk[j])].flatten() for j in range(p.J)])
        torch.cuda.synchronize()
        return rk, kept, Q.double().cpu().numpy()

    N.set_filter_kernel(True)
    try:
        base = run()
        N.set_autotune(True)
        first = run()      # times the warps per block
        second = run()     # uses the cached choice
    finally:
        N.set_autotune(False)
        N.set_filter_kernel(False)
    assert np.array_equal(first[0], second[0]) and first[1] == second[1]
    assert np.array_equal(first[2], second[2])
    assert np.array_equal(first[0], base[0])
    assert all(sorted(a) == sorted(b) for a, b in zip(first[1], base[1]))
    if first[1] == base[1]:   # the same pivot order (no near-tie parted them): Q_hat to rounding
        tol = 1e-12 if op == "q64" else 2e-7
        assert np.abs(first[2] - base[2]).max() <= tol
