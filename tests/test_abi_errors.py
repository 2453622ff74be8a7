"""Error behaviour of the C ABI, checked on the host with no GPU.

Every compute entry point of include/rfm.h validates its arguments before it
issues any CUDA call: a missing or misaligned workspace and a null required
pointer give RFM_EINVAL, a workspace smaller than the size call asks for gives
RFM_ENOSPACE, and each sets a message for rfm_last_error.  The device pointers
passed here are made-up addresses that are never dereferenced: every case
below is rejected by the host-side checks, before any copy or launch.
"""
import ctypes as C

import pytest

import synth

FAKE = 1 << 20          # a 256-byte aligned address that no call below reaches
MISALIGNED = FAKE + 8


@pytest.fixture(scope="module")
def native():
    from paper_2506_17626_gb300 import build
    build.build()
    from paper_2506_17626_gb300 import _native
    return _native


@pytest.fixture(scope="module")
def sysargs(native):
    p = synth.poisson2d(S=3, K=8, n=12)
    arr = (native.RfmProblem * 1)(native.problem_struct(p))
    cfg = native.RfmConfig(native.ASM["fp32"], native.OPS["q32"], 1e-6)
    sz = native.RfmSizes()
    assert native.load().rfm_problem_size(arr, 1, C.byref(cfg), C.byref(sz)) == native.RFM_OK
    fit = C.c_size_t()
    assert native.load().rfm_fit_size(arr, 1, C.byref(cfg), C.byref(fit)) == native.RFM_OK
    return arr, cfg, int(sz.workspace_bytes), int(fit.value)


def _no_device():
    """The cases that pass the workspace check with a made-up address are
    run only where no CUDA device exists, so that no mistake in them can
    ever reach a GPU."""
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


def _expect(native, rc, status):
    assert rc == status, native.STATUS.get(rc, rc)
    assert len(native.load().rfm_last_error()) > 0


def _calls(native, arr, cfg, ws, nbytes, fws=FAKE, fbytes=1 << 40):
    """Each compute entry point with valid non-workspace arguments (made-up
    device addresses) and the given workspace."""
    L = native.load()
    opts = native.RfmLsqrOpts(1e-8, 1e-8, 10, 0, None, 0, 0, None)
    off = (C.c_int64 * 2)(0, 4)
    return {
        "rfm_assemble": lambda: L.rfm_assemble(arr, 1, C.byref(cfg), FAKE, ws, nbytes, None),
        "rfm_rrqr_filter": lambda: L.rfm_rrqr_filter(arr, 1, C.byref(cfg), ws, nbytes, FAKE, FAKE, None),
        "rfm_lsqr_solve": lambda: L.rfm_lsqr_solve(arr, 1, C.byref(cfg), C.byref(opts), None, FAKE, FAKE, FAKE,
                                                   ws, nbytes, None),
        "rfm_coefficients": lambda: L.rfm_coefficients(arr, 1, C.byref(cfg), FAKE, FAKE, ws, nbytes, None),
        "rfm_eval": lambda: L.rfm_eval(arr, 1, C.byref(cfg), FAKE, FAKE, FAKE, off, FAKE, FAKE, ws, nbytes, None),
        "rfm_block_inputs": lambda: L.rfm_block_inputs(arr, 1, C.byref(cfg), FAKE, 5, FAKE, FAKE, ws, nbytes, None),
        "rfm_fit_prepare": lambda: L.rfm_fit_prepare(arr, 1, C.byref(cfg), FAKE, 1e-10, ws, nbytes, fws, fbytes,
                                                     None),
        "rfm_warm_start": lambda: L.rfm_warm_start(arr, 1, C.byref(cfg), FAKE, None, 10, FAKE, ws, nbytes, fws,
                                                   fbytes, None),
    }


@pytest.mark.parametrize("name", ["rfm_assemble", "rfm_rrqr_filter", "rfm_lsqr_solve", "rfm_coefficients",
                                  "rfm_eval", "rfm_block_inputs", "rfm_fit_prepare", "rfm_warm_start"])
def test_workspace_is_checked_first(native, sysargs, name):
    arr, cfg, total, _ = sysargs
    _expect(native, _calls(native, arr, cfg, None, total)[name](), native.RFM_EINVAL)
    _expect(native, _calls(native, arr, cfg, MISALIGNED, total)[name](), native.RFM_EINVAL)
    _expect(native, _calls(native, arr, cfg, FAKE, total - 1)[name](), native.RFM_ENOSPACE)
    _expect(native, _calls(native, arr, cfg, FAKE, 0)[name](), native.RFM_ENOSPACE)


def test_invalid_problem_is_checked_before_the_workspace(native, sysargs):
    _, cfg, total, _ = sysargs
    p = synth.poisson2d(S=3, K=8, n=12)
    p.K = 0
    bad = (native.RfmProblem * 1)(native.problem_struct(p))
    for name, call in _calls(native, bad, cfg, FAKE, total).items():
        _expect(native, call(), native.RFM_EINVAL)
    L = native.load()
    good = sysargs[0]
    _expect(native, L.rfm_assemble(good, 0, C.byref(cfg), FAKE, FAKE, total, None), native.RFM_EINVAL)


@pytest.mark.skipif(not _no_device(), reason="made-up addresses pass the workspace check: host-only test")
def test_null_arguments_and_bad_options_after_the_workspace_check(native, sysargs):
    arr, cfg, total, fit = sysargs
    L = native.load()
    c = C.byref(cfg)
    _expect(native, L.rfm_assemble(arr, 1, c, None, FAKE, total, None), native.RFM_EINVAL)
    for opts in (None,
                 native.RfmLsqrOpts(1e-8, 1e-8, -1, 0, None, 0, 0, None),
                 native.RfmLsqrOpts(float("nan"), 1e-8, 10, 0, None, 0, 0, None),
                 native.RfmLsqrOpts(1e-8, -1.0, 10, 0, None, 0, 0, None)):
        o = C.byref(opts) if opts is not None else None
        _expect(native, L.rfm_lsqr_solve(arr, 1, c, o, None, FAKE, FAKE, None, FAKE, total, None),
                native.RFM_EINVAL)
    opts = native.RfmLsqrOpts(1e-8, 1e-8, 10, 0, None, 0, 0, None)
    _expect(native, L.rfm_lsqr_solve(arr, 1, c, C.byref(opts), None, FAKE, None, None, FAKE, total, None),
            native.RFM_EINVAL)                                        # d_a is required
    _expect(native, L.rfm_coefficients(arr, 1, c, None, FAKE, FAKE, total, None), native.RFM_EINVAL)
    off = (C.c_int64 * 2)(0, 4)
    _expect(native, L.rfm_eval(arr, 1, c, None, FAKE, FAKE, off, FAKE, None, FAKE, total, None), native.RFM_EINVAL)
    _expect(native, L.rfm_eval(arr, 1, c, FAKE, FAKE, FAKE, None, FAKE, None, FAKE, total, None), native.RFM_EINVAL)
    for n_ctx, ctx in ((65, FAKE), (-1, FAKE), (3, None)):
        _expect(native, L.rfm_block_inputs(arr, 1, c, ctx, n_ctx, FAKE, None, FAKE, total, None), native.RFM_EINVAL)
    # the fitting workspace: missing, misaligned, short; then the fit's own arguments
    _expect(native, L.rfm_fit_prepare(arr, 1, c, FAKE, 1e-10, FAKE, total, None, fit, None), native.RFM_EINVAL)
    _expect(native, L.rfm_fit_prepare(arr, 1, c, FAKE, 1e-10, FAKE, total, MISALIGNED, fit, None),
            native.RFM_EINVAL)
    _expect(native, L.rfm_fit_prepare(arr, 1, c, FAKE, 1e-10, FAKE, total, FAKE, fit - 1, None),
            native.RFM_ENOSPACE)
    for tol_fit in (1.0, -1e-3, float("nan")):
        _expect(native, L.rfm_fit_prepare(arr, 1, c, FAKE, tol_fit, FAKE, total, FAKE, fit, None),
                native.RFM_EINVAL)
    _expect(native, L.rfm_warm_start(arr, 1, c, None, None, 10, FAKE, FAKE, total, FAKE, fit, None),
            native.RFM_EINVAL)
    _expect(native, L.rfm_warm_start(arr, 1, c, FAKE, None, -1, FAKE, FAKE, total, FAKE, fit, None),
            native.RFM_EINVAL)


@pytest.mark.parametrize("widths,ok", [([9, 128, 128, 128, 128, 1], True), ([9, 16, 1], True), ([3, 1], True),
                                       ([9, 20, 1], False), ([9, 128, 2], False), ([9, 144, 1], False),
                                       ([0, 16, 1], False), ([9] + [16] * 9 + [1], False)])
def test_network_shapes(native, widths, ok):
    L = native.load()
    m = native.RfmMlp()
    m.n_layers = min(len(widths) - 1, 9)
    for i, w in enumerate(widths[:9]):
        m.width[i] = int(w)
    npar, wsb = C.c_int64(), C.c_size_t()
    rc = L.rfm_mlp_size(C.byref(m), C.byref(npar), C.byref(wsb))
    if ok:
        assert rc == native.RFM_OK
        assert npar.value == sum(widths[i] * widths[i - 1] + widths[i] for i in range(1, len(widths)))
        tb = C.c_size_t()
        assert L.rfm_mlp_train_size(C.byref(m), 256, C.byref(tb)) == native.RFM_OK and tb.value > 0
        _expect(native, L.rfm_mlp_train_size(C.byref(m), 0, C.byref(tb)), native.RFM_EINVAL)
    else:
        _expect(native, rc, native.RFM_EINVAL)


def test_network_calls_reject_null_arguments(native):
    L = native.load()
    m = native.mlp_struct([9, 16, 1])
    _expect(native, L.rfm_mlp_forward(C.byref(m), None, FAKE, 10, FAKE, None), native.RFM_EINVAL)
    _expect(native, L.rfm_mlp_forward(C.byref(m), FAKE, None, 10, FAKE, None), native.RFM_EINVAL)
    _expect(native, L.rfm_mlp_forward(C.byref(m), FAKE, FAKE, -1, FAKE, None), native.RFM_EINVAL)
    _expect(native, L.rfm_mlp_grad(C.byref(m), FAKE, FAKE, None, 10, FAKE, None, FAKE, 1 << 30, None),
            native.RFM_EINVAL)
    _expect(native, L.rfm_adam_step(10, FAKE, FAKE, None, FAKE, 1, 1e-3, 0.9, 0.999, 1e-8, None), native.RFM_EINVAL)
    lr = (C.c_float * 1)(1e-3)
    _expect(native, L.rfm_mlp_train(C.byref(m), FAKE, FAKE, FAKE, FAKE, FAKE, None, 64, 1, 1, lr, 0.9, 0.999, 1e-8,
                                    None, FAKE, 1 << 30, None), native.RFM_EINVAL)
    _expect(native, L.rfm_mlp_train(C.byref(m), FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 64, 1, 1, None, 0.9, 0.999,
                                    1e-8, None, FAKE, 1 << 30, None), native.RFM_EINVAL)


def test_unknown_option_is_rejected(native):
    _expect(native, native.load().rfm_set_option(12345, 1), native.RFM_EINVAL)


def test_option_values_are_checked(native):
    """Warps per block and panel widths outside their sets are rejected; the
    defaults (32 warps, panels of 8) are put back afterwards."""
    L = native.load()
    for opt, bad, good, default in ((9, [0, 3, 64], [4, 8, 16], 32), (10, [0, 3, 16], [1, 2, 4], 8)):
        for v in bad:
            _expect(native, L.rfm_set_option(opt, v), native.RFM_EINVAL)
        try:
            for v in good:
                assert L.rfm_set_option(opt, v) == native.RFM_OK
        finally:
            assert L.rfm_set_option(opt, default) == native.RFM_OK


@pytest.mark.parametrize("case", ["depth", "deep_width", "act", "hard_bc_negative", "hard_bc_heat", "osc_2d",
                                  "osc_family"])
def test_invalid_networks_and_problem_kinds_are_rejected(native, case):
    """The size call rejects networks and problem kinds the path does not
    define, with a message, before anything else."""
    p = synth.poisson2d(S=3, K=8, n=12)
    if case == "depth":
        p.depth = 9
    elif case == "deep_width":
        p.depth, p.K = 3, 40
    elif case == "act":
        p.act = 3
    elif case == "hard_bc_negative":
        p.hard_bc = -1.0
    elif case == "hard_bc_heat":
        p = synth.heat3d(S=2, K=4, n=5)
        p.hard_bc = 2.0
    elif case == "osc_2d":
        p.pde = synth.PDE_OSC
    else:
        p = synth.oscillator(S=3, K=4)
        p.family = synth.FAM_SINPROD
    arr = (native.RfmProblem * 1)(native.problem_struct(p))
    cfg = native.RfmConfig(native.ASM["fp64"], native.OPS["ar64"], 1e-6)
    sz = native.RfmSizes()
    assert native.load().rfm_problem_size(arr, 1, C.byref(cfg), C.byref(sz)) == native.RFM_EINVAL
    assert native.load().rfm_last_error()
