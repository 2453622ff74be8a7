"""ctypes view of the C ABI in include/rfm.h (argument marshalling only).

The library is required: importing the binding without a built librfm.so
raises, and there is no CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librfm.so")

RFM_OK, RFM_EINVAL, RFM_ECUDA, RFM_ENUMERIC, RFM_ETIMEOUT, RFM_ENOSPACE = range(6)
STATUS = {0: "RFM_OK", 1: "RFM_EINVAL", 2: "RFM_ECUDA", 3: "RFM_ENUMERIC", 4: "RFM_ETIMEOUT", 5: "RFM_ENOSPACE"}
ASM = {"fp64": 0, "fp32": 1}
OPS = {"ar64": 0, "q32": 1, "q64": 2, "plain": 3}


class RfmProblem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("pde", C.c_int32), ("family", C.c_int32), ("n_modes", C.c_int32),
                ("S", C.c_int32 * 3), ("n", C.c_int32 * 3), ("K", C.c_int32), ("reserved0", C.c_int32),
                ("delta", C.c_double), ("kappa", C.c_double), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("lam", C.c_double * 2), ("fam", C.c_double * 64), ("depth", C.c_int32), ("act", C.c_int32),
                ("hard_bc", C.c_double)]


class RfmConfig(C.Structure):
    _fields_ = [("asm_prec", C.c_int32), ("op", C.c_int32), ("tol", C.c_double)]


class RfmSizes(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_inst", "n_blocks", "n_rows", "n_cols", "block_rows",
                                         "max_block_rows", "max_K", "workspace_bytes")]


class RfmLsqrOpts(C.Structure):
    _fields_ = [("atol", C.c_double), ("btol", C.c_double), ("max_iter", C.c_int32), ("timeout_ms", C.c_int32),
                ("d_snap", C.c_void_p), ("snap_every", C.c_int32), ("snap_cap", C.c_int32),
                ("d_phase_ms", C.c_void_p), ("refine_steps", C.c_int32), ("refine_iters", C.c_int32),
                ("d_rnorm64", C.c_void_p)]


class RfmMlp(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("width", C.c_int32 * 9)]


def mlp_struct(widths) -> RfmMlp:
    m = RfmMlp()
    m.n_layers = len(widths) - 1
    for i, w in enumerate(widths):
        m.width[i] = int(w)
    return m


REPORT_FIELDS = ("itn", "istop", "rnorm", "arnorm", "anorm", "ynorm", "bnorm", "status", "start", "r0norm")
REPORT_LEN = len(REPORT_FIELDS)

EXPORTS = ["rfm_problem_size", "rfm_assemble", "rfm_rrqr_filter", "rfm_lsqr_solve", "rfm_coefficients",
           "rfm_eval", "rfm_residual", "rfm_lsqr_multi_size", "rfm_rhs_many", "rfm_lsqr_multi", "rfm_block_info", "rfm_workspace_view", "rfm_profile_enable", "rfm_profile_reset",
           "rfm_profile_read", "rfm_set_option", "rfm_last_error", "rfm_abi_version"]

_lib = None


def load(path: str = LIB_PATH):
    """Load librfm.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with paper_2506_17626_gb300.build.build() "
                      "(there is no fallback implementation)")
    L = C.CDLL(path)
    P = C.POINTER(RfmProblem)
    CF = C.POINTER(RfmConfig)
    vp, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    sigs = {
        "rfm_problem_size": [P, C.c_int, CF, C.POINTER(RfmSizes)],
        "rfm_assemble": [P, C.c_int, CF, vp, vp, C.c_size_t, vp],
        "rfm_rrqr_filter": [P, C.c_int, CF, vp, C.c_size_t, vp, vp, vp],
        "rfm_lsqr_solve": [P, C.c_int, CF, C.POINTER(RfmLsqrOpts), vp, vp, vp, vp, vp, C.c_size_t, vp],
        "rfm_eval": [P, C.c_int, CF, vp, vp, vp, vp, vp, vp, vp, C.c_size_t, vp],
        "rfm_residual": [P, C.c_int, CF, vp, vp, vp, vp, C.c_size_t, vp],
        "rfm_block_rows": [P, C.c_int, CF, i64, vp],
        "rfm_lsqr_multi_size": [P, CF, C.c_int, C.POINTER(C.c_size_t)],
        "rfm_rhs_many": [P, C.c_int, CF, vp, vp, C.c_size_t, vp],
        "rfm_lsqr_multi": [P, CF, C.POINTER(RfmLsqrOpts), C.c_int, vp, vp, vp, vp, vp, C.c_size_t, vp, C.c_size_t, vp],
        "rfm_coefficients": [P, C.c_int, CF, vp, vp, vp, C.c_size_t, vp],
        "rfm_block_info": [P, C.c_int, CF, i64, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)],
        "rfm_workspace_view": [P, C.c_int, CF, vp, C.c_int, C.POINTER(vp)],
        "rfm_block_table": [P, C.c_int, CF, vp, vp, vp, vp],
        "rfm_qr_order": [P, C.c_int, CF, vp],
        "rfm_block_inputs": [P, C.c_int, CF, vp, C.c_int, vp, vp, vp, C.c_size_t, vp],
        "rfm_fit_size": [P, C.c_int, CF, C.POINTER(C.c_size_t)],
        "rfm_fit_prepare": [P, C.c_int, CF, vp, C.c_double, vp, C.c_size_t, vp, C.c_size_t, vp],
        "rfm_warm_start": [P, C.c_int, CF, vp, vp, C.c_int, vp, vp, C.c_size_t, vp, C.c_size_t, vp],
        "rfm_mlp_size": [C.POINTER(RfmMlp), C.POINTER(i64), C.POINTER(C.c_size_t)],
        "rfm_mlp_forward": [C.POINTER(RfmMlp), vp, vp, i64, vp, vp],
        "rfm_mlp_grad": [C.POINTER(RfmMlp), vp, vp, vp, i64, vp, vp, vp, C.c_size_t, vp],
        "rfm_adam_step": [i64, vp, vp, vp, vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, vp],
        "rfm_mlp_train_size": [C.POINTER(RfmMlp), C.c_int, C.POINTER(C.c_size_t)],
        "rfm_mlp_train": [C.POINTER(RfmMlp), vp, vp, vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, vp, C.c_float,
                          C.c_float, C.c_float, vp, vp, C.c_size_t, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.rfm_set_option.argtypes = [C.c_int, C.c_int]
    L.rfm_set_option.restype = C.c_int
    L.rfm_profile_enable.argtypes = [C.c_int]
    L.rfm_profile_enable.restype = C.c_int
    L.rfm_profile_reset.argtypes = []
    L.rfm_profile_reset.restype = C.c_int
    L.rfm_profile_read.argtypes = [C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int]
    L.rfm_profile_read.restype = C.c_int
    L.rfm_last_error.restype = C.c_char_p
    L.rfm_last_error.argtypes = []
    L.rfm_abi_version.restype = C.c_int
    L.rfm_abi_version.argtypes = []
    _lib = L
    return L


class RfmError(RuntimeError):
    def __init__(self, call, code, msg):
        super().__init__(f"{call} -> {STATUS.get(code, code)}: {msg}")
        self.code = code


def check(call: str, code: int):
    if code != RFM_OK:
        raise RfmError(call, code, load().rfm_last_error().decode(errors="replace"))


def problem_struct(p) -> RfmProblem:
    """C struct from any object with the problem attributes (dim, pde, S, n, ...)."""
    s = RfmProblem()
    s.dim, s.pde, s.family = int(p.dim), int(p.pde), int(p.family)
    s.n_modes = int(p.n_modes)
    for i in range(3):
        s.S[i] = int(p.S[i]) if i < min(p.dim, len(p.S)) else 1
        s.n[i] = int(p.n[i]) if i < min(p.dim, len(p.n)) else 1
        s.lo[i] = float(p.lo[i])
        s.hi[i] = float(p.hi[i])
    s.K = int(p.K)
    s.delta, s.kappa = float(p.delta), float(p.kappa)
    s.lam[0], s.lam[1] = float(p.lam[0]), float(p.lam[1])
    fv = p.fam_vector()
    for i in range(64):
        s.fam[i] = float(fv[i])
    s.depth = int(getattr(p, "depth", 1))
    s.act = int(getattr(p, "act", 0))
    s.hard_bc = float(getattr(p, "hard_bc", 0.0))
    return s


def profile_enable(on: bool = True):
    load().rfm_profile_enable(1 if on else 0)


def profile_reset():
    load().rfm_profile_reset()


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last reset (waits for the events)."""
    L = load()
    n = L.rfm_profile_read(None, None, None, 0)
    names = (C.c_char_p * max(n, 1))()
    cnt = (C.c_int64 * max(n, 1))()
    ms = (C.c_double * max(n, 1))()
    n = L.rfm_profile_read(names, cnt, ms, n)
    return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(n)}


def set_filter_kernel(global_memory: bool):
    """Force the global-memory QR kernel (True) or let the library choose (False)."""
    check("rfm_set_option", load().rfm_set_option(0, 1 if global_memory else 0))


def set_autotune(on: bool):
    """Time every feasible QR cluster size on the first filter call of a block
    shape and keep the fastest (RFM_OPT_AUTOTUNE)."""
    check("rfm_set_option", load().rfm_set_option(1, 1 if on else 0))


def set_lsqr_stall(mode: int):
    """Test hook (RFM_OPT_LSQR_STALL): 1 or 2 make the next solves' bounded
    waits run out (first grid barrier, or the forward tiles' waits); 0 is off."""
    check("rfm_set_option", load().rfm_set_option(3, int(mode)))


def set_mlp_tensor_cores(on: bool):
    """Network forward pass and gradient on the tensor cores when every hidden
    layer is 128 wide (True, the default) or always in FP32 (False)
    (RFM_OPT_MLP_TENSOR_CORES)."""
    check("rfm_set_option", load().rfm_set_option(4, 1 if on else 0))


def set_mlp_tc_threads(threads: int):
    """Threads per CTA of the tensor-core network kernels: 512 (default, four
    per sample) or 256 (two per sample) (RFM_OPT_MLP_TC_THREADS)."""
    check("rfm_set_option", load().rfm_set_option(6, int(threads)))


def set_qr_order(largest_first: bool):
    """Launch the QR clusters on the blocks by decreasing work (True, the
    default) or in block order (False) (RFM_OPT_QR_ORDER)."""
    check("rfm_set_option", load().rfm_set_option(5, 1 if largest_first else 0))


def set_lsqr_lag(tenths: int):
    """Lag of the explicit-operator LSQR kernel's row tiles behind their
    block's column chunks, in tenths of a grid pass (RFM_OPT_LSQR_LAG)."""
    check("rfm_set_option", load().rfm_set_option(7, int(tenths)))


def set_multi_tensor_cores(on: bool):
    """Many-right-hand-side LSQR on the FP32 operator: block products on the
    tensor cores (True, the default) or the CUDA cores
    (RFM_OPT_MULTI_TENSOR_CORES)."""
    check("rfm_set_option", load().rfm_set_option(8, 1 if on else 0))


def set_qr_warps(n: int):
    """Warps per CTA of the global-memory QR kernels (RFM_OPT_QR_WARPS)."""
    check("rfm_set_option", load().rfm_set_option(9, int(n)))


def set_qr_panel(n: int):
    """Reflectors per pass of the global-memory double-float Q_hat formation
    (RFM_OPT_QR_PANEL: 1, 2, 4 or 8)."""
    check("rfm_set_option", load().rfm_set_option(10, int(n)))


def set_qr_double_float(on):
    """Factor FP32-assembled blocks with double-float arithmetic (True or 1,
    the default) or with FP64 arithmetic (False or 0); 2 also puts
    FP64-assembled blocks with the FP32 Q_hat operator on the double-float
    kernel (RFM_OPT_QR_DOUBLE_FLOAT)."""
    v = int(on) if not isinstance(on, bool) else (1 if on else 0)
    check("rfm_set_option", load().rfm_set_option(2, v))
