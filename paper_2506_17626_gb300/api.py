"""Python face of the library: same calls as include/rfm.h, PyTorch for device
memory and streams.  Every numerical step runs in the CUDA kernels of
librfm.so; this module only allocates the workspace and passes pointers.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class System:
    """One or more problem instances solved side by side in one workspace.

    asm: "fp64" | "fp32" (assembly arithmetic); op: "ar64" (FP64 kept columns
    with R^-1 substitution), "q32" (explicit Q_hat in FP32, mixed precision),
    "q64" (explicit Q_hat in FP64), "plain" (no filter, no preconditioner);
    tol: relative drop threshold of the filter.
    """

    def __init__(self, problems, asm: str = "fp64", op: str = "ar64", tol: float = 1e-10,
                 device: str = "cuda"):
        self.problems = list(problems) if isinstance(problems, (list, tuple)) else [problems]
        self.n = len(self.problems)
        self._probs = (N.RfmProblem * self.n)(*[N.problem_struct(p) for p in self.problems])
        self._cfg = N.RfmConfig(N.ASM[asm], N.OPS[op], float(tol))
        self.asm, self.op, self.tol = asm, op, tol
        self.lib = N.load()
        sz = N.RfmSizes()
        N.check("rfm_problem_size", self.lib.rfm_problem_size(self._probs, self.n, C.byref(self._cfg), C.byref(sz)))
        self.sizes = {f: getattr(sz, f) for f, _ in N.RfmSizes._fields_}
        self.device = torch.device(device)
        self.ws = torch.empty(self.sizes["workspace_bytes"] + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_off = (-base) % 256
        self.ws_ptr = base + self._ws_off
        self.ws_bytes = self.sizes["workspace_bytes"]

    # -- the four calls of the path -------------------------------------------------
    def assemble(self, params: torch.Tensor):
        """params: FP64 device tensor, all instances' (J, K, dim+1) arrays concatenated."""
        assert params.is_cuda and params.dtype == torch.float64 and params.is_contiguous()
        self._params = params
        N.check("rfm_assemble", self.lib.rfm_assemble(self._probs, self.n, C.byref(self._cfg), _ptr(params),
                                                      C.c_void_p(self.ws_ptr), self.ws_bytes, _stream()))

    def filter(self, want_perm: bool = False):
        nb = self.sizes["n_blocks"]
        rank = torch.empty(nb, dtype=torch.int32, device=self.device) if self.op != "plain" else None
        perm = torch.empty(self.sizes["n_cols"], dtype=torch.int32, device=self.device) if want_perm else None
        N.check("rfm_rrqr_filter", self.lib.rfm_rrqr_filter(self._probs, self.n, C.byref(self._cfg),
                                                            C.c_void_p(self.ws_ptr), self.ws_bytes, _ptr(rank),
                                                            _ptr(perm), _stream()))
        return (rank, perm) if want_perm else rank

    def solve(self, atol=1e-10, btol=1e-10, max_iter=10000, y0: Optional[torch.Tensor] = None,
              timeout_ms: int = 10000, want_y: bool = False, snap: Optional[torch.Tensor] = None,
              snap_every: int = 0, phase_ms: Optional[torch.Tensor] = None, refine_steps: int = 0,
              refine_iters: int = 0, rnorm64: Optional[torch.Tensor] = None):
        """LSQR of Algorithm 2.  snap: optional (cap, n_cols) FP64 tensor that
        receives y after every snap_every-th iteration.  refine_steps > 0 adds
        that many correction solves (at most refine_iters iterations each) on
        the FP64 residual of the assembled system; rnorm64: optional FP64
        tensor of n x (refine_steps + 1) that receives those residual norms."""
        nc = self.sizes["n_cols"]
        a = torch.empty(nc, dtype=torch.float64, device=self.device)
        y = torch.empty(nc, dtype=torch.float64, device=self.device) if want_y else None
        rep = torch.empty(self.n * N.REPORT_LEN, dtype=torch.float64, device=self.device)
        cap = 0 if snap is None else snap.shape[0]
        if snap is not None:
            assert snap.is_cuda and snap.dtype == torch.float64 and snap.shape[1] == nc and snap.is_contiguous()
        if rnorm64 is not None:
            assert rnorm64.is_cuda and rnorm64.dtype == torch.float64 and rnorm64.is_contiguous()
            assert rnorm64.numel() >= self.n * (refine_steps + 1)
        opts = N.RfmLsqrOpts(float(atol), float(btol), int(max_iter), int(timeout_ms),
                             _ptr(snap), int(snap_every if snap is not None else 0), int(cap), _ptr(phase_ms),
                             int(refine_steps), int(refine_iters), _ptr(rnorm64))
        if y0 is not None:
            assert y0.is_cuda and y0.dtype == torch.float64 and y0.numel() == nc
        N.check("rfm_lsqr_solve", self.lib.rfm_lsqr_solve(self._probs, self.n, C.byref(self._cfg), C.byref(opts),
                                                          _ptr(y0), _ptr(y), _ptr(a), _ptr(rep),
                                                          C.c_void_p(self.ws_ptr), self.ws_bytes, _stream()))
        return (a, rep, y) if want_y else (a, rep)

    def residual(self, a: torch.Tensor, want_r: bool = False):
        """||h - M a|| per instance (FP64, from the assembled blocks), and r
        itself when want_r."""
        assert a.is_cuda and a.dtype == torch.float64 and a.numel() == self.sizes["n_cols"]
        r = torch.empty(self.sizes["n_rows"], dtype=torch.float64, device=self.device) if want_r else None
        rn = torch.empty(self.n, dtype=torch.float64, device=self.device)
        N.check("rfm_residual", self.lib.rfm_residual(self._probs, self.n, C.byref(self._cfg), _ptr(a), _ptr(r),
                                                      _ptr(rn), C.c_void_p(self.ws_ptr), self.ws_bytes, _stream()))
        return (rn, r) if want_r else rn

    # -- many right-hand sides on one operator ------------------------------------
    def _multi_ws(self, nrhs: int):
        nb = C.c_size_t()
        N.check("rfm_lsqr_multi_size", self.lib.rfm_lsqr_multi_size(self._probs, C.byref(self._cfg), int(nrhs),
                                                                    C.byref(nb)))
        ws = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        return ws, ws.data_ptr() + (-ws.data_ptr()) % 256, nb.value

    def rhs_many(self, problems) -> torch.Tensor:
        """h of data sets `problems` (same decomposition, features and rows as
        this one-instance system, other data), nrhs x n_rows FP64."""
        assert self.n == 1
        n = len(problems)
        arr = (N.RfmProblem * n)(*[N.problem_struct(p) for p in problems])
        H = torch.empty((n, self.sizes["n_rows"]), dtype=torch.float64, device=self.device)
        ws, ptr, nb = self._multi_ws(n)
        N.check("rfm_rhs_many", self.lib.rfm_rhs_many(arr, n, C.byref(self._cfg), _ptr(H), C.c_void_p(ptr), nb,
                                                      _stream()))
        self._mws_keep = ws
        return H

    def solve_multi(self, H: torch.Tensor, atol=1e-10, btol=1e-10, max_iter=10000, Y0: Optional[torch.Tensor] = None):
        """LSQR for every row of H (nrhs x n_rows) on this system's operator
        (one instance, explicit Q_hat), from zero or from the rows of Y0
        (nrhs x n_cols, the y layout of solve's y0; a set falls back to zero
        when its start's residual is not below ||h||); returns the
        coefficients (nrhs x n_cols) and the reports (nrhs x report fields)."""
        assert H.is_cuda and H.dtype == torch.float64 and H.is_contiguous() and H.shape[1] == self.sizes["n_rows"]
        n = H.shape[0]
        if Y0 is not None:
            assert Y0.is_cuda and Y0.dtype == torch.float64 and Y0.is_contiguous()
            assert tuple(Y0.shape) == (n, self.sizes["n_cols"])
        A = torch.empty((n, self.sizes["n_cols"]), dtype=torch.float64, device=self.device)
        rep = torch.empty(n * N.REPORT_LEN, dtype=torch.float64, device=self.device)
        ws, ptr, nb = self._multi_ws(n)
        opts = N.RfmLsqrOpts(float(atol), float(btol), int(max_iter), 10000, None, 0, 0, None, 0, 0, None)
        N.check("rfm_lsqr_multi", self.lib.rfm_lsqr_multi(self._probs, C.byref(self._cfg), C.byref(opts), n, _ptr(H),
                                                          _ptr(Y0),
                                                          _ptr(A), _ptr(rep), C.c_void_p(self.ws_ptr), self.ws_bytes,
                                                          C.c_void_p(ptr), nb, _stream()))
        self._mws_keep = ws
        return A, rep

    def coefficients(self, y: torch.Tensor) -> torch.Tensor:
        """a = S^-1 y with zeros at dropped columns (Algorithm 2, last step)."""
        a = torch.empty(self.sizes["n_cols"], dtype=torch.float64, device=self.device)
        N.check("rfm_coefficients", self.lib.rfm_coefficients(self._probs, self.n, C.byref(self._cfg), _ptr(y),
                                                              _ptr(a), C.c_void_p(self.ws_ptr), self.ws_bytes,
                                                              _stream()))
        return a

    def evaluate(self, params: torch.Tensor, a: torch.Tensor, X: Sequence[torch.Tensor], with_error=True):
        """u_hat at points X[s] (n_s x dim FP64 tensors, one per instance); error sums per instance."""
        pts = []
        offs = [0]
        for x in X:
            x3 = torch.zeros((x.shape[0], 3), dtype=torch.float64, device=self.device)
            x3[:, : x.shape[1]] = x
            pts.append(x3)
            offs.append(offs[-1] + x.shape[0])
        Xc = torch.cat(pts).contiguous()
        u = torch.empty(offs[-1], dtype=torch.float64, device=self.device)
        err = torch.zeros(4 * self.n, dtype=torch.float64, device=self.device) if with_error else None
        off_arr = (C.c_int64 * (self.n + 1))(*offs)
        N.check("rfm_eval", self.lib.rfm_eval(self._probs, self.n, C.byref(self._cfg), _ptr(params), _ptr(a),
                                              _ptr(Xc), off_arr, _ptr(u), _ptr(err), C.c_void_p(self.ws_ptr),
                                              self.ws_bytes, _stream()))
        return [u[offs[i]:offs[i + 1]] for i in range(self.n)], err

    def block_table(self):
        """(m, ld, moff, roff) of every block as int64 numpy arrays."""
        nb = self.sizes["n_blocks"]
        arrs = [np.zeros(nb, dtype=np.int64) for _ in range(4)]
        N.check("rfm_block_table", self.lib.rfm_block_table(self._probs, self.n, C.byref(self._cfg),
                                                            *[a.ctypes.data_as(C.c_void_p) for a in arrs]))
        return tuple(arrs)

    # -- learned warm start -------------------------------------------------------------
    def block_inputs(self, ctx: Optional[torch.Tensor], want_points: bool = True):
        """Network inputs at every block row (block-row layout, padding rows
        zero): [ctx of the instance, block centre, local coordinates], FP32;
        and the rows' points (block_rows x 3, FP64) when want_points."""
        n_ctx = 0 if ctx is None else ctx.shape[1]
        if ctx is not None:
            assert ctx.is_cuda and ctx.dtype == torch.float32 and ctx.is_contiguous() and ctx.shape[0] == self.n
        dim = self.problems[0].dim
        assert all(p.dim == dim for p in self.problems)
        nr = self.sizes["block_rows"]
        X = torch.empty((nr, n_ctx + 2 * dim), dtype=torch.float32, device=self.device)
        pts = torch.empty((nr, 3), dtype=torch.float64, device=self.device) if want_points else None
        N.check("rfm_block_inputs", self.lib.rfm_block_inputs(self._probs, self.n, C.byref(self._cfg), _ptr(ctx),
                                                              n_ctx, _ptr(X), _ptr(pts), C.c_void_p(self.ws_ptr),
                                                              self.ws_bytes, _stream()))
        return X, pts

    def fit_prepare(self, params: torch.Tensor, tol_fit: float = 1e-10):
        """Factor the kept features' values per block (after filter())."""
        nb = C.c_size_t()
        N.check("rfm_fit_size", self.lib.rfm_fit_size(self._probs, self.n, C.byref(self._cfg), C.byref(nb)))
        self.fit_bytes = nb.value
        self.fws = torch.empty(self.fit_bytes + 256, dtype=torch.uint8, device=self.device)
        self.fws_ptr = self.fws.data_ptr() + (-self.fws.data_ptr()) % 256
        N.check("rfm_fit_prepare", self.lib.rfm_fit_prepare(self._probs, self.n, C.byref(self._cfg), _ptr(params),
                                                            float(tol_fit), C.c_void_p(self.ws_ptr), self.ws_bytes,
                                                            C.c_void_p(self.fws_ptr), self.fit_bytes, _stream()))

    def warm_start(self, uhat: torch.Tensor, fit_iters: int = 0,
                   inst_scale: Optional[torch.Tensor] = None) -> torch.Tensor:
        """y0 (column-slot layout) from predictions at the block rows (FP32),
        optionally multiplied by a per-instance scale (FP32, one per instance):
        fit_iters = 0 fits block by block, > 0 fits all blocks at once with
        that many LSQR iterations."""
        assert uhat.is_cuda and uhat.dtype == torch.float32 and uhat.numel() >= self.sizes["block_rows"]
        if inst_scale is not None:
            assert inst_scale.is_cuda and inst_scale.dtype == torch.float32 and inst_scale.numel() == self.n
        y0 = torch.empty(self.sizes["n_cols"], dtype=torch.float64, device=self.device)
        N.check("rfm_warm_start", self.lib.rfm_warm_start(self._probs, self.n, C.byref(self._cfg), _ptr(uhat),
                                                          _ptr(inst_scale), int(fit_iters), _ptr(y0),
                                                          C.c_void_p(self.ws_ptr),
                                                          self.ws_bytes, C.c_void_p(self.fws_ptr), self.fit_bytes,
                                                          _stream()))
        return y0

    # -- views for tests --------------------------------------------------------------
    def view(self, which: int) -> int:
        p = C.c_void_p()
        N.check("rfm_workspace_view", self.lib.rfm_workspace_view(self._probs, self.n, C.byref(self._cfg),
                                                                  C.c_void_p(self.ws_ptr), which, C.byref(p)))
        return p.value

    def _tensor_at(self, ptr: int, count: int, dtype) -> torch.Tensor:
        off = ptr - self.ws.data_ptr()
        es = torch.empty(0, dtype=dtype).element_size()
        assert off % es == 0
        return self.ws[off: off + count * es].view(dtype)

    def block_info(self, b: int):
        m, ld, moff, roff = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        N.check("rfm_block_info", self.lib.rfm_block_info(self._probs, self.n, C.byref(self._cfg), int(b),
                                                          C.byref(m), C.byref(ld), C.byref(moff), C.byref(roff)))
        return m.value, ld.value, moff.value, roff.value

    def _K_of_block(self, b: int) -> int:
        for p in self.problems:
            if b < p.J:
                return p.K
            b -= p.J
        raise IndexError(b)

    def block_matrix(self, b: int, which: int = 0) -> torch.Tensor:
        """Block b of an (ldm x K) arena (0 = M, 3 = QR work, 5 = operator), as an m x K view."""
        m, ld, moff, roff = self.block_info(b)
        K = self._K_of_block(b)
        if which == 0:
            dt = torch.float32 if self.asm == "fp32" else torch.float64
        elif which == 5:
            dt = torch.float32 if self.op == "q32" else torch.float64
        else:
            dt = torch.float64
        base = self._tensor_at(self.view(which) + moff * torch.empty(0, dtype=dt).element_size(), ld * K, dt)
        return base.view(K, ld).t()[:m]

    def block_rows(self, b: int) -> torch.Tensor:
        m, ld, moff, roff = self.block_info(b)
        return self._tensor_at(self.view(2), self.sizes["block_rows"], torch.int32)[roff: roff + m]

    def rhs(self) -> torch.Tensor:
        return self._tensor_at(self.view(1), self.sizes["n_rows"], torch.float64)

    def r11(self) -> torch.Tensor:
        return self._tensor_at(self.view(4), self.sizes["n_blocks"], torch.float64)


def report_dict(rep: torch.Tensor, i: int = 0) -> dict:
    r = rep.view(-1, N.REPORT_LEN)[i].tolist()
    return {k: (int(v) if k in ("itn", "istop", "status", "start") else v) for k, v in zip(N.REPORT_FIELDS, r)}


class Mlp:
    """The warm-start network of include/rfm.h (FP32 parameters, tanh hidden
    layers, scalar linear output); forward, loss gradient and Adam run in the
    library's kernels."""

    def __init__(self, widths, device: str = "cuda"):
        self.widths = [int(w) for w in widths]
        self._net = N.mlp_struct(self.widths)
        self.lib = N.load()
        npar, wsb = C.c_int64(), C.c_size_t()
        N.check("rfm_mlp_size", self.lib.rfm_mlp_size(C.byref(self._net), C.byref(npar), C.byref(wsb)))
        self.n_params = npar.value
        self.device = torch.device(device)
        self._ws = torch.empty(wsb.value + 256, dtype=torch.uint8, device=self.device)
        self._ws_ptr = self._ws.data_ptr() + (-self._ws.data_ptr()) % 256
        self._ws_bytes = wsb.value

    def forward(self, theta: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        assert theta.dtype == torch.float32 and X.dtype == torch.float32 and X.is_contiguous()
        Y = torch.empty(X.shape[0], dtype=torch.float32, device=self.device)
        N.check("rfm_mlp_forward", self.lib.rfm_mlp_forward(C.byref(self._net), _ptr(theta), _ptr(X), X.shape[0],
                                                            _ptr(Y), _stream()))
        return Y

    def grad(self, theta: torch.Tensor, X: torch.Tensor, T: torch.Tensor, out: Optional[torch.Tensor] = None,
             loss: Optional[torch.Tensor] = None):
        assert X.dtype == torch.float32 and T.dtype == torch.float32 and X.is_contiguous() and T.is_contiguous()
        g = out if out is not None else torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        lo = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=self.device)
        N.check("rfm_mlp_grad", self.lib.rfm_mlp_grad(C.byref(self._net), _ptr(theta), _ptr(X), _ptr(T), X.shape[0],
                                                      _ptr(g), _ptr(lo), C.c_void_p(self._ws_ptr), self._ws_bytes,
                                                      _stream()))
        return g, lo

    def train_steps(self, theta, m, v, X: torch.Tensor, T: torch.Tensor, order: torch.Tensor, batch: int,
                    t0: int, lrs, b1=0.9, b2=0.999, eps=1e-8, loss: Optional[torch.Tensor] = None):
        """len(lrs) minibatch steps in one library call: step k takes the samples
        order[k batch:(k+1) batch] (int64, on the device), the loss gradient
        and an Adam step with number t0 + k and rate lrs[k]."""
        n_steps = len(lrs)
        assert order.dtype == torch.int64 and order.is_contiguous() and order.numel() >= n_steps * batch
        assert X.dtype == torch.float32 and T.dtype == torch.float32 and X.is_contiguous() and T.is_contiguous()
        wsb = C.c_size_t()
        N.check("rfm_mlp_train_size", self.lib.rfm_mlp_train_size(C.byref(self._net), int(batch), C.byref(wsb)))
        if getattr(self, "_tws_bytes", 0) < wsb.value:
            self._tws = torch.empty(wsb.value + 256, dtype=torch.uint8, device=self.device)
            self._tws_bytes = wsb.value
        ptr = self._tws.data_ptr() + (-self._tws.data_ptr()) % 256
        lr_arr = (C.c_float * max(1, n_steps))(*[float(r) for r in lrs])
        N.check("rfm_mlp_train", self.lib.rfm_mlp_train(C.byref(self._net), _ptr(theta), _ptr(m), _ptr(v), _ptr(X),
                                                        _ptr(T), _ptr(order), int(batch), int(n_steps), int(t0),
                                                        lr_arr, float(b1), float(b2), float(eps), _ptr(loss),
                                                        C.c_void_p(ptr), self._tws_bytes, _stream()))

    def adam_step(self, theta, m, v, g, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        N.check("rfm_adam_step", self.lib.rfm_adam_step(theta.numel(), _ptr(theta), _ptr(m), _ptr(v), _ptr(g), int(t),
                                                        float(lr), float(b1), float(b2), float(eps), _stream()))
