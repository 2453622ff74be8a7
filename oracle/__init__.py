"""CPU oracle for the ELM-FBPINN RRQR-filtered, right-preconditioned solver.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library never
does.  The numerics live in ``rfm_oracle.c`` (plain FP64 loops written from the
paper); this module only marshals numpy arrays through ctypes and strings the
steps of Algorithm 2 together.

Every function here is pinned by a ``-m "not gpu"`` test in
tests/test_oracle_*.py against something other than itself (closed forms,
invariants, numpy/scipy routines on tiny inputs, finite differences); the
docstring of each test names its pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "rfm_oracle.c"), os.path.join(_HERE, "mlp_oracle.c")]
_SO = os.path.join(_HERE, "_build", "librfm_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no host-specific flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(s) for s in _SRCS):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
                               "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("pde", C.c_int32), ("family", C.c_int32), ("n_modes", C.c_int32),
                ("S", C.c_int32 * 3), ("n", C.c_int32 * 3), ("K", C.c_int32), ("pad0", C.c_int32),
                ("delta", C.c_double), ("kappa", C.c_double), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("lam", C.c_double * 2), ("fam", C.c_double * 64), ("depth", C.c_int32), ("act", C.c_int32),
                ("hard_bc", C.c_double)]


class System(C.Structure):
    _fields_ = [("J", C.c_int64), ("N", C.c_int64), ("m", C.c_void_p), ("roff", C.c_void_p),
                ("grow", C.c_void_p), ("coff", C.c_void_p), ("aoff", C.c_void_p), ("Roff", C.c_void_p),
                ("r", C.c_void_p), ("Ahat", C.c_void_p), ("R", C.c_void_p), ("mode", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER(Problem)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sig = {
            "orc_num_interior": (i64, [P]), "orc_num_boundary": (i64, [P]), "orc_num_set": (i64, [P, C.c_int]),
            "orc_num_subdomains": (i64, [P]), "orc_row_point": (None, [P, i64, vp, vp]),
            "orc_subdomain": (None, [P, i64, vp, vp]), "orc_window_hat": (dbl, [P, i64, vp, vp, vp]),
            "orc_window": (dbl, [P, i64, vp, vp, vp]), "orc_exact": (dbl, [P, vp]),
            "orc_source": (dbl, [P, vp]), "orc_bdata": (dbl, [P, vp]),
            "orc_bdata_set": (dbl, [P, vp, C.c_int]), "orc_params_per_subdomain": (i64, [P]),
            "orc_block_rows": (i64, [P, i64, vp]), "orc_assemble_block": (None, [P, vp, i64, vp, i64, vp]),
            "orc_rhs": (None, [P, vp]), "orc_assemble_dense": (None, [P, vp, vp]),
            "orc_qrcp": (C.c_int, [C.c_int, C.c_int, vp, C.c_int, dbl, vp, vp, vp]),
            "orc_form_q": (None, [C.c_int, C.c_int, vp, C.c_int, vp, vp]),
            "orc_trsv_upper": (None, [C.c_int, vp, C.c_int, vp]),
            "orc_trsv_upper_t": (None, [C.c_int, vp, C.c_int, vp]),
            "orc_op_apply": (None, [C.POINTER(System), vp, vp]),
            "orc_op_apply_t": (None, [C.POINTER(System), vp, vp]),
            "orc_lsqr": (C.c_int, [C.POINTER(System), vp, vp, dbl, dbl, C.c_int, vp, vp, vp]),
            "orc_coefficients": (None, [i64, C.c_int, vp, vp, vp, vp, vp, vp, vp]),
            "orc_eval": (None, [P, vp, vp, i64, vp, vp]),
            "orc_exact_many": (None, [P, i64, vp, vp]),
            "orc_feature_values": (None, [P, vp, i64, i64, vp, vp]),
            "orc_mlp_nparams": (i64, [C.c_int, vp]),
            "orc_mlp_forward": (None, [C.c_int, vp, vp, i64, vp, vp]),
            "orc_mlp_grad": (dbl, [C.c_int, vp, vp, i64, vp, vp, vp]),
            "orc_adam_step": (None, [i64, vp, vp, vp, vp, C.c_int, dbl, dbl, dbl, dbl]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def problem_struct(p) -> Problem:
    """ctypes struct from a synth.Problem."""
    s = Problem()
    s.dim, s.pde, s.family, s.n_modes = p.dim, p.pde, p.family, p.n_modes
    for i in range(3):
        s.S[i] = int(p.S[i]) if i < p.dim else 1
        s.n[i] = int(p.n[i]) if i < p.dim else 1
        s.lo[i] = float(p.lo[i])
        s.hi[i] = float(p.hi[i])
    s.K = p.K
    s.delta, s.kappa = float(p.delta), float(p.kappa)
    s.lam[0], s.lam[1] = float(p.lam[0]), float(p.lam[1])
    fv = p.fam_vector()
    for i in range(64):
        s.fam[i] = fv[i]
    s.depth = int(getattr(p, "depth", 1))
    s.act = int(getattr(p, "act", 0))
    s.hard_bc = float(getattr(p, "hard_bc", 0.0))
    if s.depth > 1 and p.K > 128:
        raise ValueError("the oracle's deep networks are at most 128 wide")
    return s


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def sizes(p):
    s = problem_struct(p)
    L = lib()
    NI, NB = L.orc_num_interior(C.byref(s)), L.orc_num_boundary(C.byref(s))
    return dict(N_I=NI, N_B=NB, N=NI + NB, J=L.orc_num_subdomains(C.byref(s)), K=p.K)


def row_points(p, rows=None):
    s = problem_struct(p)
    L = lib()
    if rows is None:
        rows = np.arange(sizes(p)["N"])
    X = np.zeros((len(rows), 3))
    kinds = np.zeros(len(rows), dtype=np.int32)
    x = np.zeros(3)
    k = C.c_int()
    for i, r in enumerate(rows):
        L.orc_row_point(C.byref(s), int(r), _p(x), C.byref(k))
        X[i] = x
        kinds[i] = k.value
    return X[:, : p.dim], kinds


def subdomain(p, j):
    s = problem_struct(p)
    mu, sg = np.zeros(3), np.zeros(3)
    lib().orc_subdomain(C.byref(s), int(j), _p(mu), _p(sg))
    return mu[: p.dim], sg[: p.dim]


def window(p, j, x, normalised=True):
    """(w, grad w, pure second partials) of subdomain j at point x."""
    s = problem_struct(p)
    xx = np.zeros(3)
    xx[: p.dim] = x
    dw, d2w = np.zeros(3), np.zeros(3)
    f = lib().orc_window if normalised else lib().orc_window_hat
    w = f(C.byref(s), int(j), _p(xx), _p(dw), _p(d2w))
    return w, dw[: p.dim].copy(), d2w[: p.dim].copy()


def exact(p, X):
    s = problem_struct(p)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, p.dim)
    u = np.zeros(len(X))
    lib().orc_exact_many(C.byref(s), len(X), _p(X), _p(u))
    return u


def source(p, x):
    s = problem_struct(p)
    xx = np.zeros(3)
    xx[: p.dim] = x
    return lib().orc_source(C.byref(s), _p(xx))


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------

@dataclass
class Blocks:
    grow: List[np.ndarray]      # global row indices of each block (ascending)
    M: List[np.ndarray]         # blocks m_j x K (Fortran order)
    h: np.ndarray               # right-hand side over all rows
    N: int


def block_rows(p, j) -> np.ndarray:
    s = problem_struct(p)
    L = lib()
    m = L.orc_block_rows(C.byref(s), int(j), None)
    g = np.zeros(m, dtype=np.int64)
    L.orc_block_rows(C.byref(s), int(j), _p(g))
    return g


def assemble(p, params: np.ndarray, blocks=None) -> Blocks:
    """Per-block assembly of M (Eq. (6)) and h (Eq. (5))."""
    s = problem_struct(p)
    L = lib()
    params = np.ascontiguousarray(params, dtype=np.float64)
    J = L.orc_num_subdomains(C.byref(s))
    idx = range(J) if blocks is None else blocks
    grows, Ms = [], []
    for j in idx:
        g = block_rows(p, j)
        Mj = np.zeros((len(g), p.K), order="F")
        L.orc_assemble_block(C.byref(s), _p(params), int(j), _p(g), len(g), Mj.ctypes.data_as(C.c_void_p))
        grows.append(g)
        Ms.append(Mj)
    N = sizes(p)["N"]
    h = np.zeros(N)
    L.orc_rhs(C.byref(s), _p(h))
    return Blocks(grows, Ms, h, N)


def assemble_dense(p, params):
    s = problem_struct(p)
    z = sizes(p)
    M = np.zeros((z["N"], z["J"] * p.K), order="F")
    params = np.ascontiguousarray(params, dtype=np.float64)
    lib().orc_assemble_dense(C.byref(s), _p(params), M.ctypes.data_as(C.c_void_p))
    h = np.zeros(z["N"])
    lib().orc_rhs(C.byref(s), _p(h))
    return M, h


# ---------------------------------------------------------------------------
# filtering
# ---------------------------------------------------------------------------

@dataclass
class QRCP:
    rank: int
    perm: np.ndarray      # original column index of each pivoted column
    tau: np.ndarray
    QR: np.ndarray        # R above the diagonal, reflectors below (Fortran order)
    r11: float

    @property
    def R(self):
        r = self.rank
        return np.triu(self.QR[:r, :r])

    def Q(self):
        m = self.QR.shape[0]
        Q = np.zeros((m, self.rank), order="F")
        if self.rank:
            lib().orc_form_q(m, self.rank, self.QR.ctypes.data_as(C.c_void_p), m, _p(self.tau),
                             Q.ctypes.data_as(C.c_void_p))
        return Q


def qrcp(A: np.ndarray, tol: float) -> QRCP:
    """sigma-RRQR of one block (Algorithm 1, threshold relative to |R_11|)."""
    m, n = A.shape
    W = np.array(A, dtype=np.float64, order="F", copy=True)
    perm = np.zeros(n, dtype=np.int32)
    tau = np.zeros(max(1, min(m, n)))
    r11 = C.c_double()
    r = lib().orc_qrcp(m, n, W.ctypes.data_as(C.c_void_p), m, float(tol), _p(perm), _p(tau), C.byref(r11))
    return QRCP(r, perm, tau, W, r11.value)


def trsv(R: np.ndarray, x: np.ndarray, trans=False) -> np.ndarray:
    R = np.asfortranarray(R, dtype=np.float64)
    z = np.array(x, dtype=np.float64, copy=True)
    f = lib().orc_trsv_upper_t if trans else lib().orc_trsv_upper
    f(R.shape[0], R.ctypes.data_as(C.c_void_p), R.shape[0], _p(z))
    return z


# ---------------------------------------------------------------------------
# filtered system, LSQR (Algorithm 2)
# ---------------------------------------------------------------------------

class FilteredSystem:
    """Filtered blocks and their factors, packed for the oracle's operator.

    mode 0: Ahat S^-1 (Sec. 3.2); mode 1: the stored matrix as it is (either
    Ahat without preconditioner, or explicit Q_hat by Proposition 3.1)."""

    def __init__(self, N: int, grows, Ahats, Rs, mode=0, perms=None, K=None):
        self.N, self.J = N, len(grows)
        self.mode = mode
        self.m = np.array([len(g) for g in grows], dtype=np.int64)
        self.r = np.array([A.shape[1] for A in Ahats], dtype=np.int32)
        self.roff = np.concatenate([[0], np.cumsum(self.m)[:-1]]).astype(np.int64)
        self.coff = np.concatenate([[0], np.cumsum(self.r)[:-1]]).astype(np.int64)
        self.grow = np.concatenate(grows).astype(np.int64) if grows else np.zeros(0, np.int64)
        sizesA = self.m * self.r
        self.aoff = np.concatenate([[0], np.cumsum(sizesA)[:-1]]).astype(np.int64)
        self.Ahat = np.concatenate([np.asfortranarray(A).ravel(order="F") for A in Ahats] + [np.zeros(1)])
        rr = self.r.astype(np.int64) ** 2
        self.Roff = np.concatenate([[0], np.cumsum(rr)[:-1]]).astype(np.int64)
        self.Rv = np.concatenate([np.asfortranarray(R).ravel(order="F") for R in Rs] + [np.zeros(1)]) \
            if Rs is not None else np.zeros(1)
        self.perms = perms
        self.K = K
        self.n = int(self.r.sum())
        self._s = System(self.J, self.N, self.m.ctypes.data, self.roff.ctypes.data, self.grow.ctypes.data,
                         self.coff.ctypes.data, self.aoff.ctypes.data, self.Roff.ctypes.data,
                         self.r.ctypes.data, self.Ahat.ctypes.data, self.Rv.ctypes.data, mode)

    def matvec(self, x):
        out = np.zeros(self.N)
        x = np.ascontiguousarray(x, dtype=np.float64)
        lib().orc_op_apply(C.byref(self._s), _p(x), _p(out))
        return out

    def rmatvec(self, y):
        out = np.zeros(self.n + 1)
        y = np.ascontiguousarray(y, dtype=np.float64)
        lib().orc_op_apply_t(C.byref(self._s), _p(y), _p(out))
        return out[: self.n]

    def lsqr(self, h, y0=None, atol=1e-10, btol=1e-10, max_iter=10000, history=False):
        y = np.zeros(self.n + 1)
        st = np.zeros(6)
        hist = np.zeros(max_iter + 1) if history else None
        h = np.ascontiguousarray(h, dtype=np.float64)
        y0p = None
        if y0 is not None:
            y0a = np.zeros(self.n + 1)
            y0a[: self.n] = y0
            y0p = _p(y0a)
        lib().orc_lsqr(C.byref(self._s), _p(h), y0p, float(atol), float(btol), int(max_iter), _p(y), _p(st),
                       _p(hist) if history else None)
        out = dict(y=y[: self.n], itn=int(st[0]), istop=int(st[1]), rnorm=st[2], arnorm=st[3],
                   anorm=st[4], ynorm=st[5])
        if history:
            out["rhist"] = hist[: int(st[0]) + 1]
        return out

    def coefficients(self, y):
        """a = S^-1 y scattered to the J*K layout with zeros at dropped columns."""
        a = np.zeros(self.J * self.K)
        perm = np.ascontiguousarray(np.concatenate(self.perms), dtype=np.int32)
        yy = np.zeros(self.n + 1)
        yy[: self.n] = y
        lib().orc_coefficients(self.J, self.K, self.r.ctypes.data, _p(perm), self.coff.ctypes.data,
                               self.Roff.ctypes.data, self.Rv.ctypes.data, _p(yy), _p(a))
        return a


def filter_blocks(B: Blocks, tol: float, store_q=False):
    """Algorithm 1 over all blocks: returns per-block QRCP results."""
    return [qrcp(M, tol) for M in B.M]


def build_system(B: Blocks, F, mode=0, K=None) -> FilteredSystem:
    """Algorithm 2's operator: mode 0 = Ahat S^-1 with R from the filter;
    mode 1 = explicit Q_hat blocks (Proposition 3.1); mode 2 = Ahat alone."""
    K = K if K is not None else B.M[0].shape[1]
    perms = []
    for f in F:
        p = np.array(f.perm, dtype=np.int32)
        perms.append(p)
    if mode == 1:
        mats = [f.Q() for f in F]
        return FilteredSystem(B.N, B.grow, mats, None, mode=1, perms=perms, K=K)
    Ahats = [np.asfortranarray(M[:, f.perm[: f.rank]]) for M, f in zip(B.M, F)]
    if mode == 2:
        return FilteredSystem(B.N, B.grow, Ahats, None, mode=1, perms=perms, K=K)
    Rs = [f.R for f in F]
    return FilteredSystem(B.N, B.grow, Ahats, Rs, mode=0, perms=perms, K=K)


def coefficients_from(F, sysR: FilteredSystem, y):
    return sysR.coefficients(y)


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------

def test_grid(p, n_test=None):
    nt = list(n_test if n_test is not None else p.n_test)
    axes = [p.lo[i] + (np.arange(nt[i]) + 0.5) * (p.hi[i] - p.lo[i]) / nt[i] for i in range(p.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    # dimension 0 fastest
    return np.stack([m.transpose(list(range(p.dim))[::-1]).ravel() for m in mesh], axis=1)


def evaluate(p, params, a, X):
    s = problem_struct(p)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, p.dim)
    u = np.zeros(len(X))
    params = np.ascontiguousarray(params, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    lib().orc_eval(C.byref(s), _p(params), _p(a), len(X), _p(X), _p(u))
    return u


def errors(u_hat, u):
    """relative L2 error and the normalised L1 error e_L1 of Sec. 4.2."""
    d = u_hat - u
    return dict(rel_l2=float(np.linalg.norm(d) / np.linalg.norm(u)),
                e_l1=float(np.mean(np.abs(d)) / np.std(u)))


def solve(p, params, tol=1e-10, atol=1e-10, btol=1e-10, max_iter=10000, mode=0, fp32_matrix=False,
          y0=None, history=False):
    """Algorithm 2 end to end: assemble, filter, LSQR on the preconditioned
    system, a = S^-1 y with zeros at dropped columns.  fp32_matrix rounds the
    assembled blocks (and h) to FP32 first, as the mixed-precision GPU path
    does, then continues in FP64."""
    B = assemble(p, params)
    if fp32_matrix:
        B = Blocks(B.grow, [np.asfortranarray(M.astype(np.float32).astype(np.float64)) for M in B.M],
                   B.h.astype(np.float32).astype(np.float64), B.N)
    F = filter_blocks(B, tol)
    S = build_system(B, F, mode=0)
    res = S.lsqr(B.h, y0=y0, atol=atol, btol=btol, max_iter=max_iter, history=history)
    a = S.coefficients(res["y"])
    return dict(blocks=B, filt=F, system=S, a=a, **res)


# ---------------------------------------------------------------------------
# learned warm start: the network (plain loops in mlp_oracle.c) and the local
# fit of a predicted solution through each block's kept features
# ---------------------------------------------------------------------------

def feature_values(p, params, j, X):
    """phi_jk(x) for the K features of subdomain j at points X (npts x dim)."""
    s = problem_struct(p)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, p.dim)
    Phi = np.zeros((len(X), p.K), order="F")
    params = np.ascontiguousarray(params, dtype=np.float64)
    lib().orc_feature_values(C.byref(s), _p(params), int(j), len(X), _p(X), Phi.ctypes.data_as(C.c_void_p))
    return Phi


def _widths(widths):
    return (C.c_int * len(widths))(*[int(w) for w in widths])


def mlp_nparams(widths) -> int:
    return int(lib().orc_mlp_nparams(len(widths) - 1, _widths(widths)))


def mlp_forward(widths, theta, X):
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, widths[0])
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    Y = np.zeros(len(X))
    lib().orc_mlp_forward(len(widths) - 1, _widths(widths), _p(theta), len(X), _p(X), _p(Y))
    return Y


def mlp_grad(widths, theta, X, T):
    """(loss, gradient) of the mean squared error over the batch."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, widths[0])
    T = np.ascontiguousarray(T, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = np.zeros(len(theta))
    loss = lib().orc_mlp_grad(len(widths) - 1, _widths(widths), _p(theta), len(X), _p(X), _p(T), _p(g))
    return float(loss), g


def adam_step(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step(len(theta), _p(theta), _p(m), _p(v), _p(g), int(t), float(lr), float(b1), float(b2),
                        float(eps))


def _value_blocks(p, params, B: Blocks, F):
    """Window-weighted values of every block's kept features (pivot order of
    the system's filter) at the block's rows, and the window at those rows."""
    out, ws = [], []
    for j, (g, f) in enumerate(zip(B.grow, F)):
        X, _ = row_points(p, g)
        w = np.array([window(p, j, x)[0] for x in X])
        Phi = feature_values(p, params, j, X)[:, f.perm[: f.rank]]
        out.append(np.asfortranarray(w[:, None] * Phi))
        ws.append(w)
    return out, ws


def local_fit(p, params, B: Blocks, F, uhat, tol_fit=1e-10):
    """Warm start from predicted values, block by block: for every block j,
    the least-squares fit of w_j uhat[j] at the block's rows through its
    window-weighted kept features w_j phi_jk (pivot order), truncated by QR
    with column pivoting at tol_fit relative to |R_11|; then y0_j = R_j c_j,
    so that the preconditioned unknowns start at the fitted coefficients
    (a = S^-1 y).  Returns the list of y0_j and of the coefficients c_j."""
    V, ws = _value_blocks(p, params, B, F)
    ys, cs = [], []
    for j, f in enumerate(F):
        r = f.rank
        c = np.zeros(r)
        if r:
            G = qrcp(V[j], tol_fit)
            k = G.rank
            if k:
                z = G.Q().T @ (ws[j] * np.asarray(uhat[j], dtype=np.float64))
                c[G.perm[:k]] = trsv(G.R, z)
        cs.append(c)
        ys.append(f.R @ c if r else np.zeros(0))
    return ys, cs


def blend(p, B: Blocks, uhat):
    """u_bar(x_r) = sum_j w_j(x_r) uhat_j(x_r) over the blocks covering row r
    (the partition of unity applied to the per-block predictions)."""
    ub = np.zeros(B.N)
    for j, g in enumerate(B.grow):
        X, _ = row_points(p, g)
        w = np.array([window(p, j, x)[0] for x in X])
        ub[g] += w * np.asarray(uhat[j], dtype=np.float64)
    return ub


def global_fit(p, params, B: Blocks, F, uhat, tol_fit=1e-10, iters=100):
    """Warm start from predicted values through all blocks at once: the
    least-squares fit of the blended prediction u_bar at every collocation row
    by sum_j w_j phi_j c_j over the kept features, solved the paper's way --
    per block QR with column pivoting of the window-weighted values (threshold
    tol_fit), LSQR (iters iterations from zero) on the right-preconditioned
    fitting system, c = R_V^-1 z -- and finally y0_j = R_j c_j.  Returns y0_j,
    c_j per block and the LSQR result of the fit."""
    V, _ = _value_blocks(p, params, B, F)
    G = [qrcp(Vj, tol_fit) for Vj in V]
    fitsys = FilteredSystem(B.N, B.grow, [g.Q() for g in G], None, mode=1)
    res = fitsys.lsqr(blend(p, B, uhat), atol=0.0, btol=0.0, max_iter=iters)
    z = res["y"]
    ys, cs = [], []
    off = 0
    for f, g in zip(F, G):
        c = np.zeros(f.rank)
        k = g.rank
        if k:
            c[g.perm[:k]] = trsv(g.R, z[off:off + k])
        off += k
        cs.append(c)
        ys.append(f.R @ c if f.rank else np.zeros(0))
    return ys, cs, res
