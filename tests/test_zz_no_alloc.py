"""The allocation-free evaluation entry point against the workspace one.

rfm_eval_noalloc serves callers that cannot allocate device memory or keep a
workspace (code inside another framework's memory pool, plugin hosts that
only pass in their input and output buffers).  It keeps its scratch in a
static device array instead.  Here it is called twice in a row through the C
ABI and must give the same points and error sums as rfm_eval, within the
evaluation tolerance of the parity tests (1e-12 of the largest value); once
captured into a CUDA graph and replayed, after its coefficients have
changed in place, it must match rfm_eval at the new coefficients.
This file is collected last so that a run stopping at the first failure has
run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, probs, n, d_params, d_a, Xc, offs, u, err):
    lib.rfm_eval_noalloc.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 7
    lib.rfm_eval_noalloc.restype = C.c_int
    off_arr = (C.c_int64 * (n + 1))(*offs)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rfm_eval_noalloc(C.cast(probs, C.c_void_p), n, C.c_void_p(d_params.data_ptr()),
                                C.c_void_p(d_a.data_ptr()), C.c_void_p(Xc.data_ptr()),
                                C.cast(off_arr, C.c_void_p), C.c_void_p(u.data_ptr()),
                                C.c_void_p(err.data_ptr()), stream)


def test_noalloc_eval_matches_workspace_eval_twice():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N

    probs = [synth.poisson2d(S=4, K=20, n=17), synth.poisson1d(S=5, K=12, n=60)]
    prms = [synth.feature_params(p) for p in probs]
    S = R.System(probs, op="ar64", tol=1e-8)
    d_params = torch.from_numpy(np.concatenate([q.ravel() for q in prms])).cuda()
    S.assemble(d_params)
    rng = np.random.default_rng(5)
    d_a = torch.from_numpy(rng.standard_normal(S.sizes["n_cols"])).cuda()
    Xs = [torch.from_numpy(oracle.test_grid(p, [9] * p.dim)).cuda() for p in probs]
    ref_u, ref_err = S.evaluate(d_params, d_a, Xs)
    ref_u = torch.cat(ref_u)
    torch.cuda.synchronize()

    # the same points, padded to 3 coordinates, for the C call
    offs = [0]
    pts = []
    for x in Xs:
        x3 = torch.zeros((x.shape[0], 3), dtype=torch.float64, device="cuda")
        x3[:, : x.shape[1]] = x
        pts.append(x3)
        offs.append(offs[-1] + x.shape[0])
    Xc = torch.cat(pts).contiguous()
    lib = N.load()
    for call in range(2):
        u = torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda")
        err = torch.full((4 * len(probs),), float("nan"), dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, S._probs, len(probs), d_params, d_a, Xc, offs, u, err)
        assert rc == 0, lib.rfm_last_error()
        torch.cuda.synchronize()
        scale = max(1.0, float(ref_u.abs().max()))
        assert float((u - ref_u).abs().max()) <= 1e-12 * scale, call
        assert torch.allclose(err, ref_err, rtol=1e-12, atol=1e-12 * scale), call


def test_noalloc_eval_rejects_too_many_instances():
    from paper_2506_17626_gb300 import _native as N
    lib = N.load()
    probs = [synth.poisson1d(S=3, K=4, n=12) for _ in range(17)]
    arr = (N.RfmProblem * 17)(*[N.problem_struct(p) for p in probs])
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    offs = [0] * 18
    rc = _noalloc(lib, arr, 17, z, z, z, offs, z, z)
    assert rc == N.RFM_EINVAL
    assert b"at most 16" in lib.rfm_last_error()


def test_noalloc_eval_in_a_cuda_graph():
    from paper_2506_17626_gb300 import build
    build.build()
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N

    probs = [synth.poisson2d(S=4, K=20, n=17), synth.poisson1d(S=5, K=12, n=60)]
    prms = [synth.feature_params(p) for p in probs]
    S = R.System(probs, op="ar64", tol=1e-8)
    d_params = torch.from_numpy(np.concatenate([q.ravel() for q in prms])).cuda()
    S.assemble(d_params)
    rng = np.random.default_rng(7)
    d_a = torch.from_numpy(rng.standard_normal(S.sizes["n_cols"])).cuda()
    Xs = [torch.from_numpy(oracle.test_grid(p, [7] * p.dim)).cuda() for p in probs]
    offs, pts = [0], []
    for x in Xs:
        x3 = torch.zeros((x.shape[0], 3), dtype=torch.float64, device="cuda")
        x3[:, : x.shape[1]] = x
        pts.append(x3)
        offs.append(offs[-1] + x.shape[0])
    Xc = torch.cat(pts).contiguous()
    lib = N.load()
    u = torch.zeros(offs[-1], dtype=torch.float64, device="cuda")
    err = torch.zeros(4 * len(probs), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert _noalloc(lib, S._probs, len(probs), d_params, d_a, Xc, offs, u, err) == 0   # first call: uncaptured
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = _noalloc(lib, S._probs, len(probs), d_params, d_a, Xc, offs, u, err)
    assert rc == 0, lib.rfm_last_error()
    for trial in range(2):
        d_a.copy_(torch.from_numpy(rng.standard_normal(S.sizes["n_cols"])).cuda())
        u.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref_u, ref_err = S.evaluate(d_params, d_a, Xs)
        ref_u = torch.cat(ref_u)
        scale = max(1.0, float(ref_u.abs().max()))
        assert float((u - ref_u).abs().max()) <= 1e-12 * scale, trial
        assert torch.allclose(err, ref_err, rtol=1e-12, atol=1e-12 * scale), trial
