"""Throughput of the warm-start network's kernels (forward pass and loss
gradient) on synthetic inputs, through the C ABI.

    python -m paper_2506_17626_gb300.mlp_bench [--n 4194304] [--reps 5] [--fp32]

Prints one JSON line: samples per second and TFLOP/s of each kernel, for the
9-128x4-1 network (2 x 50,945 flops per sample forward, three times that for
the gradient), CUDA-event timing after one warm-up call.  --fp32 selects the
CUDA-core kernels instead of the tensor-core ones.
"""
import argparse
import json

import torch

from . import _native as N
from .api import Mlp

WIDTHS = [9, 128, 128, 128, 128, 1]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--fp32", action="store_true")
    args = ap.parse_args()
    dev = torch.device("cuda:0")
    M = Mlp(WIDTHS, device=str(dev))
    g = torch.Generator(device=dev).manual_seed(0)
    th = torch.randn(M.n_params, device=dev, generator=g) * 0.3
    X = torch.rand((args.n, WIDTHS[0]), device=dev, generator=g) * 2 - 1
    T = torch.randn(args.n, device=dev, generator=g)
    out = {"network": "-".join(map(str, WIDTHS)), "n": args.n, "reps": args.reps,
           "kernels": "fp32" if args.fp32 else "tensor cores"}
    flops = 2.0 * M.n_params
    N.set_mlp_tensor_cores(not args.fp32)
    try:
        for name, fn, mult in (("forward", lambda: M.forward(th, X), 1.0), ("grad", lambda: M.grad(th, X, T), 3.0)):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) / args.reps / 1e3
            out[name] = {"ms": s * 1e3, "samples_per_s": args.n / s, "tflops": mult * flops * args.n / s / 1e12}
    finally:
        N.set_mlp_tensor_cores(True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
