"""Benchmark: solve time to a fixed error for the RRQR-filtered, preconditioned
ELM-FBPINN solver on one GB300 (and N independent instances on N GPUs).

Workload (N = 1, the largest single-GPU configuration): (2+1)D heat
u_t = kappa Lap u on [0,1]^2 x [0,1], kappa = 0.01, u = exp(-2 kappa pi^2 k^2
t) sin(k pi x) sin(k pi y) with k = 6, 10 x 10 x 10 space-time subdomains
(overlap ratio 1.2), 500 tanh features each, 100^3 interior collocation points
plus 50,000 boundary and initial rows, filter threshold 1e-6, error on the
50^3 test grid.  --case p2d takes the 2D Poisson workload (20 x 20 subdomains,
300 features, 360^2 + 1440 rows, 400^2 test grid) instead; --case small a
heat instance with the same block shapes on 4 x 4 x 4 subdomains (profiler
captures).

A step is one pass of the whole path over one instance:
  assemble (FP32) -> RRQR filter (QR with column pivoting, Q_hat rounded to
  FP32) -> LSQR on Q_hat (FP32 products, FP64 vectors and scalars) for the
  iteration count that reaches the target error -> a = S^-1 y -> u_hat and
  its error on the test grid.
The target error and the iteration counts come from an untimed calibration
that records LSQR iterates every SNAP iterations up to the paper's budget of
10,000 iterations and evaluates each one; the target is the tightest value of
a fixed ladder that both the mixed path and the plain FP64 path (FP64
assembly, FP64 QR, explicit FP64 Q_hat of Proposition 3.1, zero start)
reach.  "solved" in the line says whether that target is at or below 1e-2;
above it the time is that of a solve that has not converged, and the line
says so.  Both paths are timed; "value" is the mixed path.

At N = 1 the line also carries, each measured in the same run: the 2D
Poisson workload's time to its target ("poisson2d"), the time to 1e-6
relative L2 error on the 1D Poisson workload, which converges, for the FP64
operators and the mixed path with refinement ("poisson1d"), many data sets
of a source family on one operator ("multi_rhs"), 64 uneven instances in
memory-budgeted waves ("batched"), the learned warm start
("learned"), and the oracle timed on a sample of the workload on one core and
on all cores ("cpu_baseline", "cpu_baseline_all_cores").  --impl reference
times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

TARGET_LADDER = [1e-6, 2e-6, 5e-6, 1e-5, 2e-5, 5e-5, 1e-4, 2e-4, 5e-4, 1e-3, 2e-3, 5e-3, 1e-2, 2e-2, 5e-2,
                 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.99]
SOLVED_AT = 1e-2
TOL = 1e-6
CAL_ITERS = 10000
# Nominal FP64 rate derived from the unit count and clock: 152 SMs x 4 FP64
# flop/clk/SM (2 DFMA lanes) x 2.07 GHz = 1258 GFLOP/s (a DFMA probe measured
# 1194 GFLOP/s on this part).
FP64_PEAK_GFLOPS = 152 * 4 * 2.07
# Ceiling of the cluster QR on FP32-assembled blocks, which runs in double-float
# arithmetic on the FP32 pipe: the issue rate (152 SMs x 4 schedulers x 32 lanes
# x 2.07 GHz = 40.3 T lane-instructions/s) over the 27 instructions of one
# column-update element (4 FP64-equivalent flops) = 5967 GFLOP/s.
DF_PEAK_GFLOPS = 152 * 4 * 32 * 2.07 * 4 / 27
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of ncu captures,
# per workload and kernel: a profile constant, not measured in this run.  Each
# entry names its capture (profiles/) and the SHA-256 prefix of the kernel's
# source file when it was taken; the line reports the traffic only while the
# source is unchanged (else null).  "per": iteration (scaled by the launch's
# iteration count) or launch.
NCU_TRAFFIC = {
    ("heat", "k_lsqr"): {"bytes": (984653102592 + 8471289088) / 200, "per": "iteration", "source": "csrc/lsqr.cu",
                         "sha16": "ae5c3b1d0a235697", "profile": "profiles/heat3d_10x10x10_K500_launches.md"},
}


def source_sha16(rel: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2506_17626_gb300", rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def workload(case: str = "heat"):
    """The benchmark's workload.  "small" keeps the heat blocks' shapes (same
    centre spacing and points per block) on 4 x 4 x 4 subdomains of the box
    [0, 1/3]^3, for profiler captures."""
    if case == "small":
        p = synth.heat3d(S=4, n=33)
        p.hi = (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)
        p.n_test = [20, 20, 20]
        return p
    if case == "p2d":
        return synth.poisson2d()
    return synth.heat3d()


def workload_name(p) -> str:
    if p.dim == 3:
        return (f"(2+1)D heat, {p.S[0]}x{p.S[1]}x{p.S[2]} space-time subdomains, delta {p.delta:g}, K={p.K}, "
                f"{p.n[0]}^3 interior + boundary/initial rows, kappa {p.kappa:g}, k=6, filter tol {TOL:g}, "
                f"error on {p.n_test[0]}^3 test grid")
    if p.dim == 2:
        return (f"2D Poisson {p.S[0]}x{p.S[1]} subdomains, delta {p.delta:g}, K={p.K}, {p.n[0]}^2 interior + "
                f"{4 * p.n[0]} boundary rows, filter tol {TOL:g}, error on {p.n_test[0]}^2 test grid")
    return f"1D Poisson, {p.S[0]} subdomains, delta {p.delta:g}, K={p.K}, {p.n[0]} interior + 2 boundary rows"


def instance_seed(base_seed: int, rank: int) -> int:
    """Seed of the instance rank `rank` solves: with N ranks every rank takes
    its own independent instance (weak scaling, no collective in the data
    path), seeds base_seed .. base_seed + N - 1."""
    return base_seed + rank


def max_over_ranks(v: float, world: int, device) -> float:
    """Largest value of `v` over the ranks (the job's time is its slowest
    rank's); a tensor on `device` (the rank's GPU under NCCL, the CPU under
    gloo) carries it through one all-reduce."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# accounting
# ---------------------------------------------------------------------------

def qrcp_flops(m: np.ndarray, K: int, r: np.ndarray) -> float:
    """Algorithmic flops of the Householder steps taken: sum_i<k 4 (m-i)(K-i)."""
    tot = 0.0
    for mj, rj in zip(m, r):
        i = np.arange(int(rj), dtype=np.float64)
        tot += float(np.sum(4.0 * (mj - i) * (K - i)))
    return tot


def formq_flops(m: np.ndarray, r: np.ndarray) -> float:
    tot = 0.0
    for mj, rj in zip(m, r):
        i = np.arange(int(rj), dtype=np.float64)
        tot += float(np.sum(4.0 * (mj - i) * (rj - i)))
    return tot


def lsqr_bytes_per_iter(m, r, N, val_bytes):
    nnz = float(np.sum(m * r))
    return 2.0 * nnz * val_bytes + 2.0 * (N + float(np.sum(r))) * 8.0


def smi_device_id(env=None) -> str:
    """nvidia-smi id of this rank's GPU: entry LOCAL_RANK of
    CUDA_VISIBLE_DEVICES when it is set (an index or a UUID), else the index
    LOCAL_RANK."""
    env = os.environ if env is None else env
    local = int(env.get("LOCAL_RANK", "0"))
    ids = [x.strip() for x in env.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
    return ids[local] if local < len(ids) else str(local)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            dev = smi_device_id()
            self.p = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, nm in enumerate(names):
            if any(r[5 + k].strip().lower() == "active" for r in rows if len(r) > 5 + k):
                reasons.append(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def calibrate(S, d_prm, Xt, cal_iters, every, dev):
    """Zero-start LSQR for cal_iters iterations, the iterate every `every`
    iterations evaluated (relative L2 on the test grid) and the residual of
    the assembled system at it (FP64); returns (errors, residuals, kept)."""
    import torch
    S.assemble(d_prm)
    rank = S.filter()
    cap = cal_iters // every
    snap = torch.zeros((cap, S.sizes["n_cols"]), dtype=torch.float64, device=dev)
    S.solve(atol=0, btol=0, max_iter=cal_iters, snap=snap, snap_every=every)
    errs, res = [], []
    for k in range(cap):
        a_k = S.coefficients(snap[k])
        _, err = S.evaluate(d_prm, a_k, [Xt])
        e = err.cpu().numpy()
        errs.append(float(np.sqrt(e[0] / e[1])))
        res.append(float(S.residual(a_k)[0].item()))
    del snap
    return np.array(errs), np.array(res), int(rank.sum().item())


def time_to_error(p, args, dev, world, rank_id, headline):
    """Both paths (mixed: FP32 assembly and Q_hat; FP64: FP64 assembly, QR
    and Q_hat) on workload p: calibration, target, timed steps, kernel
    profile.  `headline` adds the end-to-end run through host buffers."""
    import torch
    import torch.distributed as dist
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N

    prm = synth.feature_params(p)
    h_prm = torch.from_numpy(prm.ravel()).pin_memory()
    d_prm = h_prm.to(dev)
    Xt = torch.from_numpy(oracle_free_test_grid(p)).to(dev)
    paths = {"mixed": R.System([p], asm="fp32", op="q32", tol=TOL, device=str(dev)),
             "fp64": R.System([p], asm="fp64", op="q64", tol=TOL, device=str(dev))}
    every = args.snap_every
    curves, resid, conv = {}, {}, {}
    if args.iters_mixed is None:
        for name, S in paths.items():
            e, r, kept = calibrate(S, d_prm, Xt, args.cal_iters, every, dev)
            curves[name], resid[name] = e, r
            conv[name] = {"min_rel_l2": float(e.min()), "at_iteration": every * (1 + int(e.argmin())),
                          "rel_l2_at_end": float(e[-1]), "kept_columns": kept,
                          "rel_l2_history": [float(v) for v in e[:: max(1, len(e) // 20)]],
                          "residual_history": [float(v) for v in r[:: max(1, len(r) // 20)]],
                          "history_every": every * max(1, len(e) // 20)}
            log(f"[cal] {p.name} {name}: min rel L2 {e.min():.3e} at it {every * (1 + int(e.argmin()))}")
        target = None
        for t in TARGET_LADDER:
            if all((c <= t).any() for c in curves.values()):
                target = t
                break
        if target is None:
            target = float(max(c.min() for c in curves.values())) * 1.01
        kstar = {n: every * (1 + int(np.argmax(c <= target))) for n, c in curves.items()}
    else:
        kstar = {"mixed": args.iters_mixed, "fp64": args.iters_fp64 or args.iters_mixed}
        target = args.target
    log(f"[cal] {p.name}: target {target}, iterations {kstar}")

    st = torch.cuda.current_stream()

    def step(S, k, e2e=False):
        if e2e:
            d_prm.copy_(h_prm, non_blocking=True)
        S.assemble(d_prm)
        S.filter()
        a, rep = S.solve(atol=0, btol=0, max_iter=k)
        _, err = S.evaluate(d_prm, a, [Xt])
        if e2e:
            a_h = torch.empty(a.numel(), dtype=torch.float64, pin_memory=True)
            e_h = torch.empty(err.numel(), dtype=torch.float64, pin_memory=True)
            a_h.copy_(a, non_blocking=True)
            e_h.copy_(err, non_blocking=True)
            return a, err, a_h, e_h
        return a, err

    def timed(S, k, steps, warm, e2e=False, prof=False):
        for _ in range(warm):
            step(S, k, e2e)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if prof:
            N.profile_reset()
            N.profile_enable(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(st)
        outs = None
        for i in range(steps):
            outs = step(S, k, e2e)
            ev[i + 1].record(st)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        prof_data = None
        if prof:
            N.profile_enable(False)
            prof_data = N.profile_read()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        return per, outs, prof_data

    steps_m = args.steps if headline else min(args.steps, 3)
    warm_m = args.warmup if headline else max(1, min(args.warmup, 2))
    steps_f = min(args.steps, 3) if headline else min(args.steps, 2)
    clk = None
    if headline:
        with Clocks(args.clocks_log) as clk:
            per_mixed, outs, prof = timed(paths["mixed"], kstar["mixed"], steps_m, warm_m, prof=True)
    else:
        per_mixed, outs, prof = timed(paths["mixed"], kstar["mixed"], steps_m, warm_m, prof=True)
    per_fp64, outs64, _ = timed(paths["fp64"], kstar["fp64"], steps_f, 1)
    out = {"workload": workload_name(p), "target_rel_l2": target, "solved": bool(target <= SOLVED_AT),
           "iterations": kstar}
    if target > SOLVED_AT:
        out["note"] = (f"no path reaches {SOLVED_AT:g} relative L2 within {args.cal_iters} LSQR iterations: the "
                       f"times are those of solves that have not converged (tightest common error {target:g})")
    err_m, err_f = outs[1].cpu().numpy(), outs64[1].cpu().numpy()
    out["rel_l2_reached"] = {"mixed": float(np.sqrt(err_m[0] / err_m[1])), "fp64": float(np.sqrt(err_f[0] / err_f[1]))}
    out["convergence"] = conv
    ms_mixed = max_over_ranks(float(np.mean(per_mixed)), world, dev)
    ms_fp64 = max_over_ranks(float(np.mean(per_fp64)), world, dev)
    out.update({"ms_mixed": ms_mixed, "ms_fp64": ms_fp64, "steps_mixed": steps_m, "steps_fp64": steps_f})
    if headline:
        per_e2e, _, _ = timed(paths["mixed"], kstar["mixed"], steps_f, 1, e2e=True)
        out["e2e"] = {"value": max_over_ranks(float(np.mean(per_e2e)), world, dev), "unit": "ms",
                      "h2d_bytes_per_step": int(h_prm.numel() * 8),
                      "d2h_bytes_per_step": int(paths["mixed"].sizes["n_cols"] * 8 + 4 * 8),
                      "steps": steps_f}
        out["clocks"] = clk.summary() if clk else None

    # ---- rates and the roofline of the dominant kernel (mixed path)
    S = paths["mixed"]
    ranks = S.filter().cpu().numpy()
    m = S.block_table()[0]
    K = p.K
    tot = dict(prof)
    per_launch_ms = {k: v[1] / v[0] for k, v in tot.items()}
    out["kernels_ms_per_step"] = {k: v[1] / steps_m for k, v in tot.items()}
    out["gpu_launches"] = int(sum(v[0] for v in tot.values()))
    dom = max(tot, key=lambda k: tot[k][1])
    qr_names = [k for k in ("k_qrcp_cluster", "k_qrcp", "k_form_q") if k in per_launch_ms]
    qr_ms = sum(per_launch_ms[k] for k in qr_names)
    fused_q = "k_qrcp_cluster" in per_launch_ms
    qr_alg = qrcp_flops(m, K, ranks) + formq_flops(m, ranks)
    out["qr_gflops"] = qr_alg / (qr_ms * 1e-3) / 1e9
    lsqr_by = lsqr_bytes_per_iter(m, ranks, S.sizes["n_rows"], 4) * kstar["mixed"]
    out["spmv_gbs"] = lsqr_by / (per_launch_ms["k_lsqr"] * 1e-3) / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    if dom in ("k_qrcp_cluster", "k_qrcp", "k_form_q"):
        # the QR and the formation of Q_hat: algorithmic flops over their time
        ach = qr_alg / (qr_ms * 1e-3) / 1e12
        if fused_q:
            pk, src = DF_PEAK_GFLOPS / 1e3, ("derived double-float: FP32 issue 152 SMs x 4 x 32 lanes x 2.07 GHz / "
                                             "27 instructions per 4-flop update element")
        else:
            pk, src = FP64_PEAK_GFLOPS / 1e3, "derived FP64: 152 SMs x 4 flop/clk x 2.07 GHz (DFMA probe 1.19)"
        roof = {"kernel": "+".join(qr_names), "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "peak_source": src, "algorithmic_per_launch": qr_alg,
                "algorithmic": "sum over blocks and QR steps i < r_j of 4 (m_j - i)(K - i), plus 4 (m_j - i)(r_j - i) "
                               "for Q_hat"}
    else:
        ach = lsqr_by / (per_launch_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "algorithmic_per_launch": lsqr_by,
                "algorithmic": "2 nnz(Q_hat) x 4 B + 2 (N + sum r_j) x 8 B per iteration x iterations"}
    case = "heat" if p.dim == 3 else ("p2d" if p.dim == 2 else "p1d")
    tr = NCU_TRAFFIC.get((case, dom))
    roof["traffic"] = None
    if tr is not None and source_sha16(tr["source"]) == tr["sha16"]:
        per = kstar["mixed"] if tr["per"] == "iteration" else 1
        roof["traffic"] = tr["bytes"] * per
        roof["traffic_source"] = (f"profile constant: ncu capture {tr['profile']} of the same kernel source "
                                  f"(sha256 {tr['sha16']}), scaled per {tr['per']}")
        if roof["bound"] == "hbm":
            dram = roof["traffic"] / (per_launch_ms[dom] * 1e-3) / 1e9
            roof["dram_achieved"] = dram
            roof["dram_frac"] = dram / peaks["hbm_gbs"]
    out["roofline"] = roof
    return out, paths


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2506_17626_gb300 import build as B
    B.build()
    from paper_2506_17626_gb300 import _native as N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    # the QR cluster size is autotuned on the first filter call of each block
    # shape (untimed: calibration or warm-up) unless --no-autotune
    N.set_autotune(not args.no_autotune)

    p = workload(args.case)
    if world > 1:           # independent instances, one per rank (weak scaling)
        p.seed = instance_seed(p.seed, rank)
    head, paths = time_to_error(p, args, dev, world, rank, headline=True)
    out = {
        "metric": "solve time to fixed error (mixed FP32/FP64, zero start)",
        "value": head["ms_mixed"], "unit": "ms", "n_gpus": world, "steps": head["steps_mixed"],
        "warmup": args.warmup, "ms_per_step": head["ms_mixed"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": head["workload"], "target_rel_l2": head["target_rel_l2"], "solved": head["solved"],
                   "iterations": head["iterations"], "rel_l2_reached": head["rel_l2_reached"],
                   "convergence_10000_iterations": head["convergence"],
                   "l2_flush": "none: the working set (M, QR work, Q_hat: > 1.5 GB) exceeds L2 every step",
                   "parallelism": f"independent instances x{world}" if world > 1 else "1 instance",
                   "qr_cluster_autotune": not args.no_autotune},
        "fp64_zero_start_ms": head["ms_fp64"],
        "qr_gflops": head["qr_gflops"], "spmv_gbs": head["spmv_gbs"],
        "kernels_ms_per_step": head["kernels_ms_per_step"],
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"],
    }
    if "note" in head:
        out["config"]["note"] = head["note"]
    del paths
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        prm = synth.feature_params(p)
        out["cpu_baseline"] = cpu_baseline(p, prm, head["iterations"]["fp64"], stride=args.cpu_stride)
        out["cpu_baseline_all_cores"] = guarded(cpu_baseline_pool, p, prm, head["iterations"]["fp64"],
                                                args.cpu_stride_pool, out["cpu_baseline"])
    if rank == 0 and world == 1 and args.case != "p2d" and not args.no_p2d:
        sec = guarded(lambda: time_to_error(synth.poisson2d(), args, dev, 1, 0, headline=False)[0])
        out["poisson2d"] = sec
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_poisson1d:
        out["poisson1d"] = guarded(run_poisson1d, args, dev)
    if rank == 0 and world == 1 and args.multi_rhs > 0:
        out["multi_rhs"] = guarded(run_multi_rhs, args, dev)
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.batched > 0:
        out["batched"] = guarded(run_batched, args, dev)
        N.set_autotune(not args.no_autotune)   # also when the section failed part-way
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and args.learned_train > 0:
        out["learned"] = guarded(run_learned, args, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, dev):
    """The batched family: 64 instances of uneven size (per instance seeded S
    in [8, 24]^2 subdomains, K in [100, 400] features, four separable sine
    modes) with p_lo..p_hi points per subdomain edge, mixed path, a fixed
    number of LSQR iterations.  Instances run side by side, one launch per
    call of the path, in memory-budgeted waves (consecutive systems whose
    workspace fits the budget).  Phase times by CUDA events; the first
    wave's filter also in block order (RFM_OPT_QR_ORDER = 0)."""
    import copy
    import torch
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N
    from paper_2506_17626_gb300.waves import plan_waves
    n_inst, iters = args.batched, args.batched_iters
    p_lo, p_hi = (int(v) for v in args.batched_points.split(","))
    probs = [synth.batched_instance(i, p_range=(p_lo, p_hi)) for i in range(n_inst)]
    budget = int(args.batched_budget * 288e9)
    waves = plan_waves(probs, budget)
    # every wave is a new block shape: the QR autotuner would time its
    # variants inside each wave's timed filter, so this section runs the
    # library's default variants (32 warps per block, panels of 8)
    N.set_autotune(False)
    totals = {"assemble": 0.0, "filter": 0.0, "lsqr": 0.0, "eval": 0.0, "step": 0.0}
    rel, m_all, r_all, K_all, per_wave = [], [], [], [], []
    rows = cols = kept = nnz = 0
    lsqr_bytes = 0.0
    order_ms = None
    for wi, idx in enumerate(waves):
        ps = [probs[i] for i in idx]
        d = torch.from_numpy(np.concatenate([synth.feature_params(p).ravel() for p in ps])).to(dev)
        grids = []
        for p in ps:
            q = copy.copy(p)
            q.n_test = [100, 100]
            grids.append(torch.from_numpy(oracle_free_test_grid(q)).to(dev))
        S = R.System(ps, asm="fp32", op="q32", tol=TOL, device=str(dev))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]

        def step(timed):
            if timed:
                ev[0].record()
            S.assemble(d)
            if timed:
                ev[1].record()
            rank = S.filter()
            if timed:
                ev[2].record()
            a, rep = S.solve(atol=0, btol=0, max_iter=iters)
            if timed:
                ev[3].record()
            _, err = S.evaluate(d, a, grids)
            if timed:
                ev[4].record()
            return rank, err

        if wi == 0:
            step(False)       # module loading and first-launch costs stay out of the timing
        rank, err = step(True)
        if wi == 0:
            N.set_qr_order(False)
            try:
                ev[5].record()
                S.filter()
                ev[6].record()
            finally:
                N.set_qr_order(True)
        torch.cuda.synchronize()
        ms = {"assemble": ev[0].elapsed_time(ev[1]), "filter": ev[1].elapsed_time(ev[2]),
              "lsqr": ev[2].elapsed_time(ev[3]), "eval": ev[3].elapsed_time(ev[4]), "step": ev[0].elapsed_time(ev[4])}
        if wi == 0:
            order_ms = ev[5].elapsed_time(ev[6])
        for k in totals:
            totals[k] += ms[k]
        e = err.cpu().numpy().reshape(len(ps), 4)
        rel += list(np.sqrt(e[:, 0] / e[:, 1]))
        m_blk = S.block_table()[0]
        r_blk = rank.cpu().numpy().astype(np.int64)
        K_blk = np.repeat([p.K for p in ps], [p.J for p in ps])
        m_all.append(m_blk)
        r_all.append(r_blk)
        K_all.append(K_blk)
        rows += int(S.sizes["n_rows"])
        cols += int(S.sizes["n_cols"])
        kept += int(r_blk.sum())
        nnz += int((m_blk * r_blk).sum())
        lsqr_bytes += lsqr_bytes_per_iter(m_blk, r_blk, S.sizes["n_rows"], 4) * iters
        per_wave.append({"instances": len(ps), "workspace_gb": S.sizes["workspace_bytes"] / 1e9, "ms": ms})
        del S, d, grids
        torch.cuda.empty_cache()
    N.set_autotune(not args.no_autotune)
    m_blk, r_blk, K_blk = np.concatenate(m_all), np.concatenate(r_all), np.concatenate(K_all)
    i = [np.arange(int(rj), dtype=np.float64) for rj in r_blk]
    qr_fl = float(sum(np.sum(4.0 * (mj - ii) * (Kj - ii) + 4.0 * (mj - ii) * (rj - ii))
                      for mj, Kj, rj, ii in zip(m_blk, K_blk, r_blk, i)))
    rel = np.array(rel)
    ws_all = sum(w["workspace_gb"] for w in per_wave) * 1e9
    return {
        "workload": f"batched 2D Poisson: {n_inst} instances, S in [8, 24]^2, K in [100, 400], "
                    f"{p_lo}-{p_hi} points per subdomain edge, 4 separable sine modes; mixed path, filter tol {TOL:g}, "
                    f"{iters} LSQR iterations, error on a 100^2 grid per instance",
        "point_range_note": "the family's 40-200 points per edge need 2.75 TB of workspace (blocks of up to 62,500 "
                            "rows); this section runs the 40-60 fraction of that range in memory-budgeted waves",
        "waves": len(waves), "budget_gb": budget / 1e9, "workspace_gb_total": ws_all / 1e9, "per_wave": per_wave,
        "blocks": int(len(m_blk)), "rows": rows, "columns": cols, "kept_columns": kept,
        "ms": {**totals, "filter_block_order_first_wave": order_ms},
        "qr_variants": "defaults (no autotuning: every wave is a new block shape)",
        "ms_per_lsqr_iteration": totals["lsqr"] / iters, "nnz_q_hat": nnz,
        "lsqr_gbs_algorithmic": lsqr_bytes / (totals["lsqr"] * 1e-3) / 1e9,
        "qr_gflops_algorithmic": qr_fl / (totals["filter"] * 1e-3) / 1e9,
        "rel_l2": {"median": float(np.median(rel)), "max": float(rel.max())},
    }


def run_multi_rhs(args, dev):
    """Many right-hand sides on one operator: the parametric source family on
    the 20 x 20 x 300 decomposition (overlap ratio 1.25, 360^2 interior +
    1440 boundary rows, mixed path, filter tol 1e-6), nrhs data sets solved
    at once (rfm_lsqr_multi) against one data set at a time (rfm_lsqr_solve),
    a fixed number of LSQR iterations each; CUDA events after one untimed
    call of each."""
    import torch
    import paper_2506_17626_gb300 as R
    nrhs, iters = args.multi_rhs, args.multi_iters
    probs = [synth.param5(*synth.param5_draw(s), S=20, K=300, n=360, delta=1.25) for s in range(nrhs)]
    prm = torch.from_numpy(synth.feature_params(probs[0]).ravel()).to(dev)
    out = {"workload": f"2D Poisson source family f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y) on 20x20 "
                       f"subdomains, delta 1.25, K=300, 360^2 + 1440 rows, filter tol {TOL:g}; {nrhs} data sets, "
                       f"{iters} LSQR iterations", "nrhs": nrhs, "iterations": iters}
    for asm, op in (("fp32", "q32"), ("fp64", "q64")):
        S = R.System([probs[0]], asm=asm, op=op, tol=TOL, device=str(dev))
        S.assemble(prm)
        rank = S.filter()
        H = S.rhs_many(probs)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        S.solve_multi(H, atol=0, btol=0, max_iter=2)
        ev[0].record()
        A, rep = S.solve_multi(H, atol=0, btol=0, max_iter=iters)
        ev[1].record()
        S.solve(atol=0, btol=0, max_iter=2)
        ev[2].record()
        S.solve(atol=0, btol=0, max_iter=iters)
        ev[3].record()
        torch.cuda.synchronize()
        m = S.block_table()[0]
        r = rank.cpu().numpy()
        nnz = float(np.sum(m * r))
        t_multi = ev[0].elapsed_time(ev[1])
        t_single = ev[2].elapsed_time(ev[3])
        flops = 4.0 * nnz * nrhs * iters
        out[op] = {"ms_multi": t_multi, "ms_single_one_data_set": t_single,
                   "rhs_iterations_per_s_multi": nrhs * iters / (t_multi * 1e-3),
                   "rhs_iterations_per_s_single": iters / (t_single * 1e-3),
                   "speedup_per_data_set": nrhs * t_single / t_multi,
                   "block_product_tflops": flops / (t_multi * 1e-3) / 1e12,
                   "nnz_q_hat": nnz}
        del S, H, A
        torch.cuda.empty_cache()
    return out


def run_poisson1d(args, dev):
    """Time to 1e-6 relative L2 error on the 1D Poisson workload (-u'' = f on
    [0,1], u = sin 2 pi x + 0.1 sin 50 pi x, 20 subdomains, overlap ratio
    1.3, K = 100, 1600 interior points), which, unlike the 2D and heat
    workloads, reaches it.  Calibration (untimed): zero-start LSQR for 10,000
    iterations, the iterate evaluated every 100, for plain LSQR on the
    unfiltered M and for the filtered, preconditioned solver at threshold
    1e-8 with three operators: the paper's form (FP64 kept columns and
    R_hat^-1 substitution, ar64), the explicit FP64 Q_hat (q64, FP64 path),
    and the mixed path's FP32 Q_hat (FP64 blocks factored in double-float;
    also with one to three refinement steps on the FP64 residual, each
    correction solve as long as the first).  Timed (CUDA
    events, after warm-up): assemble -> filter -> LSQR for the first
    recorded iteration count at 1e-6 -> a = S^-1 y -> u_hat and its error,
    for each run that reaches 1e-6."""
    import torch
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N
    from paper_2506_17626_gb300 import sweep as SW
    p = synth.poisson1d()
    prm = torch.from_numpy(synth.feature_params(p).ravel()).to(dev)
    X = torch.from_numpy(SW.grid_points(p)).to(dev)
    sig = 1e-8
    st = torch.cuda.current_stream()
    out = {"workload": "1D Poisson, 20 subdomains, delta 1.3, K=100, 1600 interior + 2 boundary rows, "
                       "error on 1000 test points", "target_rel_l2": 1e-6, "sigma": sig, "runs": []}
    specs = [("plain", "fp64", "plain", 1), ("paper operator (ar64), FP64", "fp64", "ar64", 1),
             ("explicit Q_hat (q64), FP64", "fp64", "q64", 1),
             ("mixed: FP32 Q_hat (q32), FP64 blocks, double-float QR", "fp64", "q32", 2)]

    def timed_step(S, k, refine=0, refine_iters=0):
        def step():
            S.assemble(prm)
            S.filter()
            a, _ = S.solve(atol=0.0, btol=0.0, max_iter=k, refine_steps=refine, refine_iters=refine_iters)
            return S.evaluate(prm, a, [X])[1]
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        n = max(1, min(args.steps, 10))
        ev[0].record(st)
        for _ in range(n):
            err = step()
        ev[1].record(st)
        torch.cuda.synchronize()
        e = SW.errors_from_sums(err.cpu().numpy(), X.shape[0])
        return ev[0].elapsed_time(ev[1]) / n, e["rel_l2"]

    for label, asm, op, qdf in specs:
        N.set_qr_double_float(qdf)
        try:
            r = SW.run_one(p, prm, X, asm, op, 0.0 if op == "plain" else sig, 10000, 100, dev)
            row = {"run": label, **{k: r[k] for k in ("op", "sigma", "dropped_pct", "min_rel_l2", "min_rel_l2_at",
                                                       "min_e_l1", "iterations_to", "lsqr_ms")}}
            k = r["iterations_to"]["1e-06"]
            S = R.System([p], asm=asm, op=op, tol=0.0 if op == "plain" else sig, device=str(dev))
            if k is not None:
                t, e = timed_step(S, k)
                row.update({"iterations": k, "time_to_target_ms": t, "rel_l2_reached": e})
            if op == "q32":
                # correction solves as long as the first one (this operator's
                # own iteration count to 1e-4): shorter ones stop before LSQR
                # has started to converge on it
                k1 = r["iterations_to"]["0.0001"] or 3000
                ref = []
                for nref in (1, 2, 3):
                    t, e = timed_step(S, k1, refine=nref, refine_iters=k1)
                    ref.append({"iterations": f"{k1} + {nref} x {k1}", "ms": t, "rel_l2": e})
                    if e <= 1e-6:
                        break
                row["refined"] = {"runs": ref, "reaches_target": ref[-1]["rel_l2"] <= 1e-6}
                if ref[-1]["rel_l2"] <= 1e-6:
                    row["time_to_target_ms_refined"] = ref[-1]["ms"]
            del S
        finally:
            N.set_qr_double_float(1)
        out["runs"].append(row)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_p1d(p, out["runs"], sig)
    return out


def cpu_baseline_p1d(p, runs, sig):
    """The oracle as it stands on one host core, the whole 1D step (assembly,
    QR with column pivoting, LSQR for the GPU run's iteration count to 1e-6,
    coefficients, evaluation on the test points), for the two FP64 operator
    forms that reach 1e-6.  Not sampled."""
    import oracle
    from paper_2506_17626_gb300 import sweep as SW
    prm = synth.feature_params(p)
    X = SW.grid_points(p)
    ue = oracle.exact(p, X)
    res = {"kind": "oracle", "cores": 1, "sample": "the whole step, not sampled", "runs": {}}
    for r in runs:
        k = r.get("iterations")
        if r["op"] not in ("ar64", "q64") or not k:
            continue
        t0 = time.perf_counter()
        B = oracle.assemble(p, prm)
        F = oracle.filter_blocks(B, sig)
        S0 = oracle.build_system(B, F, mode=0)
        So = S0 if r["op"] == "ar64" else oracle.build_system(B, F, mode=1)
        y = So.lsqr(B.h, atol=0, btol=0, max_iter=k)["y"]
        u = oracle.evaluate(p, prm, S0.coefficients(y), X)
        ms = (time.perf_counter() - t0) * 1e3
        res["runs"][r["op"]] = {"ms": ms, "iterations": k,
                                "rel_l2": float(np.linalg.norm(u - ue) / np.linalg.norm(ue)),
                                "gpu_ms": r.get("time_to_target_ms")}
    return res


def guarded(fn, *a):
    """A section of the JSON line that reports its failure instead of
    aborting the benchmark."""
    try:
        return fn(*a)
    except Exception as exc:           # noqa: BLE001
        return {"error": f"{type(exc).__name__}: {exc}"}


def run_learned(args, dev):
    """The learned warm start on the parametric-source family (held-out
    instances): training solves by the mixed path, the network trained by the
    library's kernels, then LSQR from zero and from the fitted prediction.
    Errors are relative L2 on a 100^2 grid against a long FP64 solve."""
    import math
    import torch
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300.warm import LearnedWarmStart, block_row_mask, instance_row_ranges
    S_, K_, D_ = 10, 120, 2.9
    n = S_ * math.ceil(math.sqrt(K_))
    base = dict(S=S_, K=K_, delta=D_, n=n)
    fam = lambda seeds: [synth.param5(*synth.param5_draw(s), **base) for s in seeds]
    ctx = lambda ps: torch.from_numpy(np.stack([synth.param5_context(p.fparams) for p in ps])).to(dev)
    scl = lambda ps: [synth.param5_amplitude_scale(p.fparams) for p in ps]
    prm0 = synth.feature_params(fam([0])[0])
    params = lambda ps: torch.from_numpy(np.tile(prm0.ravel(), len(ps))).to(dev)
    ax = (np.arange(100) + 0.5) / 100
    gx, gy = np.meshgrid(ax, ax, indexing="xy")
    grid = torch.from_numpy(np.stack([gx.ravel(), gy.ravel()], 1)).to(dev)

    def rel(u, r):
        return [float(torch.linalg.norm(ui - ri) / torch.linalg.norm(ri)) for ui, ri in zip(u, r)]

    ntr, train_iters, epochs = args.learned_train, 3000, args.learned_epochs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, Ts = [], []
    tr = fam(range(ntr))
    # the family shares the operator: its solves run 256 data sets at a time
    # on one system (rfm_lsqr_multi), mixed path
    S0 = R.System([tr[0]], asm="fp32", op="q32", tol=TOL, device=str(dev))
    d0 = params(tr[:1])
    S0.assemble(d0)
    S0.filter()
    t_solve = 0.0
    for i in range(0, ntr, 256):
        ps = tr[i:i + 256]
        H = S0.rhs_many(ps)
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record()
        A, _ = S0.solve_multi(H, atol=0, btol=0, max_iter=train_iters)
        e1_.record()
        torch.cuda.synchronize()
        t_solve += e0_.elapsed_time(e1_) / 1e3
        for j, p in enumerate(ps):
            X, T = LearnedWarmStart.samples(S0, d0, A[j].contiguous(), ctx([p]), inst_scale=scl([p]))
            Xs.append(X)
            Ts.append(T)
        del H, A
    X, T = torch.cat(Xs), torch.cat(Ts)
    del S0, Xs, Ts
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    W = LearnedWarmStart([9, 128, 128, 128, 128, 1], seed=0, device=str(dev))
    scale = float(T.abs().max())
    t0 = time.perf_counter()
    hist = W.train(X, T / scale, epochs=epochs, batch=4096, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    W.theta[-129:] *= scale
    n_samples = int(X.shape[0])
    del X, T
    # forward throughput of the network (the tensor-core kernel for this shape), 2^22 samples
    Xf = torch.empty((1 << 22, 9), device=dev).uniform_(-1, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    W.net.forward(W.theta, Xf)
    ev0.record()
    for _ in range(5):
        W.net.forward(W.theta, Xf)
    ev1.record()
    torch.cuda.synchronize()
    fwd_s = ev0.elapsed_time(ev1) / 5e3
    fwd = {"samples_per_s": Xf.shape[0] / fwd_s, "tflops": 2.0 * W.net.n_params * Xf.shape[0] / fwd_s / 1e12,
           "kernel": "k_mlp_fwd_tc (tcgen05, BF16 operands, FP32 accumulation)"}
    del Xf

    held = fam(range(10000, 10000 + args.learned_heldout))
    d = params(held)
    Xt = [grid for _ in held]
    R64 = R.System(held, asm="fp64", op="q64", tol=TOL, device=str(dev))
    R64.assemble(d)
    R64.filter()
    a_ref, _ = R64.solve(atol=0, btol=0, max_iter=10000)
    u_ref, _ = R64.evaluate(d, a_ref, Xt, with_error=False)
    S = R.System(held, asm="fp32", op="q32", tol=TOL, device=str(dev))
    S.assemble(d)
    S.filter()
    S.fit_prepare(d, tol_fit=1e-8)
    # prediction error at the block rows against the reference there
    _, pts = S.block_inputs(ctx(held))
    rr = instance_row_ranges(S)
    ub, _ = R64.evaluate(d, a_ref, [pts[r0:r1, :2].contiguous() for r0, r1 in rr], with_error=False)
    live = block_row_mask(S)
    inv = torch.tensor([1.0 / v for v in scl(held)], dtype=torch.float32, device=dev)
    pred = W.predict(S, ctx(held))
    scale_rows = torch.cat([torch.full((r1 - r0,), float(inv[i]), device=dev) for i, (r0, r1) in enumerate(rr)])
    pl = (pred.double() * scale_rows).index_select(0, live)
    tl = torch.cat(ub).index_select(0, live)
    pred_err = float(torch.linalg.norm(pl - tl) / torch.linalg.norm(tl))
    ev0.record()
    y0 = W.warm_start(S, ctx(held), fit_iters=300, inst_scale=inv)
    ev1.record()
    torch.cuda.synchronize()
    t_ws = ev0.elapsed_time(ev1)
    u0, _ = S.evaluate(d, S.coefficients(y0), Xt, with_error=False)
    e0 = rel(u0, u_ref)
    every, iters = 100, 3000
    curves, med, ms_it, used = {}, {}, {}, 0
    for name, yy in (("zero_start", None), ("learned_start", y0)):
        snap = torch.zeros((iters // every, S.sizes["n_cols"]), dtype=torch.float64, device=dev)
        ev0.record()
        _, rep = S.solve(atol=0, btol=0, max_iter=iters, snap=snap, snap_every=every, y0=yy)
        ev1.record()
        torch.cuda.synchronize()
        ms_it[name] = ev0.elapsed_time(ev1) / iters
        if yy is not None:
            used = sum(R.report_dict(rep, i)["start"] for i in range(len(held)))
        errs = np.array([rel(S.evaluate(d, S.coefficients(snap[k]), Xt, with_error=False)[0], u_ref)
                         for k in range(snap.shape[0])])
        curves[name] = errs.max(axis=1)
        med[name] = np.median(errs, axis=1)

    def first(c, th):
        k = np.nonzero(c <= th)[0]
        return int(every * (1 + k[0])) if len(k) else None

    # many held-out instances: the family shares its operator, so the fitted
    # starts (32 instances per fitting system) and LSQR for all of them run
    # as one many-data-set solve, from zero and from the fitted starts
    # (rfm_lsqr_multi with its warm starts), errors at checkpoints against a
    # 10,000-iteration mixed-path solve of the same data sets
    many = {}
    nh = args.learned_heldout_many
    if nh > 0:
        held2 = fam(range(20000, 20000 + nh))
        d1 = params(held2[:1])
        Sm = R.System([held2[0]], asm="fp32", op="q32", tol=TOL, device=str(dev))
        Sm.assemble(d1)
        Sm.filter()
        Hm = Sm.rhs_many(held2)
        ev0.record()
        Aref, _ = Sm.solve_multi(Hm, atol=0, btol=0, max_iter=10000)
        ev1.record()
        torch.cuda.synchronize()
        t_ref = ev0.elapsed_time(ev1)
        uref = [Sm.evaluate(d1, Aref[j].contiguous(), [grid], with_error=False)[0][0] for j in range(nh)]
        del Aref
        ncols = Sm.sizes["n_cols"]
        Y0 = torch.zeros((nh, ncols), dtype=torch.float64, device=dev)
        ev0.record()
        for c0 in range(0, nh, 32):
            ps = held2[c0:c0 + 32]
            dc = params(ps)
            Sc = R.System(ps, asm="fp32", op="q32", tol=TOL, device=str(dev))
            Sc.assemble(dc)
            Sc.filter()
            Sc.fit_prepare(dc, tol_fit=1e-8)
            invc = torch.tensor([1.0 / v for v in scl(ps)], dtype=torch.float32, device=dev)
            Y0[c0:c0 + len(ps)] = W.warm_start(Sc, ctx(ps), fit_iters=300, inst_scale=invc).view(len(ps), ncols)
            del Sc
        ev1.record()
        torch.cuda.synchronize()
        t_fit = ev0.elapsed_time(ev1)
        cps = (100, 300, 1000, 3000)
        res, kept, ms_multi, resid = {}, 0, {}, {}
        for name, yy in (("zero_start", None), ("learned_start", Y0)):
            res[name], resid[name] = {}, {}
            for it in cps:
                ev0.record()
                A, rep = Sm.solve_multi(Hm, atol=0, btol=0, max_iter=it, Y0=yy)
                ev1.record()
                torch.cuda.synchronize()
                ms_multi[f"{name}_{it}"] = ev0.elapsed_time(ev1)
                if yy is not None and it == cps[0]:
                    kept = sum(int(R.report_dict(rep, j)["start"]) for j in range(nh))
                e = np.array([float(torch.linalg.norm(Sm.evaluate(d1, A[j].contiguous(), [grid],
                                                                  with_error=False)[0][0] - uref[j]) /
                                    torch.linalg.norm(uref[j])) for j in range(nh)])
                res[name][str(it)] = {"median": float(np.median(e)), "max": float(e.max()),
                                      "p90": float(np.percentile(e, 90))}
                rr = np.array([R.report_dict(rep, j)["rnorm"] / R.report_dict(rep, j)["bnorm"] for j in range(nh)])
                resid[name][str(it)] = {"median": float(np.median(rr)), "max": float(rr.max())}
            if yy is not None:
                e0m = np.array([float(torch.linalg.norm(Sm.evaluate(d1, Sm.coefficients(Y0[j].contiguous()), [grid],
                                                                    with_error=False)[0][0] - uref[j]) /
                                      torch.linalg.norm(uref[j])) for j in range(nh)])
        # LSQR's own stopping rule (atol = btol = tau, ||b|| = ||h|| for both
        # starts): iterations each data set takes to stop, at most 3000
        stop = {}
        for tau in (1e-2, 1e-3):
            stop[f"{tau:g}"] = {}
            for name, yy in (("zero_start", None), ("learned_start", Y0)):
                _, rep = Sm.solve_multi(Hm, atol=tau, btol=tau, max_iter=3000, Y0=yy)
                torch.cuda.synchronize()
                itn = np.array([R.report_dict(rep, j)["itn"] for j in range(nh)])
                ist = np.array([R.report_dict(rep, j)["istop"] for j in range(nh)])
                stop[f"{tau:g}"][name] = {"median": float(np.median(itn)), "p90": float(np.percentile(itn, 90)),
                                          "max": float(itn.max()), "stopped": int(np.sum((ist == 1) | (ist == 2)))}
        many = {"instances": nh, "seeds": f"20000-{20000 + nh - 1}",
                "solver": "rfm_lsqr_multi, all instances in one call per checkpoint (Y0 = the fitted starts)",
                "reference": "mixed path, 10000 iterations, the same many-data-set solver",
                "reference_ms": t_ref, "fit_ms": t_fit, "fit_systems": "32 instances per fitting system",
                "start_error": {"median": float(np.median(e0m)), "max": float(e0m.max())},
                "learned_starts_kept": kept, "rel_l2_after_iterations": res,
                "relative_residual_after_iterations": resid,
                "iterations_to_stopping_tolerance": stop, "solve_ms": ms_multi}

    return {
        "workload": f"2D Poisson, f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y), {S_}x{S_} subdomains, "
                    f"overlap ratio {D_}, K={K_}, {n}^2 interior + boundary rows, filter tol {TOL:g}, "
                    f"mixed path; {len(held)} held-out instances (seeds 10000-{10000 + len(held) - 1})",
        "network": "9 -> 128 x4 (tanh) -> 1 on the tensor cores (BF16 operands, FP32 accumulation and master "
                   "weights), Adam lr 2e-3 -> 1e-4, batch 4096, targets x pi^2 (a^2+b^2)",
        "forward": fwd,
        "training_solves": ntr, "training_lsqr_iterations": train_iters, "training_samples": n_samples,
        "training_solves_s": t_solve,
        "training_solver": "rfm_lsqr_multi, 256 data sets per call on one operator",
        "epochs": epochs, "data_s": t_data, "train_s": t_train, "train_samples_per_s": n_samples * epochs / t_train,
        "loss_first_last": [hist[0], hist[-1]],
        "heldout_prediction_rel_l2_at_block_rows": pred_err,
        "warm_start_ms": t_ws, "fit_lsqr_iterations": 300,
        "start_error": {"zero_start": 1.0, "learned_start_max": max(e0), "learned_start_median": float(np.median(e0))},
        "learned_starts_kept": int(used),
        "learned_starts_kept_note": "instances whose fitted start had a residual below ||h|| (the others fall back "
                                    "to the zero start inside the solver)",
        "error_after_iterations_max": {name: {str(it): float(c[it // every - 1]) for it in (100, 500, 1000, 2000,
                                                                                                3000)}
                                       for name, c in curves.items()},
        "error_after_iterations_median": {name: {str(it): float(c[it // every - 1]) for it in (100, 500, 1000, 2000,
                                                                                                  3000)}
                                          for name, c in med.items()},
        "iterations_to_0.1_max": {name: first(c, 0.1) for name, c in curves.items()},
        "iterations_to_0.1_median": {name: first(c, 0.1) for name, c in med.items()},
        "ms_per_lsqr_iteration": ms_it,
        "reference": "FP64 explicit-Q LSQR, 10000 iterations, same discretisation",
        "many_heldout": many,
    }


def oracle_free_test_grid(p):
    """400 x 400 cell-centred test grid (dimension 0 fastest)."""
    nt = list(p.n_test)
    axes = [p.lo[i] + (np.arange(nt[i]) + 0.5) * (p.hi[i] - p.lo[i]) / nt[i] for i in range(p.dim)]
    g = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([a.transpose(list(range(p.dim))[::-1]).ravel() for a in g], axis=1))


# ---------------------------------------------------------------------------
# CPU oracle leg (bounded sample)
# ---------------------------------------------------------------------------

def _oracle_block(args):
    """One block through the oracle (assembly and QR with column pivoting);
    returns its wall times.  Top-level so that a spawned worker can run it."""
    p, prm, j = args
    import oracle
    t0 = time.perf_counter()
    Bk = oracle.assemble(p, prm, blocks=[j])
    t1 = time.perf_counter()
    oracle.filter_blocks(Bk, TOL)
    return t1 - t0, time.perf_counter() - t1


def _oracle_sample(p, prm, blocks, iters, pt_stride):
    """The oracle on the sampled blocks: assembly and QR timed per block, 10
    LSQR iterations of the sampled-block subsystem, evaluation at every
    pt_stride-th test point; each part scaled to the whole workload."""
    import oracle
    J = p.J
    t0 = time.perf_counter()
    Bk = oracle.assemble(p, prm, blocks=blocks)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    F = oracle.filter_blocks(Bk, TOL)
    t_qr = time.perf_counter() - t0
    Ssub = oracle.build_system(Bk, F, mode=0)
    t0 = time.perf_counter()
    Ssub.lsqr(Bk.h, atol=0, btol=0, max_iter=10)
    t_it = (time.perf_counter() - t0) / 10
    X = oracle_free_test_grid(p)[::pt_stride]
    t0 = time.perf_counter()
    oracle.evaluate(p, prm, np.zeros(J * p.K), X)
    t_ev = (time.perf_counter() - t0) * pt_stride
    scale = J / len(blocks)
    parts = {"assembly": t_asm * scale, "qrcp": t_qr * scale, "lsqr": t_it * scale * iters, "eval": t_ev}
    return parts, sum(parts.values())


def sample_blocks(p, stride: int, offset: int = 0):
    return list(range(offset % stride, p.J, stride))


def cpu_baseline(p, prm, iters, stride=100):
    """The oracle (single-threaded FP64 C, as it stands) on every stride-th
    block of the workload: assembly, QRCP and 10 LSQR iterations of the
    sampled-block subsystem, evaluation at every 10th test point; each part
    scaled to the full workload (blocks x J / sample, iterations x the FP64
    path's iteration count, points x 10).  Extrapolated, not a full run."""
    blocks = sample_blocks(p, stride)
    parts, total_s = _oracle_sample(p, prm, blocks, iters, 10)
    return {"value": total_s * 1e3, "unit": "ms", "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": f"{len(blocks)} of {p.J} blocks (one in {stride}): assembly + QRCP + 10 LSQR iterations on "
                      f"the sampled subsystem scaled x{p.J / len(blocks):g} and to {iters} iterations; evaluation at "
                      f"every 10th test point scaled x10",
            "parts_s": parts}


def cpu_baseline_pool(p, prm, iters, stride=25, single=None):
    """The oracle's assembly and QR of every stride-th block on all of this
    host's cores (a process pool over blocks, started with spawn; core count
    from sched_getaffinity), scaled to the workload; the LSQR and evaluation
    parts are those of the single-threaded oracle (its LSQR products and
    evaluation are sequential code), taken from the single-core leg."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    blocks = sample_blocks(p, stride)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_block, [(p, prm, blocks[0])] * min(cores, len(blocks)))   # warm: workers load the oracle
        t0 = time.perf_counter()
        pool.map(_oracle_block, [(p, prm, j) for j in blocks], chunksize=1)
        t_blocks = time.perf_counter() - t0
    parts = single["parts_s"] if single else _oracle_sample(p, prm, blocks[:: max(1, len(blocks) // 4)], iters, 10)[0]
    scale = p.J / len(blocks)
    total = t_blocks * scale + parts["lsqr"] + parts["eval"]
    return {"value": total * 1e3, "unit": "ms", "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": f"assembly + QRCP of {len(blocks)} of {p.J} blocks (one in {stride}) over {cores} processes, "
                      f"scaled x{scale:g}; LSQR and evaluation single-threaded as in cpu_baseline",
            "parts_s": {"assembly_qrcp": t_blocks * scale, "lsqr": parts["lsqr"], "eval": parts["eval"]}}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands on the headline workload,
    one bounded sample per step: step i runs block sample[i mod len] of the
    same one-in-stride sample as cpu_baseline (assembly, QRCP, 10 LSQR
    iterations of that block's subsystem) and evaluation at every 100th test
    point, scaled to the workload; the mean over the steps estimates the
    same extrapolated time as cpu_baseline."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = workload(args.case)
    prm = synth.feature_params(p)
    iters = args.ref_iters
    blocks = sample_blocks(p, args.cpu_stride)
    vals = []
    t_start = time.perf_counter()
    for s in range(args.warmup + args.steps):
        j = blocks[s % len(blocks)]
        parts, total = _oracle_sample(p, prm, [j], iters, 100)
        if s >= args.warmup:
            vals.append(total * 1e3)
    wall = time.perf_counter() - t_start
    v = float(np.mean(vals))
    smp = (f"per step one of the {len(blocks)} blocks of the one-in-{args.cpu_stride} sample (cycled): assembly + "
           f"QRCP + 10 LSQR iterations of its subsystem scaled x{p.J} and to {iters} iterations; evaluation at every "
           f"100th test point scaled x100")
    out = {"impl": "reference", "metric": "solve time to fixed error (mixed FP32/FP64, zero start)",
           "value": v, "unit": "ms", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "extrapolated": True,
           "config": {"workload": workload_name(p), "lsqr_iterations": iters,
                      "wall_s_of_this_run": wall},
           "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": smp,
                            "extrapolated": True},
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-stride", type=int, default=100,
                    help="the CPU baseline runs the oracle on every n-th block (one core); the reference arm "
                         "cycles through the same sample, one block per step")
    ap.add_argument("--cpu-stride-pool", type=int, default=25,
                    help="block sample of the all-cores oracle leg")
    ap.add_argument("--ref-iters", type=int, default=8300,
                    help="LSQR iteration count the reference arm extrapolates to (the FP64 path's calibrated count "
                         "on the headline workload)")
    ap.add_argument("--cal-iters", type=int, default=CAL_ITERS, help="calibration budget (LSQR iterations)")
    ap.add_argument("--snap-every", type=int, default=100, help="calibration: iterate recorded every n iterations")
    ap.add_argument("--iters-mixed", type=int, default=None, help="skip calibration: LSQR iterations (mixed)")
    ap.add_argument("--iters-fp64", type=int, default=None, help="skip calibration: LSQR iterations (FP64)")
    ap.add_argument("--target", type=float, default=None, help="target recorded when calibration is skipped")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default QR cluster size")
    ap.add_argument("--learned-train", type=int, default=2000,
                    help="training solves of the learned warm start section (0 skips it)")
    ap.add_argument("--learned-epochs", type=int, default=2)
    ap.add_argument("--learned-heldout", type=int, default=32, help="held-out instances of the learned section")
    ap.add_argument("--learned-heldout-many", type=int, default=256,
                    help="held-out instances solved together in the learned section (0 skips)")
    ap.add_argument("--clocks-log", default=os.path.join(tempfile.gettempdir(), "bench_clocks.csv"),
                    help="CSV of the nvidia-smi clock samples taken during the timed region")
    ap.add_argument("--batched", type=int, default=64, help="instances of the batched section (0 skips it)")
    ap.add_argument("--no-poisson1d", action="store_true", help="skip the 1D time-to-1e-6 section")
    ap.add_argument("--batched-iters", type=int, default=500)
    ap.add_argument("--multi-rhs", type=int, default=64, help="data sets of the multi-right-hand-side section (0 skips)")
    ap.add_argument("--multi-iters", type=int, default=200)
    ap.add_argument("--batched-points", default="40,60", help="points per subdomain edge of the batched family")
    ap.add_argument("--batched-budget", type=float, default=0.6,
                    help="device memory budget of one wave of the batched section (fraction of 288 GB)")
    ap.add_argument("--no-p2d", action="store_true", help="skip the 2D Poisson section")
    ap.add_argument("--case", default="heat", choices=["heat", "p2d", "small"],
                    help="heat: the (2+1)D heat workload (default); p2d: the 2D Poisson workload; small: heat "
                         "blocks on 4x4x4 subdomains (profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
