"""Benchmark: solve time to a fixed error for the RRQR-filtered, preconditioned
ELM-FBPINN solver on one GB300 (and N independent instances on N GPUs).

Workload (N = 1): 2D Poisson on [0,1]^2, u = sin2pix sin2piy + 0.05
sin30pix sin30piy, 20 x 20 subdomains (overlap ratio 1.25), 300 tanh features
each, 360 x 360 cell-centred interior grid (the paper's S*ceil(K^(1/d)) rule)
plus 1440 boundary points, filter threshold 1e-6 on both paths (a threshold
below the FP32 rounding level of the assembled matrix would keep rounding-noise
columns on the mixed path).

A step is one pass of the whole path over one instance:
  assemble (FP32) -> RRQR filter (FP64 QRCP, Q_hat rounded to FP32) ->
  LSQR on Q_hat (FP32 products, FP64 vectors and scalars) for the iteration
  count that reaches the target error -> a = S^-1 y -> u_hat and its error on
  the 400 x 400 test grid.
The target error and the iteration counts come from an untimed calibration
that records LSQR iterates every 100 iterations up to the paper's budget of
10,000 iterations and evaluates each one; the target is the tightest value of
a fixed ladder that both the mixed path and the plain FP64 path (FP64
assembly, FP64 QRCP, explicit FP64 Q_hat of Proposition 3.1, zero start)
reach.  Both paths are timed; "value" is the mixed path.

At N = 1 the line also carries, each measured in the same run: the oracle
timed on a sample of the workload ("cpu_baseline"), 64 uneven instances in one
launch per call ("batched"), the learned warm start ("learned"), and the time
to 1e-6 relative L2 error on the 1D Poisson workload against plain LSQR
("poisson1d").  --impl reference times the oracle alone.
"""
from __future__ import annotations

import argparse
import json
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
                 0.1, 0.2, 0.3, 0.5, 0.7, 0.8, 0.9, 0.95, 0.99]
TOL = 1e-6
SNAP_EVERY = 100
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
# DRAM traffic from ncu captures of the current kernels (profiles/): per LSQR
# iteration for k_lsqr ((10.690 + 0.283) GB over a 50-iteration capture, scaled
# by the launch's iteration count), per launch otherwise; a kernel without an
# entry reports None.
NCU_TRAFFIC_PER_ITER = {"k_lsqr": (7.072e9 + 0.222e9) / 50}
NCU_TRAFFIC = {"k_qrcp_cluster": 0.264e9 + 0.868e9}


def workload(case: str = "full"):
    """The 20x20x300 workload; "small" keeps its block shapes (same spacing,
    same points per block) on 10 x 10 subdomains of the box [0, 9/19]^2, for
    profiler captures."""
    if case == "small":
        p = synth.poisson2d(S=10, n=180)
        p.hi = (9.0 / 19.0, 9.0 / 19.0, 1.0)
        p.n_test = [180, 180]
        return p
    return synth.poisson2d()


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

def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2506_17626_gb300 import build as B
    B.build()
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)

    p = workload(args.case)
    if world > 1:           # independent instances, one per rank (weak scaling)
        p.seed = instance_seed(p.seed, rank)
    prm = synth.feature_params(p)
    h_prm = torch.from_numpy(prm.ravel()).pin_memory()
    d_prm = h_prm.to(dev)
    Xt = torch.from_numpy(oracle_free_test_grid(p)).to(dev)

    def make(asm, op):
        S = R.System([p], asm=asm, op=op, tol=TOL, device=str(dev))
        return S

    paths = {"mixed": make("fp32", "q32"), "fp64": make("fp64", "q64")}
    # the QR cluster size is autotuned on the first filter call of each path
    # (untimed: calibration or warm-up) unless --no-autotune
    N.set_autotune(not args.no_autotune)

    # ---- calibration (untimed): error after every SNAP_EVERY iterations
    curves, conv = {}, {}
    for name, S in (paths.items() if args.iters_mixed is None else []):
        S.assemble(d_prm)
        S.filter()
        cap = CAL_ITERS // SNAP_EVERY
        snap = torch.zeros((cap, S.sizes["n_cols"]), dtype=torch.float64, device=dev)
        a, rep = S.solve(atol=0, btol=0, max_iter=CAL_ITERS, snap=snap, snap_every=SNAP_EVERY)
        errs = []
        for s in range(cap):
            a_s = S.coefficients(snap[s])
            _, err = S.evaluate(d_prm, a_s, [Xt])
            e = err.cpu().numpy()
            errs.append(float(np.sqrt(e[0] / e[1])))
        curves[name] = np.array(errs)
        conv[name] = {"min_rel_l2": float(curves[name].min()),
                      "at_iteration": SNAP_EVERY * (1 + int(curves[name].argmin())),
                      "rel_l2_at_10000": float(curves[name][-1]), "kept_columns": int(S.filter().sum().item())}
        log(f"[cal] {name}: min rel L2 {curves[name].min():.3e} at it {SNAP_EVERY * (1 + int(curves[name].argmin()))}")
    target = None
    if args.iters_mixed is not None:
        kstar = {"mixed": args.iters_mixed, "fp64": args.iters_fp64 or args.iters_mixed}
        target = args.target
    else:
        for t in TARGET_LADDER:
            if all((c <= t).any() for c in curves.values()):
                target = t
                break
        if target is None:
            target = float(max(c.min() for c in curves.values())) * 1.01
        kstar = {n: SNAP_EVERY * (1 + int(np.argmax(c <= target))) for n, c in curves.items()}
    log(f"[cal] target {target}, iterations {kstar}")

    # ---- timed steps
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

    with Clocks(args.clocks_log) as clk:
        per_mixed, outs, prof = timed(paths["mixed"], kstar["mixed"], args.steps, args.warmup, prof=True)
    per_fp64, outs64, prof64 = timed(paths["fp64"], kstar["fp64"], args.steps, args.warmup, prof=True)
    per_e2e, outs_e2e, _ = timed(paths["mixed"], kstar["mixed"], args.steps, max(1, args.warmup // 2), e2e=True)

    def mx(v):
        return max_over_ranks(v, world, dev)

    ms_mixed = mx(float(np.mean(per_mixed)))
    ms_fp64 = mx(float(np.mean(per_fp64)))
    ms_e2e = mx(float(np.mean(per_e2e)))
    err_m = outs[1].cpu().numpy()
    err_f = outs64[1].cpu().numpy()
    rel_m = float(np.sqrt(err_m[0] / err_m[1]))
    rel_f = float(np.sqrt(err_f[0] / err_f[1]))

    # ---- roofline of the dominant kernel (mixed path)
    S = paths["mixed"]
    ranks = S.filter().cpu().numpy()
    m = np.array([S.block_info(j)[0] for j in range(S.sizes["n_blocks"])])
    K = p.K
    steps = args.steps
    tot = {k: v for k, v in prof.items()}
    dom = max(tot, key=lambda k: tot[k][1])
    launches = sum(v[0] for v in tot.values())
    per_launch_ms = {k: v[1] / v[0] for k, v in tot.items()}
    roof = None
    qr_name = "k_qrcp_cluster" if "k_qrcp_cluster" in per_launch_ms else "k_qrcp"
    fused_q = qr_name == "k_qrcp_cluster"     # Q_hat accumulated in the same kernel
    qr_alg = qrcp_flops(m, K, ranks) + (formq_flops(m, ranks) if fused_q else 0.0)
    if dom == qr_name:
        # the mixed path's blocks are FP32-assembled: the cluster kernel factors
        # them in double-float, the global-memory fallback in FP64
        fl = qr_alg
        ach = fl / (per_launch_ms[dom] * 1e-3) / 1e12
        if fused_q:
            pk, src = DF_PEAK_GFLOPS / 1e3, ("derived double-float: FP32 issue 152 SMs x 4 x 32 lanes x 2.07 GHz / "
                                             "27 instructions per 4-flop update element")
        else:
            pk, src = FP64_PEAK_GFLOPS / 1e3, "derived FP64: 152 SMs x 4 flop/clk x 2.07 GHz"
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "peak_source": src, "algorithmic_per_launch": fl}
    elif dom == "k_form_q":
        fl = formq_flops(m, ranks)
        ach = fl / (per_launch_ms[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": ach / (FP64_PEAK_GFLOPS / 1e3), "peak_source": "derived FP64: 152 SMs x 4 flop/clk x 2.07 GHz",
                "algorithmic_per_launch": fl}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        by = lsqr_bytes_per_iter(m, ranks, S.sizes["n_rows"], 4) * kstar["mixed"]
        ach = by / (per_launch_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                "algorithmic_per_launch": by}
    roof["traffic"] = (NCU_TRAFFIC_PER_ITER[dom] * kstar["mixed"] if dom in NCU_TRAFFIC_PER_ITER
                       else NCU_TRAFFIC.get(dom))
    qr_gflops = qr_alg / (per_launch_ms[qr_name] * 1e-3) / 1e9
    lsqr_ms = per_launch_ms["k_lsqr"]
    spmv_gbs = lsqr_bytes_per_iter(m, ranks, S.sizes["n_rows"], 4) * kstar["mixed"] / (lsqr_ms * 1e-3) / 1e9

    clocks = clk.summary()
    out = {
        "metric": "solve time to fixed error (mixed FP32/FP64, zero start)",
        "value": ms_mixed, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_mixed, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "2D Poisson 20x20 subdomains, delta 1.25, K=300, 360^2 interior + 1440 boundary "
                               "rows, filter tol 1e-6, error on 400^2 test grid",
                   "target_rel_l2": target, "iterations": kstar, "rel_l2_reached": {"mixed": rel_m, "fp64": rel_f},
                   "convergence_10000_iterations": conv,
                   "l2_flush": "none: working set (M, QR work, Q_hat > 1.5 GB) exceeds L2 every step",
                   "parallelism": f"independent instances x{world}" if world > 1 else "1 instance",
                   "qr_cluster_autotune": not args.no_autotune},
        "fp64_zero_start_ms": ms_fp64,
        "qr_gflops": qr_gflops, "spmv_gbs": spmv_gbs,
        "kernels_ms_per_step": {k: v[1] / steps for k, v in tot.items()},
        "roofline": roof,
        "e2e": {"value": ms_e2e, "unit": "ms", "h2d_bytes_per_step": int(h_prm.numel() * 8),
                "d2h_bytes_per_step": int(S.sizes["n_cols"] * 8 + 4 * 8)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, prm, kstar["fp64"], stride=args.cpu_stride)
    if rank == 0 and world == 1 and args.batched > 0:
        out["batched"] = guarded(run_batched, args, dev)
    if rank == 0 and world == 1 and args.learned_train > 0:
        out["learned"] = guarded(run_learned, args, dev)
    if rank == 0 and world == 1 and not args.no_poisson1d:
        out["poisson1d"] = guarded(run_poisson1d, args, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, dev):
    """The batched family in one launch per call: 64 instances of uneven size
    (per instance seeded S in [8, 24]^2 subdomains, K in [100, 400] features,
    four separable sine modes), p_lo..p_hi points per subdomain edge (the
    family's 40..200 would need about 450 GB for the FP32 blocks alone), mixed
    path, a fixed number of LSQR iterations.  Phase times by CUDA events after
    one untimed pass; the filter also in block order (RFM_OPT_QR_ORDER = 0)."""
    import copy
    import torch
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import _native as N
    n_inst, (p_lo, p_hi), iters = args.batched, (8, 16), args.batched_iters
    probs = [synth.batched_instance(i, p_range=(p_lo, p_hi)) for i in range(n_inst)]
    d = torch.from_numpy(np.concatenate([synth.feature_params(p).ravel() for p in probs])).to(dev)
    grids = []
    for p in probs:
        q = copy.copy(p)
        q.n_test = [100, 100]
        grids.append(torch.from_numpy(oracle_free_test_grid(q)).to(dev))
    S = R.System(probs, asm="fp32", op="q32", tol=TOL, device=str(dev))
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

    step(False)
    rank, err = step(True)
    N.set_qr_order(False)
    try:
        ev[5].record()
        S.filter()
        ev[6].record()
    finally:
        N.set_qr_order(True)
    torch.cuda.synchronize()
    e = err.cpu().numpy().reshape(n_inst, 4)
    rel = np.sqrt(e[:, 0] / e[:, 1])
    nblk = [p.J for p in probs]
    m_blk = S.block_table()[0]
    r_blk = rank.cpu().numpy().astype(np.int64)
    K_blk = np.repeat([p.K for p in probs], nblk)
    nnz = int((m_blk * r_blk).sum())
    ms_it = ev[2].elapsed_time(ev[3]) / iters
    lsqr_gbs = lsqr_bytes_per_iter(m_blk, r_blk, S.sizes["n_rows"], 4) / (ms_it * 1e-3) / 1e9
    qr_fl = 0.0
    for mj, Kj, rj in zip(m_blk, K_blk, r_blk):
        i = np.arange(int(rj), dtype=np.float64)
        qr_fl += float(np.sum(4.0 * (mj - i) * (Kj - i) + 4.0 * (mj - i) * (rj - i)))
    return {
        "workload": f"batched 2D Poisson: {n_inst} instances, S in [8, 24]^2, K in [100, 400], "
                    f"{p_lo}-{p_hi} points per subdomain edge, 4 separable sine modes; mixed path, filter tol {TOL:g}, "
                    f"{iters} LSQR iterations, error on a 100^2 grid per instance",
        "blocks": int(sum(nblk)), "blocks_per_instance": [int(min(nblk)), int(max(nblk))],
        "rows": int(S.sizes["n_rows"]), "columns": int(S.sizes["n_cols"]), "kept_columns": int(rank.sum().item()),
        "ms": {"assemble": ev[0].elapsed_time(ev[1]), "filter": ev[1].elapsed_time(ev[2]),
               "lsqr": ev[2].elapsed_time(ev[3]), "eval": ev[3].elapsed_time(ev[4]),
               "step": ev[0].elapsed_time(ev[4]), "filter_block_order": ev[5].elapsed_time(ev[6])},
        "ms_per_lsqr_iteration": ms_it, "nnz_q_hat": nnz,
        "lsqr_gbs_algorithmic": lsqr_gbs,
        "qr_gflops_algorithmic": qr_fl / (ev[1].elapsed_time(ev[2]) * 1e-3) / 1e9,
        "rel_l2": {"median": float(np.median(rel)), "max": float(rel.max())},
    }


def run_poisson1d(args, dev):
    """Time to 1e-6 relative L2 error on the 1D Poisson workload (-u'' = f on
    [0,1], u = sin 2 pi x + 0.1 sin 50 pi x, 20 subdomains, overlap ratio
    1.3, K = 100, 1600 interior points, FP64), which, unlike the 2D workload,
    reaches it.  Calibration (untimed): zero-start LSQR for 10,000 iterations
    with the iterate evaluated every 100, plain LSQR on the unfiltered M and
    the filtered, preconditioned solver (R_hat^-1 operator) at thresholds 1e-6
    and 1e-8.  Timed (CUDA events, after warm-up): assemble -> filter -> LSQR
    for the first recorded iteration count at 1e-6 -> a = S^-1 y -> u_hat and
    its error, for each threshold that reaches 1e-6; plain LSQR does not reach
    it, and its best error and the time of its 10,000 iterations are
    reported."""
    import torch
    import paper_2506_17626_gb300 as R
    from paper_2506_17626_gb300 import sweep as SW
    p = synth.poisson1d()
    prm = torch.from_numpy(synth.feature_params(p).ravel()).to(dev)
    X = torch.from_numpy(SW.grid_points(p)).to(dev)
    runs = SW.sweep(p, prm, X, asm="fp64", op="ar64", sigmas=(1e-6, 1e-8), iters=10000, every=100, device=dev)
    st = torch.cuda.current_stream()
    out = {"workload": "1D Poisson, 20 subdomains, delta 1.3, K=100, 1600 interior + 2 boundary rows, FP64, "
                       "error on 1000 test points", "target_rel_l2": 1e-6, "runs": []}
    for r in runs:
        row = {k: r[k] for k in ("op", "sigma", "dropped_pct", "min_rel_l2", "min_rel_l2_at", "min_e_l1",
                                 "iterations_to", "lsqr_ms")}
        k = r["iterations_to"]["1e-06"]
        if k is not None:
            S = R.System([p], asm="fp64", op=r["op"], tol=r["sigma"] or 0.0, device=str(dev))

            def step():
                S.assemble(prm)
                S.filter()
                a, _ = S.solve(atol=0.0, btol=0.0, max_iter=k)
                return S.evaluate(prm, a, [X])[1]

            for _ in range(max(3, args.warmup)):
                step()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(st)
            for _ in range(args.steps):
                err = step()
            ev[1].record(st)
            torch.cuda.synchronize()
            e = SW.errors_from_sums(err.cpu().numpy(), X.shape[0])
            row.update({"iterations": k, "time_to_target_ms": ev[0].elapsed_time(ev[1]) / args.steps,
                        "rel_l2_reached": e["rel_l2"]})
        out["runs"].append(row)
    return out


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
    for i in range(0, ntr, 32):
        ps = tr[i:i + 32]
        S = R.System(ps, asm="fp32", op="q32", tol=TOL, device=str(dev))
        d = params(ps)
        S.assemble(d)
        S.filter()
        a, _ = S.solve(atol=0, btol=0, max_iter=train_iters)
        X, T = LearnedWarmStart.samples(S, d, a, ctx(ps), inst_scale=scl(ps))
        Xs.append(X)
        Ts.append(T)
        del S
    X, T = torch.cat(Xs), torch.cat(Ts)
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
    del X, T, Xs, Ts
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

    held = fam(range(10000, 10008))
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
    curves, ms_it = {}, {}
    for name, yy in (("zero_start", None), ("learned_start", y0)):
        snap = torch.zeros((iters // every, S.sizes["n_cols"]), dtype=torch.float64, device=dev)
        ev0.record()
        S.solve(atol=0, btol=0, max_iter=iters, snap=snap, snap_every=every, y0=yy)
        ev1.record()
        torch.cuda.synchronize()
        ms_it[name] = ev0.elapsed_time(ev1) / iters
        curves[name] = np.array([max(rel(S.evaluate(d, S.coefficients(snap[k]), Xt, with_error=False)[0], u_ref))
                                 for k in range(snap.shape[0])])

    def first(c, th):
        k = np.nonzero(c <= th)[0]
        return int(every * (1 + k[0])) if len(k) else None

    return {
        "workload": f"2D Poisson, f = sin(a pi x) sin(b pi y) + c sin(d pi x + e pi y), {S_}x{S_} subdomains, "
                    f"overlap ratio {D_}, K={K_}, {n}^2 interior + boundary rows, filter tol {TOL:g}, "
                    f"mixed path; 8 held-out instances (seeds 10000-10007)",
        "network": "9 -> 128 x4 (tanh) -> 1 on the tensor cores (BF16 operands, FP32 accumulation and master "
                   "weights), Adam lr 2e-3 -> 1e-4, batch 4096, targets x pi^2 (a^2+b^2)",
        "forward": fwd,
        "training_solves": ntr, "training_lsqr_iterations": train_iters, "training_samples": n_samples,
        "epochs": epochs, "data_s": t_data, "train_s": t_train, "train_samples_per_s": n_samples * epochs / t_train,
        "loss_first_last": [hist[0], hist[-1]],
        "heldout_prediction_rel_l2_at_block_rows": pred_err,
        "warm_start_ms": t_ws, "fit_lsqr_iterations": 300,
        "start_error": {"zero_start": 1.0, "learned_start": max(e0)},
        "error_after_iterations": {name: {str(it): float(c[it // every - 1]) for it in (100, 500, 1000, 2000, 3000)}
                                   for name, c in curves.items()},
        "iterations_to_0.1": {name: first(c, 0.1) for name, c in curves.items()},
        "ms_per_lsqr_iteration_8_instances": ms_it,
        "reference": "FP64 explicit-Q LSQR, 10000 iterations, same discretisation",
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

def cpu_baseline(p, prm, iters, stride=2):
    """The oracle (single-threaded FP64 C, as it stands) on every stride-th
    block of the workload: assembly, QRCP and 10 LSQR iterations of the
    sampled-block subsystem, plus evaluation at every 10th test point; each
    part scaled to the full workload (blocks x J/sample, iterations x the FP64
    path's iteration count, points x 10)."""
    import oracle
    J = p.J
    blocks = list(range(0, J, stride))
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
    X = oracle_free_test_grid(p)[::10]
    a = np.zeros(J * p.K)
    t0 = time.perf_counter()
    oracle.evaluate(p, prm, a, X)
    t_ev = (time.perf_counter() - t0) * 10
    scale = J / len(blocks)
    total_s = (t_asm + t_qr) * scale + t_it * scale * iters + t_ev
    return {"value": total_s * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"{len(blocks)} of {J} blocks (one in {stride}): assembly + QRCP + 10 LSQR iterations on "
                      f"the sampled subsystem scaled x{scale:g} and to {iters} iterations; evaluation at every "
                      f"10th of the 400^2 test points scaled x10",
            "parts_s": {"assembly": t_asm * scale, "qrcp": t_qr * scale, "lsqr": t_it * scale * iters,
                        "eval": t_ev}}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, one bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = workload()
    prm = synth.feature_params(p)
    iters = args.ref_iters
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(p, prm, iters, stride=8)
        if s >= args.warmup:
            vals.append(r["value"])
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": "solve time to fixed error (mixed FP32/FP64, zero start)",
           "value": v, "unit": "ms", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "2D Poisson 20x20 subdomains, delta 1.25, K=300, 360^2 interior + 1440 boundary "
                                  "rows, filter tol 1e-6, error on 400^2 test grid", "lsqr_iterations": iters},
           "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": r["sample"]},
           "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-stride", type=int, default=2,
                    help="the CPU baseline runs the oracle on every n-th block (about 10-30 s at 2)")
    ap.add_argument("--ref-iters", type=int, default=2600,
                    help="LSQR iteration count the reference arm extrapolates to (the calibrated count of the "
                         "GPU arm on this workload)")
    ap.add_argument("--iters-mixed", type=int, default=None, help="skip calibration: LSQR iterations (mixed)")
    ap.add_argument("--iters-fp64", type=int, default=None, help="skip calibration: LSQR iterations (FP64)")
    ap.add_argument("--target", type=float, default=None, help="target recorded when calibration is skipped")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default QR cluster size")
    ap.add_argument("--learned-train", type=int, default=384,
                    help="training solves of the learned warm start section (0 skips it)")
    ap.add_argument("--learned-epochs", type=int, default=6)
    ap.add_argument("--clocks-log", default=os.path.join(tempfile.gettempdir(), "bench_clocks.csv"),
                    help="CSV of the nvidia-smi clock samples taken during the timed region")
    ap.add_argument("--batched", type=int, default=64, help="instances of the batched section (0 skips it)")
    ap.add_argument("--no-poisson1d", action="store_true", help="skip the 1D time-to-1e-6 section")
    ap.add_argument("--batched-iters", type=int, default=2000)
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: 10x10 subdomains with the same block shapes (profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
