"""Multi-rank path of the benchmark on CPU (two gloo ranks, no GPU).

With N ranks the solver runs replicas: every rank solves its own independent
instance (seed base + rank) and no collective touches the data path; the only
collectives are the barriers around the timed region and one all-reduce that
takes the slowest rank's time.  These tests run that host logic as two
processes over gloo, each rank solving its instance with the CPU oracle in
place of the GPU step, and check that the ranks' instances are the
single-process ones, that they differ, and that every rank reports the
maximum time.
"""
from __future__ import annotations

import contextlib
import io
import os
import pickle
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _small_problem():
    import synth
    return synth.poisson1d(S=4, K=12, n=48, n_test=64)


def _solve(p):
    """The oracle's Algorithm 2 on one instance, and its error on the test grid."""
    import oracle
    import synth
    prm = synth.feature_params(p)
    r = oracle.solve(p, prm, tol=1e-10, atol=1e-12, btol=1e-12, max_iter=300)
    X = oracle.test_grid(p)
    err = oracle.errors(oracle.evaluate(p, prm, r["a"], X), oracle.exact(p, X))["rel_l2"]
    return r["a"], err


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _small_problem()
        p.seed = bench.instance_seed(p.seed, rank)
        a, err = _solve(p)
        dist.barrier()
        # a stand-in for the rank's measured step time: the ranks differ
        t_max = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
        got = [None] * world
        dist.all_gather_object(got, {"rank": rank, "seed": p.seed, "a": a, "err": err, "t_max": t_max})
        if rank == 0:
            with open(out_path, "wb") as f:
                pickle.dump(got, f)
    finally:
        dist.destroy_process_group()


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_solve_independent_instances(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import oracle
    oracle.build()          # once, before the ranks start (they only load it)

    out = str(tmp_path / "ranks.pkl")
    mp.spawn(_rank_main, args=(WORLD, _free_port(), out), nprocs=WORLD, join=True)
    with open(out, "rb") as f:
        got = pickle.load(f)

    assert [g["rank"] for g in got] == list(range(WORLD))
    base = _small_problem().seed
    assert [g["seed"] for g in got] == [base + r for r in range(WORLD)]
    # every rank reports the slowest rank's time
    assert all(g["t_max"] == 10.0 * WORLD for g in got)
    # each rank's result is exactly the single-process solve of its instance
    for g in got:
        p = _small_problem()
        p.seed = g["seed"]
        a, err = _solve(p)
        np.testing.assert_array_equal(g["a"], a)
        assert g["err"] == err
    # the instances are independent draws, not copies
    assert not np.array_equal(got[0]["a"], got[1]["a"])


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.instance_seed(7, 0) == 7


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    """Under torchrun only rank 0 times the oracle and prints the line; the
    other ranks return at once and print nothing."""
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        r = bench.run_reference(argparse.Namespace(steps=1, warmup=3, ref_iters=10))
    assert r is None
    assert buf.getvalue() == ""


def test_clock_sampler_watches_the_ranks_own_gpu():
    import bench
    assert bench.smi_device_id({}) == "0"
    assert bench.smi_device_id({"LOCAL_RANK": "3"}) == "3"
    assert bench.smi_device_id({"LOCAL_RANK": "1", "CUDA_VISIBLE_DEVICES": "4,5,6"}) == "5"
    assert bench.smi_device_id({"CUDA_VISIBLE_DEVICES": "GPU-abc, GPU-def", "LOCAL_RANK": "1"}) == "GPU-def"


def test_reference_arm_prints_the_contract_line(monkeypatch):
    """Rank 0 of the reference arm times the oracle on a bounded sample and
    prints one JSON line with the benchmark's keys: the metric, its unit and
    direction, an extrapolated value, a cpu_baseline of kind oracle on one
    core, and an e2e object without host-device copies."""
    import argparse
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(argparse.Namespace(case="small", steps=1, warmup=0, ref_iters=10, cpu_stride=100))
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["metric"] == "solve time to fixed error (mixed FP32/FP64, zero start)"
    assert d["value"] > 0 and d["value"] == d["ms_per_step"] == d["cpu_baseline"]["value"] == d["e2e"]["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["extrapolated"] is True and d["cpu_baseline"]["extrapolated"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["vs_baseline"] is None
