"""Memory-budgeted waves of a batch of instances.

A batch whose workspace (rfm_problem_size) exceeds the device memory it may
use runs as consecutive systems ("waves"), each one launch per call of the
path.  This module only groups the instance list: every workspace size comes
from the library's host-only rfm_problem_size.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence

from . import _native as N


def workspace_bytes(problems: Sequence, asm: str = "fp32", op: str = "q32", tol: float = 1e-6) -> int:
    """Workspace bytes of one system holding `problems` side by side."""
    arr = (N.RfmProblem * len(problems))(*[N.problem_struct(p) for p in problems])
    cfg = N.RfmConfig(N.ASM[asm], N.OPS[op], float(tol))
    sz = N.RfmSizes()
    N.check("rfm_problem_size", N.load().rfm_problem_size(arr, len(problems), C.byref(cfg), C.byref(sz)))
    return int(sz.workspace_bytes)


def plan_waves(problems: Sequence, budget_bytes: int, asm: str = "fp32", op: str = "q32", tol: float = 1e-6,
               max_per_wave: int = 64) -> List[List[int]]:
    """Consecutive groups of instance indices whose system fits the budget
    (greedy in list order, at most max_per_wave instances, the LSQR kernel's
    limit per system).  An instance that alone exceeds the budget raises
    ValueError."""
    waves: List[List[int]] = []
    cur: List[int] = []
    for i in range(len(problems)):
        trial = cur + [i]
        if len(trial) <= max_per_wave and workspace_bytes([problems[k] for k in trial], asm, op, tol) <= budget_bytes:
            cur = trial
            continue
        if not cur:
            raise ValueError(f"instance {i} alone needs more than {budget_bytes} bytes")
        waves.append(cur)
        cur = [i]
        if workspace_bytes([problems[i]], asm, op, tol) > budget_bytes:
            raise ValueError(f"instance {i} alone needs more than {budget_bytes} bytes")
    if cur:
        waves.append(cur)
    return waves
