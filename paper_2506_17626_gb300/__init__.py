"""GB300-native ELM-FBPINN solver with local RRQR filtering and right
preconditioning: block assembly, batched pivoted QR with threshold dropping,
and preconditioned LSQR, as hand-written sm_103a CUDA kernels behind the C ABI
of include/rfm.h.  This package is the thin Python binding over that library.
"""
from .api import Mlp, System, report_dict  # noqa: F401
from . import _native  # noqa: F401

__all__ = ["Mlp", "System", "report_dict"]
