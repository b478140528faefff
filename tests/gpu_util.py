"""Shared helpers of the GPU tests (test infrastructure)."""
from __future__ import annotations

import numpy as np
import pytest

TOL = {1: 1e-12, 2: 1e-28, 4: 1e-58, 8: 1e-118}


def cuda_ok() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def need_gpu():
    if not cuda_ok():
        pytest.skip("no CUDA device")
    from paper_2301_12659_gb300 import build
    build.build()
    from paper_2301_12659_gb300 import mdnewton
    mdnewton.load()
    return mdnewton


def to_np(t) -> np.ndarray:
    return t.detach().cpu().numpy()


def planted(cfg, with_cst=True):
    """Planted workload with the oracle's constant term (tests only)."""
    from oracle import oracle
    from paper_2301_12659_gb300 import workloads as wl
    s, xstar, x0 = wl.planted_system(cfg)
    if with_cst:
        s.cst = oracle.planted_constant(s, xstar)
    return s, xstar, x0
