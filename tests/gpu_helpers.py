"""Shared helpers for the GPU parity tests (inputs rounded to float32 once, so
the oracle and the CUDA path see identical values)."""
import copy

import numpy as np
import pytest


def f32(a):
    """Round to float32 and back to float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def f32_geom(geom):
    g = copy.deepcopy(geom)
    g.wavelet = f32(g.wavelet)
    return g


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_ctx(case, device=0):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_17518_gb300 import build
    from paper_2403_17518_gb300.ops import Context

    build()
    return Context(case.nz, case.nx, case.h, case.dt, case.nb, device=device)


def to_dev(a):
    import torch

    return torch.as_tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)
