"""Shared helpers for the GPU parity tests (device buffers via torch, library via the C ABI)."""
import numpy as np
import pytest


def need_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but CUDA is not available")
    return torch


def lib():
    from paper_1001_5460_gb300 import build

    build.build()
    from paper_1001_5460_gb300 import tca

    return tca


def to_dev(a, dtype):
    torch = need_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=dtype))
    return t.cuda()


def empty_dev(shape, dtype):
    torch = need_cuda()
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    return torch.full(tuple(shape), float("nan"), dtype=tdt, device="cuda")


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Tolerances (relative L2 error against the FP64 oracle), derived in the design
# notes: FP64 path ~ 1e-15 * sqrt(terms); FP32 path: unit roundoff 6e-8 times the
# growth over a chain of <= 4 banded/dense products of <= ~100 terms each.
TOL_F64 = 1e-12
TOL_F32 = 2e-5
