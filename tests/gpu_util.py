"""Helpers for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(torch, a, fp64=False):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if fp64 else torch.float32, device="cuda")
