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


def max_rel(a, b):
    """max |a - b| / max |b| over all cells and components (the max-norm
    companion of the relative L2 error)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def assert_close(got, ref, tol, max_tol=None):
    """Parity bound: relative L2 error AND max-norm relative error
    max|got - ref| / max|ref| both below their bounds (max_tol defaults to
    tol), so a local error (one ragged tile, one fold row) cannot hide under
    the global norm."""
    e2, em = rel_l2(got, ref), max_rel(got, ref)
    mt = tol if max_tol is None else max_tol
    assert e2 < tol and em < mt, "rel L2 %.3e (bound %.1e), max|d|/max|ref| %.3e (bound %.1e)" % (e2, tol, em, mt)
    return e2, em
