"""Shared helpers of the GPU tests (not collected as tests)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_11558_gb300 import fvim
    import __graft_entry__

    if not __import__("os").path.exists(fvim.LIB_PATH):
        __graft_entry__.build()
    return torch


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all entries (real or complex)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(torch, arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr)).to(device="cuda", dtype=dtype)
