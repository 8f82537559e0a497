"""Shared helpers of the GPU tests (no test logic)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lib():
    import __graft_entry__ as g
    g.build()
    import paper_0704_2341_gb300 as gs
    return gs


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxrel(a, b):
    """Element-wise error: max_i |a_i - b_i| / max_i |b_i| (a component that
    is wrong by more than the tolerance fails it, however small the others)."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    mb = np.abs(b).max() if b.size else 0.0
    return np.abs(a - b).max() / (mb if mb > 0 else 1.0) if a.size else 0.0


def close(a, b, tol):
    """Both the norm-wise and the element-wise relative error within tol."""
    return rel(a, b) <= tol and maxrel(a, b) <= tol
