"""Helpers shared by the GPU tests (marshalling only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_4331_gb300 import wilson_mg  # fails loudly when the library is missing
    return wilson_mg


def lattice(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
