"""Helpers for the GPU parity tests (inputs from the seeded generators, expected values
from the CPU oracle)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


TOL_F64 = 1e-10   # relative L2 against the fp64 oracle (float64 values)
TOL_F32 = 1e-4    # relative L2 against the fp64 oracle (float32 values, float32 accumulation)
