"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

import oracle
from oracle import coeffs as oc

TOL_FP64 = 1e-12   # relative Frobenius error, double-accurate paths


def relerr(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def oracle_set(name):
    """Coefficient dict from the oracle's exact sets (used for both sides)."""
    return oc.oracle_coeffs(name)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch
