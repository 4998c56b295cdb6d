"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import os

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


def _spread_table():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "diffusion_spread.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        s, b, sp, se = line.split()
        rows[int(s)] = (int(b), float(sp), float(se))
    return rows


SPREAD_FACTOR = 2.0


def diffusion_bar(s, which):
    """Bar for phi_1 ("phi1") or exp ("exp") of the stiff diffusion workload
    after s doublings: SPREAD_FACTOR times the largest distance measured
    between two correct double evaluations of the oracle at the same s (the
    matrix and its permuted copy, tests/golden/diffusion_spread.txt), and at
    least the 1e-12 of every double-accurate path."""
    rows = _spread_table()
    if s in rows:
        v = rows[s][1 if which == "phi1" else 2]
    else:  # outside the measured range: the nearest entry, scaled by 2^(s - s')
        near = min(rows, key=lambda k: abs(k - s))
        v = rows[near][1 if which == "phi1" else 2] * 2.0 ** (s - near)
    return max(TOL_FP64, SPREAD_FACTOR * v)
