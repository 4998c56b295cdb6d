"""The autotuner (fm_autotune) and the split it drives: batched matrix
functions in FM_MIXED with FM_PATH_AUTO run the orders below the measured d*
on the one-CTA kernels and the rest on the batched grid path.  Whatever d* is,
every result must match the oracle at the 1e-12 bar, and each part must leave
the other's matrices and status alone."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def check_batch(fm, dims, seed):
    import torch
    mats = [wl.dense_scaled(d, 1.0 + (i % 5), seed + i, scale_sqrt=True) for i, d in enumerate(dims)]
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F, info, s = fm.expm_batched(P, 1.0, "R8", precision="mixed")
    st = fm.last_stats()
    assert int((info != 0).sum()) == 0
    for b, M in enumerate(mats):
        ref, s_ref, _ = oracle.expm(M, 1.0, "R8")
        assert int(s[b]) == s_ref
        assert relerr(P.get(F, b).cpu().numpy(), ref) <= TOL_FP64, (b, dims[b])
    return st


def test_autotune_measures_and_splits(fm):
    fm.lib().fm_autotune_reset()
    dstar, table = fm.autotune("expm", "R8", dmax=256)
    assert len(table) == 10 and [r[0] for r in table] == [16, 32, 48, 64, 96, 128, 160, 192, 224, 256]
    assert all(r[1] > 0 and r[2] > 0 for r in table)
    assert 1 <= dstar <= 257
    # a ragged batch around the measured order
    lo = max(1, dstar - 17)
    dims = sorted({lo, max(1, dstar - 1), min(256, dstar), min(256, dstar + 23), 7, 200})
    check_batch(fm, dims, 900)
    fm.lib().fm_autotune_reset()


def test_split_from_cache_file(fm):
    """A d* read from FM_TUNE_CACHE (64 here) splits a batch: orders 16..63 on
    the one-CTA kernels, 64 and up on the grid path (whose products the call
    counts), with every result at the bar."""
    import torch
    key = torch.cuda.get_device_name().replace(" ", "_").replace("|", "_")
    with tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False) as f:
        f.write("%s|0|64\n" % key)
        path = f.name
    old = os.environ.get("FM_TUNE_CACHE")
    os.environ["FM_TUNE_CACHE"] = path
    try:
        fm.lib().fm_autotune_reset()
        st = check_batch(fm, [16, 33, 63, 64, 65, 100, 130], 950)
        assert st["products"] > 0  # the grid part ran
        st = check_batch(fm, [16, 33, 63], 960)  # all below d*: the one-CTA kernels only
        assert st["products"] == 0
    finally:
        if old is None:
            del os.environ["FM_TUNE_CACHE"]
        else:
            os.environ["FM_TUNE_CACHE"] = old
        os.unlink(path)
        fm.lib().fm_autotune_reset()
