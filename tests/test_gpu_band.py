"""Parity of the banded action path (fm_band_expmv_batched) with the FP64
oracle: pentadiagonal A_b (half bandwidth 2), every shifted matrix factored
once by banded LU without pivoting and solved in each of the N steps; the
oracle runs the same action recurrence with dense GEPP on the same matrix
(Sec. 1: a pentadiagonal system costs 15d flops; Sec. 5.1: banded actions).

Bar: as the tridiagonal path, 1e-12 relative, or, where a set's weights are
large (Sec. 4.3), N times the round-off of one step: 2 N u (sum_i |b_i c_i|
theta + 1) in the roundoff form and 2 N u sum_i |b_i| in the plain form."""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def T(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def bar(cs, form, N):
    if form == "plain":
        return max(TOL_FP64, 2 * N * U * sum(abs(b) for b in cs["b_re"]))
    s = sum(abs(b * c) for b, c in zip(cs["b_re"], cs["c_re"])) * cs["theta"] + 1
    return max(TOL_FP64, 2 * N * U * s)


@pytest.mark.parametrize("name", ["R10", "R5", "R4", "R8"])
@pytest.mark.parametrize("form", ["roundoff", "plain"])
def test_penta_ragged(fm, name, form):
    cs = oracle_set(name)
    for d in (1, 2, 3, 5, 17, 100):
        diags, v, t = wl.penta_batch(6, d, eta=4.0, seed=700 + d)
        W, info, N = fm.band_expmv_batched(T(diags), T(v), T(t), fm.Coeffs(cs), form=form)
        W, info, N = W.cpu().numpy(), info.cpu().numpy(), N.cpu().numpy()
        for b in range(6):
            A = wl.band_dense(diags, b)
            ofm = oracle.PLAIN if form == "plain" else oracle.ROUNDOFF
            ref, N_ref, inf_ref = oracle.expmv(A, v[:, b], t[b], cs, ofm)
            assert info[b] == inf_ref == 0 and N[b] == N_ref, (d, b)
            assert relerr(W[:, b], ref) <= bar(cs, form, N_ref), (d, b)


def test_tridiagonal_through_band_entry(fm):
    """p = 1 on the banded layout is the tridiagonal path: same results."""
    dl, dd, du, v, t = wl.trid_batch(64, 50, eta=6.0, seed=710)
    diags = np.stack([dl, dd, du])
    W1, i1, N1 = fm.band_expmv_batched(T(diags), T(v), T(t), "R10")
    W2, i2, N2 = fm.trid_expmv_batched(T(dl), T(dd), T(du), T(v), T(t), "R10")
    assert bool((W1 == W2).all()) and bool((N1 == N2).all()) and bool((i1 == i2).all())


def test_penta_status(fm):
    """Non-finite entries give -2 for that system only; an exactly zero pivot
    (A = 5 I with t = 1 and one step: I - c B singular for c = 1/5) gives
    i d + row; the set's conjugate pairs and p = 3 are rejected."""
    d, n = 8, 4
    diags, v, t = wl.penta_batch(n, d, seed=720)
    diags[2, 3, 1] = np.nan
    W, info, N = fm.band_expmv_batched(T(diags), T(v), T(t), "R10")
    info = info.cpu().numpy()
    assert info[1] == -2 and info[0] == 0 and info[2] == 0
    cs = {"c_re": [0.0, 0.2], "c_im": [0.0, 0.0], "b_re": [0.5, 0.5], "b_im": [0.0, 0.0],
          "a0": 1.0, "theta": 10.0}
    z = np.zeros((5, d, 1))
    z[2, :, 0] = 1.0
    W, info, N = fm.band_expmv_batched(T(z), T(np.ones((d, 1))), T(np.array([5.0])), cs,
                                       nsteps=1)
    _, _, inf_ref = oracle.expmv(5.0 * np.eye(d), np.ones(d), 1.0, cs, nsteps=1)
    assert int(info[0]) == inf_ref == 1 * d + 1
    import torch
    with pytest.raises(fm.FmError):
        fm.band_expmv_batched(T(diags), T(v), T(t), "pade22")
    with pytest.raises(ValueError):
        fm.band_expmv_batched(torch.zeros((7, d, n), dtype=torch.float64, device="cuda"), T(v), 1.0)


def test_penta_full_size_sampled(fm):
    """32768 pentadiagonal systems of order 1000 (the paper's d for its
    tridiagonal example) in one call, the launch the bench times; sampled
    systems against the oracle's dense action."""
    diags, v, t = wl.penta_batch(32768, 1000, eta=8.0, seed=730)
    W, info, N = fm.band_expmv_batched(T(diags), T(v), T(t), "R10")
    assert int((info != 0).sum()) == 0
    Wc = W[:, [0, 9999, 32767]].cpu().numpy()
    for j, b in enumerate((0, 9999, 32767)):
        ref, N_ref, _ = oracle.expmv(wl.band_dense(diags, b), v[:, b], t[b], "R10")
        assert int(N[b]) == N_ref
        assert relerr(Wc[:, j], ref) <= TOL_FP64
