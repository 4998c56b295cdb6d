"""Parity of the tridiagonal action path (fm_trid_expmv_batched) with the
oracle's dense action on the same matrices.

Sec. 2.1 and Sec. 5: the shifted matrices of a tridiagonal B are tridiagonal,
and the library solves them by the Thomas algorithm.  The oracle solves the
same systems densely (LU with partial pivoting), with the same N and the same
rational function, so the two agree to rounding.  The bar is 1e-12 relative
error, except for sets whose weights are large (Sec. 4.3), where any two
double evaluations may differ by N times the round-off of one step:
2 N u (sum_i |b_i c_i| theta + 1) in the roundoff form and 2 N u sum_i |b_i|
in the plain form.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
FORMS = {"roundoff": oracle.ROUNDOFF, "plain": oracle.PLAIN}


def bound(cs, N, form):
    if form == "roundoff":
        s = sum(abs(b * c) for b, c in zip(cs["b_re"], cs["c_re"])) * cs["theta"] + 1
    else:
        s = sum(abs(b) for b in cs["b_re"])
    return max(TOL_FP64, 2 * N * U * s)


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def D(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def run(fm, dl, dd, du, v, t, cs, form, **kw):
    W, info, N = fm.trid_expmv_batched(D(dl), D(dd), D(du), D(v), D(t), fm.Coeffs(cs),
                                       form=form, **kw)
    return W.cpu().numpy(), info.cpu().numpy(), N.cpu().numpy()


@pytest.mark.parametrize("form", ["roundoff", "plain"])
@pytest.mark.parametrize("name", ["R10", "R10star", "R5", "R8", "R4"])
def test_trid_ragged(fm, name, form):
    """Orders 1, 2, 3, 17, 100; 37 systems (not a multiple of a warp or a
    block) with different times, so N differs between systems."""
    cs = oracle_set(name)
    for d in (1, 2, 3, 17, 100):
        dl, dd, du, v, t = wl.trid_batch(37, d, eta=2.5, seed=100 + d)
        t = t * np.random.default_rng(d).uniform(0.3, 1.0, 37)
        W, info, N = run(fm, dl, dd, du, v, t, cs, form)
        assert (info == 0).all()
        for b in range(37):
            ref, Nr, inf = oracle.expmv(wl.trid_dense(dl, dd, du, b), v[:, b], t[b], cs,
                                        FORMS[form])
            assert inf == 0 and N[b] == Nr, (d, b)
            assert relerr(W[:, b], ref) <= bound(cs, Nr, form), (d, b)


def test_trid_step_options(fm):
    """A caller bound in place of ||A||_1, a forced N, and a negative time."""
    cs = oracle_set("R10")
    dl, dd, du, v, t = wl.trid_batch(20, 40, eta=3.0, seed=7)
    t[3] = -t[3]
    for kw, okw in (({"anorm": 5.0}, {"anorm": 5.0}), ({"nsteps": 3}, {"nsteps": 3})):
        W, info, N = run(fm, dl, dd, du, v, t, cs, "roundoff", **kw)
        assert (info == 0).all()
        for b in range(20):
            ref, Nr, _ = oracle.expmv(wl.trid_dense(dl, dd, du, b), v[:, b], t[b], cs,
                                      oracle.ROUNDOFF, **okw)
            assert N[b] == Nr
            assert relerr(W[:, b], ref) <= bound(cs, Nr, "roundoff")


def test_trid_status(fm):
    """A non-finite entry flags its own system only; an exactly zero pivot
    reports (term index) d + row, as the oracle does; a zero matrix gives v."""
    cs = oracle_set("R10")
    dl, dd, du, v, t = wl.trid_batch(9, 12, eta=2.0, seed=8)
    dd[5, 2] = np.nan
    v[0, 6] = np.inf
    dl[0, :] = np.nan   # slots outside A are not read
    du[11, :] = np.nan
    W, info, N = run(fm, dl, dd, du, v, t, cs, "roundoff")
    assert info[2] == -2 and info[6] == -2
    dl[0, :] = 0.0
    du[11, :] = 0.0
    for b in (0, 1, 3, 4, 5, 7, 8):
        assert info[b] == 0
        ref, _, _ = oracle.expmv(wl.trid_dense(dl, dd, du, b), v[:, b], t[b], cs)
        assert relerr(W[:, b], ref) <= TOL_FP64
    # 1 - c h a = 0 exactly for c = 1/8 (term 1 of R10), h = 1, a = 8
    one = np.ones((1, 1))
    W, info, N = run(fm, 0 * one, 8 * one, 0 * one, one, np.ones(1), cs, "roundoff", nsteps=1)
    _, _, inf_ref = oracle.expmv(8 * one, np.ones(1), 1.0, cs, oracle.ROUNDOFF, nsteps=1)
    assert info[0] == inf_ref == 1 * 1 + 1
    z = np.zeros((30, 4))
    W, info, N = run(fm, z, z, z, np.ones((30, 4)), np.ones(4), cs, "roundoff")
    assert (info == 0).all() and (N == 1).all() and (W == 1.0).all()


def test_trid_rejects_bad_sets(fm):
    import torch
    one = torch.ones((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(fm.FmError):
        fm.trid_expmv_batched(one, one, one, one, 1.0, "pade22")   # complex nodes


def test_trid_full_size_sampled(fm):
    """The benchmark's configuration: 32768 systems of order 1000 (the
    paper's d), R10 in the roundoff form (R'_10), ||t A||_1 = 8; sampled
    systems against the oracle, every status and N checked."""
    cs = oracle_set("R10")
    batch, d = 32768, 1000
    dl, dd, du, v, t = wl.trid_batch(batch, d, eta=8.0, seed=5000)
    W, info, N = fm.trid_expmv_batched(D(dl), D(dd), D(du), D(v), D(t), fm.Coeffs(cs))
    info, N = info.cpu().numpy(), N.cpu().numpy()
    assert (info == 0).all()
    assert (N == int(np.ceil(8.0 / cs["theta"]))).all()
    for b in (0, 12345, batch - 1):
        ref, Nr, _ = oracle.expmv(wl.trid_dense(dl, dd, du, b), v[:, b], t[b], cs)
        assert N[b] == Nr
        assert relerr(W[:, b].cpu().numpy(), ref) <= TOL_FP64
