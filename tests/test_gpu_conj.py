"""Conjugate-pair coefficient sets on the GPU (Eq. Pade4, Eq. Pade4phi1).

A conjugate-pair term 2 Re(b c x / (1 - c x)) is evaluated on real matrices as
one real system I - 2 Re(c) B + |c|^2 B^2 after one product B^2 (Sec. 1: one
product, x^2, and one inverse per pair of complex-conjugate roots); the oracle
solves the complex system (I - c B) Y = c B R and takes 2 Re(b Y).  Same
rational function, different rounding: the bar is the 1e-12 of every
double-accurate path.  Complex matrices take the analytic form (two complex
systems, the set written out), compared with the oracle on the written-out set.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu

PREC_PATH = [("fp64", "cta"), ("mixed", "cta"), ("fp64", "grid"), ("mixed", "grid")]


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def T(x):
    import torch
    x = np.ascontiguousarray(x)
    dt = torch.complex128 if np.iscomplexobj(x) else torch.float64
    return torch.tensor(x, dtype=dt, device="cuda")


def written_out(cs):
    """The analytic form of a conjugate-pair set: terms (c, b) and (conj c, conj b)."""
    c = [complex(r, i) for r, i in zip(cs["c_re"], cs["c_im"])]
    b = [complex(r, i) for r, i in zip(cs["b_re"], cs["b_im"])]
    cc = [x for v in c for x in (v, v.conjugate())]
    bb = [x for v in b for x in (v, v.conjugate())]
    out = dict(cs)
    out.update(c_re=[v.real for v in cc], c_im=[v.imag for v in cc], b_re=[v.real for v in bb],
               b_im=[v.imag for v in bb], conj_pair=0)
    return out


@pytest.mark.parametrize("prec,path", PREC_PATH)
@pytest.mark.parametrize("form", ["roundoff", "plain"])
def test_pade22_expm(fm, prec, path, form):
    cs = oracle_set("pade22")
    A = wl.dense_scaled(70, 3.0, 31)
    ofm = oracle.ROUNDOFF if form == "roundoff" else oracle.PLAIN
    F_ref, s_ref, _ = oracle.expm(A, 0.8, cs, ofm)
    F, info, s = fm.expm(T(A), 0.8, fm.Coeffs(cs), precision=prec, path=path, form=form)
    assert info == 0 and s == s_ref
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_pade22_phi1_set_no_squaring(fm, prec, path):
    """The phi_1 Pade set of Eq. (Pade4phi1) as r(tA) itself (s = 0)."""
    cs = oracle_set("pade22_phi1")
    A = wl.dense_scaled(48, 0.002, 32)
    F_ref, _, _ = oracle.expm(A, 1.0, cs, s=0)
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision=prec, path=path, s_fixed=0)
    assert info == 0 and s == 0
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_pade22_two_functions(fm, prec, path):
    """Two weight vectors over the same conjugate-pair system (the phi_1 call
    with both sets on the r22 nodes), with the doubling of Sec. 1."""
    cs = oracle_set("pade22")
    A = wl.dense_scaled(40, 2.0, 33)
    Phi_ref, E_ref, s_ref, _ = oracle.phi1(A, 1.0, cs, cs)
    Phi, E, info, s = fm.phi1(T(A), 1.0, fm.Coeffs(cs), fm.Coeffs(cs), precision=prec, path=path)
    assert info == 0 and s == s_ref
    assert relerr(Phi.cpu().numpy(), Phi_ref) <= TOL_FP64
    assert relerr(E.cpu().numpy(), E_ref) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pade22_batched(fm, prec):
    """A ragged batch (orders across tile edges); mixed with dmax >= 64 runs
    the batched grid path, double the one-CTA kernels."""
    import torch
    cs = oracle_set("pade22")
    dims = [1, 7, 33, 64, 65, 130]
    mats = [wl.dense_scaled(d, 1.0 + 0.5 * i, 40 + i, scale_sqrt=True) for i, d in enumerate(dims)]
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F, info, s = fm.expm_batched(P, 1.0, fm.Coeffs(cs), precision=prec)
    assert int((info != 0).sum()) == 0
    for b, M in enumerate(mats):
        ref, s_ref, _ = oracle.expm(M, 1.0, cs)
        assert int(s[b]) == s_ref
        assert relerr(P.get(F, b).cpu().numpy(), ref) <= TOL_FP64, b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("form", ["roundoff", "plain"])
def test_pade22_action(fm, prec, form):
    """The action: one real quadratic system per pair, factored once and
    solved in every step (right-hand side g W + a B W + b B^2 W)."""
    cs = oracle_set("pade22")
    A = wl.dense_scaled(50, 0.05, 34)
    V = np.random.default_rng(35).standard_normal((50, 3))
    ofm = oracle.ROUNDOFF if form == "roundoff" else oracle.PLAIN
    W_ref, N_ref, _ = oracle.expmv(A, V, 1.0, cs, ofm)
    W, info, N = fm.expmv(T(A), T(V), 1.0, fm.Coeffs(cs), precision=prec, path="cta", form=form)
    assert info == 0 and N == N_ref
    assert relerr(W.cpu().numpy(), W_ref) <= TOL_FP64


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_pade22_complex_matrix(fm, prec, path):
    """Complex A: the analytic form, two complex systems per pair."""
    cs = oracle_set("pade22")
    g = np.random.default_rng(36)
    A = (g.standard_normal((40, 40)) + 1j * g.standard_normal((40, 40))) / 40
    F_ref, s_ref, _ = oracle.zexpm(A, 1.0, written_out(cs))
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision=prec, path=path)
    assert info == 0 and s == s_ref
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


def test_conjugate_pair_rejected_by_adjoint_and_trid(fm):
    import torch
    P = fm.Packed([T(np.eye(4))])
    v = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(fm.FmError):
        fm.expmv_adjoint_batched(P, v, v, [2], 1.0, "pade22")
    one = torch.ones((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(fm.FmError):
        fm.trid_expmv_batched(one, one, one, one, 1.0, "pade22")
