"""Other functions from the same shifted solves on the GPU (Sec. 1, Sec. 2):
cos and sin with the double-angle formulae (fm_cossin), and r(tA) with no
range reduction (fm_rfun: the printed log(1 - x) weights, phi_2), against the
oracle's orc_trig and orc_rfun on the same seeded inputs.

Bars.  r(tA): 1e-12 as every double-accurate path.  cos/sin: each
double-angle step (C, S) <- (2C^2 - I, 2SC) can multiply the rounding by
about 4||C||, and the cos and sin weights cancel more than exp's (sum |b_i c_i|
= 4052 and 2235); two correct double evaluations therefore differ by about
4^s u sum|b_i c_i| theta: the bar is max(1e-12, 4^s * 64 u)."""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
PREC_PATH = [("fp64", "cta"), ("mixed", "cta"), ("fp64", "grid"), ("mixed", "grid")]


@pytest.fixture(scope="module")
def fm():
    need_gpu()
    import paper_2210_03714_gb300 as fm_
    fm_.lib()
    return fm_


def T(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def trig_bar(s):
    return max(TOL_FP64, 4.0 ** s * 64 * U)


@pytest.mark.parametrize("prec,path", PREC_PATH)
def test_cossin_single(fm, prec, path):
    A = wl.dense_scaled(72, 3.0, 61, scale_sqrt=True)
    cc, cs = oracle_set("R8_cos"), oracle_set("R8_sin")
    C_ref, S_ref, s_ref, _ = oracle.trig(A, 0.8, cc, cs)
    C, S, info, s = fm.cossin(T(A), 0.8, fm.Coeffs(cc), fm.Coeffs(cs), precision=prec, path=path)
    assert info == 0 and s == s_ref
    assert relerr(C.cpu().numpy(), C_ref) <= trig_bar(s)
    assert relerr(S.cpu().numpy(), S_ref) <= trig_bar(s)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cossin_batched_ragged(fm, prec):
    """Orders across tile edges and the one-CTA solve's column grouping; mixed
    with dmax >= 64 runs the batched grid path."""
    import torch
    dims = [1, 5, 17, 33, 64, 65, 100, 130]
    mats = [wl.dense_scaled(d, 0.5 + 0.6 * i, 70 + i, scale_sqrt=True) for i, d in enumerate(dims)]
    ts = np.linspace(0.6, 1.4, len(dims))
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    Cf, Sf, info, s = fm.cossin_batched(P, T(ts), "R8_cos", "R8_sin", precision=prec)
    assert int((info != 0).sum()) == 0
    for b, (M, t) in enumerate(zip(mats, ts)):
        C_ref, S_ref, s_ref, _ = oracle.trig(M, t, "R8_cos", "R8_sin")
        assert int(s[b]) == s_ref
        assert relerr(P.get(Cf, b).cpu().numpy(), C_ref) <= trig_bar(s_ref), b
        assert relerr(P.get(Sf, b).cpu().numpy(), S_ref) <= trig_bar(s_ref), b


@pytest.mark.parametrize("prec,path", PREC_PATH)
@pytest.mark.parametrize("name", ["frac4_log1m", "R8_phi2", "frac4_exp"])
def test_rfun_single(fm, prec, path, name):
    """r(tA) as it is, with ||tA||_1 just below the set's theta (the log(1 - x)
    set of Sec. 2 has theta 1.3e-3 for double accuracy)."""
    cs = oracle_set(name)
    A = wl.dense_scaled(80, 0.99 * cs["theta"], 62, scale_sqrt=True)
    F_ref, _ = oracle.rfun(A, 1.0, cs)
    F, info = fm.rfun(T(A), 1.0, fm.Coeffs(cs), precision=prec, path=path)
    assert info == 0
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rfun_batched_and_range_flag(fm, prec):
    """The batched form; a matrix with ||tA||_1 > theta is still evaluated and
    reported with info -5."""
    import torch
    cs = oracle_set("frac4_log1m")
    dims = [9, 64, 96]
    norms = [0.5 * cs["theta"], 0.99 * cs["theta"], 3 * cs["theta"]]
    mats = [wl.dense_scaled(d, n, 80 + i, scale_sqrt=True) for i, (d, n) in enumerate(zip(dims, norms))]
    P = fm.Packed([torch.from_numpy(m) for m in mats], device="cuda")
    F, info = fm.rfun_batched(P, 1.0, fm.Coeffs(cs), precision=prec)
    assert info.cpu().tolist() == [0, 0, -5]
    for b, M in enumerate(mats):
        ref, _ = oracle.rfun(M, 1.0, cs)
        assert relerr(P.get(F, b).cpu().numpy(), ref) <= TOL_FP64
