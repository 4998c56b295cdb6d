"""The team path: exp(tA) of one matrix of small order with every step spread
over many thread blocks of one cooperative launch (the shifted systems of
Eq. ParallRoundOff factored on separate blocks at once, Sec. 2; the solves'
right-hand-side columns, B^2 and the squarings split over the grid).  Double
arithmetic throughout, so the bar is the 1e-12 of every double-accurate path,
against the oracle, with the same s; for a set or form whose weights cancel it
is twice the measured spread of two correct double evaluations."""
import numpy as np
import pytest

import oracle
from paper_2210_03714_gb300 import workloads as wl

from _common import TOL_FP64, need_gpu, oracle_set, relerr

pytestmark = pytest.mark.gpu


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


def spread_bar(A, cs, form, F_ref):
    """max(1e-12, twice the measured spread of two correct double evaluations):
    the oracle on P A P^T mapped back against the oracle on A.  Sets whose
    weights cancel (Sec. 4.3: sum |b_i c_i| of R10* is 1.3e6) and the plain form
    of Eq. rat1 amplify rounding by that much, so two correct evaluations differ
    by about 1e-10 there; for R4, R8 and the Pade set in the roundoff form the
    spread is far below 1e-12."""
    d = A.shape[0]
    p = np.random.default_rng(5).permutation(d)
    F2, _, _ = oracle.expm(A[np.ix_(p, p)], 1.0, cs, form)
    q = np.argsort(p)
    return max(TOL_FP64, 2.0 * relerr(F2[np.ix_(q, q)], F_ref))


# orders: one element, below one 8 x 8 tile, ragged tiles, the d = 64 problem,
# several column blocks per system, the largest order of the path
@pytest.mark.parametrize("d", [1, 5, 16, 37, 64, 130, 256, 512])
@pytest.mark.parametrize("name", ["R4", "R8", "R10star", "pade22"])
def test_team_expm_vs_oracle(fm, d, name):
    cs = oracle_set(name)
    A = wl.dense_scaled(d, 3.0, 900 + d, scale_sqrt=True)
    F_ref, s_ref, _ = oracle.expm(A, 1.0, cs)
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision="fp64", path="team")
    assert info == 0 and s == s_ref
    bar = spread_bar(A, cs, oracle.ROUNDOFF, F_ref) if name == "R10star" else TOL_FP64
    assert relerr(F.cpu().numpy(), F_ref) <= bar


def test_team_single_d64_is_the_default_route(fm):
    """The d = 64 problem (R4, ||A||_1 = 2, s = 10) on the default path and
    precision lands on the team path and matches the oracle."""
    A, _ = wl.single_d64()
    cs = oracle_set("R4")
    F_ref, s_ref, _ = oracle.expm(A, 1.0, cs)
    for prec in ("fp64", "mixed"):
        F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision=prec)
        assert fm.last_stats()["launches"] == 1  # one cooperative launch
        assert info == 0 and s == s_ref == 10
        assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


@pytest.mark.parametrize("form", ["roundoff", "plain"])
def test_team_forms_against_one_cta(fm, form):
    """Both forms of Eq. ParallRoundOff / Eq. rat1 against the oracle and
    against the one-CTA kernel in double (same systems, same element-wise
    steps: only the association of the dot products differs).  The roundoff
    form at 1e-12; the plain form within twice the measured spread of two
    correct double evaluations (about 1.2e-10 here: Sec. 4.3, the rounding of
    each (I - c_i B)^-1 is multiplied by |b_i|, sum |b_i| = 5.8e3 for R8)."""
    cs = oracle_set("R8")
    A = wl.dense_scaled(96, 6.0, 77)
    ofm = oracle.ROUNDOFF if form == "roundoff" else oracle.PLAIN
    F_ref, s_ref, _ = oracle.expm(A, 1.0, cs, ofm)
    F1, i1, s1 = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision="fp64", path="team", form=form)
    F2, i2, s2 = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision="fp64", path="cta", form=form)
    assert i1 == i2 == 0 and s1 == s2 == s_ref
    bar = TOL_FP64 if form == "roundoff" else spread_bar(A, cs, ofm, F_ref)
    assert relerr(F1.cpu().numpy(), F_ref) <= bar
    assert relerr(F1.cpu().numpy(), F2.cpu().numpy()) <= bar


@pytest.mark.parametrize("d", [24, 200])
def test_team_complex_hermitian(fm, d):
    g = np.random.default_rng(61 + d)
    G = (g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))) / np.sqrt(d)
    H = (G + G.conj().T) / 2
    A = -1j * H * (6.0 / np.abs(np.linalg.eigvalsh(H)).max())
    cs = oracle_set("R8")
    F_ref, s_ref, _ = oracle.zexpm(A, 1.0, cs)
    F, info, s = fm.expm(T(A), 1.0, fm.Coeffs(cs), precision="fp64", path="team")
    assert info == 0 and s == s_ref
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64


def test_team_rfun_and_range_flag(fm):
    """r(tA) without scaling (s = 0), and info -5 when ||tA||_1 > theta."""
    cs = oracle_set("frac4_log1m")
    A = wl.dense_scaled(80, 0.99 * cs["theta"], 62, scale_sqrt=True)
    F_ref, _ = oracle.rfun(A, 1.0, cs)
    F, info = fm.rfun(T(A), 1.0, fm.Coeffs(cs), precision="fp64", path="team")
    assert info == 0
    assert relerr(F.cpu().numpy(), F_ref) <= TOL_FP64
    _, info = fm.rfun(T(A), 2.0, fm.Coeffs(cs), precision="fp64", path="team")
    assert info == -5


def test_team_status(fm):
    import torch
    A = np.eye(6)
    A[1, 4] = np.inf
    _, info, _ = fm.expm(T(A), 1.0, "R8", path="team")
    assert info == -2
    # the zero pivot of the pair c = +-2/15 (terms 3 and 4): fl(c^2) 7.5^2 = 1
    A = np.diag([7.5, 0.1, 0.2])
    _, info, _ = fm.expm(T(A), 1.0, "R8", anorm=1e-3, path="team")
    assert info == 3 * 3 + 1
    F, info, s = fm.expm(T(np.zeros((11, 11))), 1.0, "R8", path="team")
    assert info == 0 and s == 0
    assert float((F - torch.eye(11, dtype=torch.float64, device="cuda")).abs().max()) == 0


def test_team_rejects(fm):
    """FM_PATH_TEAM takes single-matrix exp in double, d <= 512."""
    A = wl.dense_scaled(32, 1.0, 3)
    for prec in ("fp32_ir", "bf16_ir"):
        with pytest.raises(fm.FmError):
            fm.expm(T(A), 1.0, "R8", precision=prec, path="team")
    with pytest.raises(fm.FmError):
        fm.phi1(T(A), 1.0, "R8", "R8_phi1", path="team")
    with pytest.raises(fm.FmError):
        fm.expm(T(wl.dense_scaled(600, 1.0, 3)), 1.0, "R8", path="team")
    P = fm.Packed([T(A), T(A)])
    with pytest.raises(fm.FmError):
        fm.expm_batched(P, 1.0, "R8", path="team")
