"""Pins for the oracle's other functions from the same resolvents (no GPU):
cos/sin with the double-angle formulae of Sec. 1 (orc_trig) and r(tA) without
range reduction (orc_rfun: the log(1 - x) weights printed after Eq. Frac4bi0,
and phi_2).  Every check uses something other than the oracle itself:
exact rational Taylor sums, 50-digit scalar recurrences, the separately
pinned complex exponential, and the closed form of log(1 - x)."""
from fractions import Fraction as Fr
from math import factorial

import numpy as np
import pytest

import oracle
from oracle import coeffs as oc

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50
U = 2.0 ** -53


def r_exact(name, x):
    """r(x) of a real set in 50-digit arithmetic (Eq. rat1)."""
    cs = oc.SETS[name]
    x = mp.mpmathify(x)
    v = mp.mpf(cs.d[0].numerator) / cs.d[0].denominator if cs.d[0] else mp.mpf(0)
    for c, b in zip(cs.c, cs.b):
        v += (mp.mpf(b.numerator) / b.denominator) / (1 - (mp.mpf(c.numerator) / c.denominator) * x)
    return v


def sym(d, seed, scale):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((d, d)))
    lam = g.uniform(-1, 1, d) * scale
    return Q, lam, (Q * lam) @ Q.T


# ---------------------------------------------------------------------------
# cos and sin (orc_trig)
# ---------------------------------------------------------------------------

def test_trig_nilpotent_no_doubling():
    """s = 0 on a nilpotent B (B^9 = 0): both results are exactly the Taylor
    sums of cos and sin to order 8 (the sets' order), so every weight, node
    and the sharing of the resolvents between the two functions is pinned."""
    n = 9
    g = np.random.default_rng(11)
    Bq = [[Fr(int(g.integers(-30, 31)), 128) if j > i else Fr(0) for j in range(n)] for i in range(n)]
    B = np.array([[float(v) for v in row] for row in Bq])
    C, S, s, info = oracle.trig(B, 1.0, s=0)
    assert info == 0 and s == 0
    P = [[Fr(int(i == j)) for j in range(n)] for i in range(n)]
    cref = [[Fr(0)] * n for _ in range(n)]
    sref = [[Fr(0)] * n for _ in range(n)]
    for k in range(n):
        ac, as_ = oc.taylor_cos(k), oc.taylor_sin(k)
        for i in range(n):
            for j in range(n):
                cref[i][j] += ac * P[i][j]
                sref[i][j] += as_ * P[i][j]
        P = [[sum(P[i][l] * Bq[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
    cref = np.array([[float(v) for v in r] for r in cref])
    sref = np.array([[float(v) for v in r] for r in sref])
    # the roundoff form rounds at u sum_i |b_i c_i| ||B|| (Sec. 4.3); the cos
    # and sin weights cancel more than exp's (sum |b_i c_i| = 4052 and 2235)
    nb = np.abs(B).sum(0).max()
    for name, out, ref in (("R8_cos", C, cref), ("R8_sin", S, sref)):
        canc = sum(abs(float(b) * float(c)) for b, c in zip(oc.SETS[name].b, oc.SETS[name].c))
        assert np.abs(out - ref).max() <= 4 * U * (canc * nb + 1), name


def test_trig_symmetric_scalar_recurrence():
    """A = Q diag(lam) Q^T: the method's result is Q diag(c_s(lam)) Q^T, where
    c_0 = r_cos(lam/2^s), s_0 = r_sin(lam/2^s) and each double-angle step takes
    (c, s) -> (2c^2 - 1, 2 s c), all in 50-digit arithmetic.  Each step can
    grow rounding by 4 |c|, so the bar is 4^s times a few u."""
    Q, lam, A = sym(24, 12, 3.0)
    C, S, s, info = oracle.trig(A, 0.9)
    assert info == 0
    th = min(oc.theta(oc.SETS["R8_cos"], oc.U_FP64), oc.theta(oc.SETS["R8_sin"], oc.U_FP64))
    assert s == oracle.select_s(oracle.norm1(0.9 * A), th)
    cl, sl = [], []
    for x in lam:
        b = mp.mpf(0.9) * mp.mpf(x) / 2 ** s
        c, sn = r_exact("R8_cos", b), r_exact("R8_sin", b)
        for _ in range(s):
            c, sn = 2 * c * c - 1, 2 * sn * c
        cl.append(float(c))
        sl.append(float(sn))
    Cref = (Q * np.array(cl)) @ Q.T
    Sref = (Q * np.array(sl)) @ Q.T
    tol = 4.0 ** s * 64 * U
    assert np.abs(C - Cref).max() <= tol
    assert np.abs(S - Sref).max() <= tol
    # and against the true functions: the truncation of order 8 at theta is
    # below u, so the same bar holds
    assert np.abs(C - (Q * np.cos(0.9 * lam)) @ Q.T).max() <= tol
    assert np.abs(S - (Q * np.sin(0.9 * lam)) @ Q.T).max() <= tol


def test_trig_is_the_complex_exponential():
    """For real A, cos(tA) = Re exp(i t A) and sin(tA) = Im exp(i t A): the
    double-angle path against the separately pinned complex exponential
    (another coefficient set, another recurrence)."""
    g = np.random.default_rng(13)
    A = g.standard_normal((20, 20)) / np.sqrt(20)
    C, S, s, info = oracle.trig(A, 1.3)
    assert info == 0
    E, _, _ = oracle.zexpm(1j * A, 1.3, "R8")
    tol = 4.0 ** s * 256 * U * max(1.0, np.abs(E).max())
    assert np.abs(C - E.real).max() <= tol
    assert np.abs(S - E.imag).max() <= tol


def test_trig_pythagoras():
    """cos^2 + sin^2 = I: (2c^2 - 1)^2 + (2sc)^2 - 1 = 4c^2 (c^2 + s^2 - 1), so
    the identity survives the doublings up to the amplified rounding."""
    g = np.random.default_rng(14)
    A = g.standard_normal((16, 16)) / 4
    C, S, s, _ = oracle.trig(A, 1.0)
    I = np.eye(16)
    assert np.abs(C @ C + S @ S - I).max() <= 4.0 ** s * 256 * U
    # the even/odd symmetry: cos(-tA) = cos(tA), sin(-tA) = -sin(tA) (the +c
    # and -c terms trade places, so the sums round in another order)
    C2, S2, _, _ = oracle.trig(A, -1.0)
    assert np.abs(C2 - C).max() <= 4.0 ** s * 256 * U
    assert np.abs(S2 + S).max() <= 4.0 ** s * 256 * U


# ---------------------------------------------------------------------------
# r(tA) with no range reduction (orc_rfun)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", [oracle.ROUNDOFF, oracle.PLAIN])
def test_log1m_nilpotent(form):
    """The printed log(1 - x) weights (c_i = 1/(i+1), Sec. 2) on a nilpotent B
    with B^5 = 0: r(B) = -(B + B^2/2 + B^3/3 + B^4/4) exactly (order 4)."""
    n = 5
    g = np.random.default_rng(15)
    B = np.triu(g.integers(-20, 21, (n, n)) / 64.0, 1)
    F, info = oracle.rfun(B, 1.0, "frac4_log1m", form)
    assert info == 0
    ref = -sum(np.linalg.matrix_power(B, k) / k for k in range(1, n))
    sum_b = sum(abs(float(b)) for b in oc.SETS["frac4_log1m"].b)
    tol = 8 * U * (sum_b if form == oracle.PLAIN else 1.0)
    assert np.abs(F - ref).max() <= tol


@pytest.mark.parametrize("name,f", [
    ("frac4_log1m", lambda x: mp.log(1 - x)),
    ("frac4_exp", mp.exp),
    ("R8_phi2", lambda x: (mp.exp(x) - 1 - x) / x ** 2 if x != 0 else mp.mpf(0.5))])
def test_rfun_symmetric(name, f):
    """A = Q diag(lam) Q^T with |lam| <= theta: r(tA) = Q diag(r(t lam)) Q^T
    (50-digit r), and r is within the forward bound of Sec. 3 of the function."""
    cs = oc.SETS[name]
    th = oc.theta(cs, oc.U_FP64)
    Q, lam, A = sym(12, 16, th)
    F, info = oracle.rfun(A, 1.0, name)
    assert info == 0
    rl = [r_exact(name, x) for x in lam]
    ref = (Q * np.array([float(v) for v in rl])) @ Q.T
    assert np.abs(F - ref).max() <= 64 * U
    for x, v in zip(lam, rl):
        assert abs(float(v - f(mp.mpf(x)))) <= 2 * U  # eps(theta) = u by the choice of theta


def test_rfun_scales_t():
    """r(tA) uses B = tA (one rounding per entry): t = 2 on A equals t = 1 on 2A."""
    A = np.random.default_rng(17).standard_normal((8, 8)) * 1e-4
    F1, _ = oracle.rfun(A, 2.0, "frac4_log1m")
    F2, _ = oracle.rfun(2 * A, 1.0, "frac4_log1m")
    assert np.array_equal(F1, F2)
