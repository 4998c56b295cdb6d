"""Pins for oracle/coeffs.py against values printed in the paper.

Every printed coefficient set must come out of the Vandermonde / hybrid
systems (Sec. 2, Eq. LinearEqsbi; Sec. 4.3, Eq. ParallHybrid) exactly, and
the forward-bound thetas must reproduce Tables 1 and 2 of Sec. 5.1.
"""
import os
from fractions import Fraction as Fr

import pytest

from oracle import coeffs as oc

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([p.strip() for p in line.split("|")])
    return rows


@pytest.mark.parametrize("row", _read("paper_coefficients.txt"), ids=lambda r: r[0])
def test_printed_sets_reproduced_exactly(row):
    name, cite, c, b = row[0], row[1], row[2], row[3]
    cs = oc.SETS[name]
    assert [Fr(x) for x in c.split()] == [Fr(x) for x in cs.c], cite
    assert [Fr(x) for x in b.split()] == [Fr(x) for x in cs.b], cite
    if len(row) > 4 and row[4]:
        assert [Fr(x) for x in row[4].split()] == list(cs.d), cite


@pytest.mark.parametrize("name", ["frac4_exp", "frac4_phi1", "R4", "R4_phi1", "R8", "R8_phi1",
                                  "R5", "R10", "R10star"])
def test_order_conditions(name):
    """alpha_k = a_k for k <= s (Eq. approx1) and the first neglected one differs."""
    cs = oc.SETS[name]
    a = oc.TAYLOR[cs.func]
    for k in range(cs.order + 1):
        assert cs.alpha(k) == a(k)
    assert cs.alpha(cs.order + 1) != a(cs.order + 1)


def test_roundoff_constant_is_r0():
    """Eq. ParallRoundOff uses sum_i b_i = a0 = f(0)."""
    for name in ["R4", "R4_phi1", "R8", "R8_phi1", "R5", "R10", "R10star"]:
        assert oc.SETS[name].a0() == 1


def test_log_set_targets_log():
    cs = oc.SETS["frac4_log1m"]
    assert cs.a0() == 0 and cs.alpha(1) == -1 and cs.alpha(4) == Fr(-1, 4)


@pytest.mark.parametrize("row", _read("paper_theta.txt"), ids=lambda r: r[0])
def test_theta_tables(row):
    """Tables 1 and 2 (u <= 2^-24), printed to 3 decimals."""
    name, cite, val = row[0], row[1], float(row[2])
    if name.startswith("taylor"):
        th = oc.theta_taylor(int(name[6:]), oc.U_FP32)
    else:
        th = oc.theta(oc.SETS[name], oc.U_FP32)
    assert abs(th - val) <= 0.0015, (cite, th)


def test_theta_defines_the_bound():
    """At theta the bound equals the tolerance; just above it exceeds it."""
    for name in ["R4", "R8", "R8_phi1"]:
        cs = oc.SETS[name]
        th = oc.theta(cs, oc.U_FP64)
        assert abs(oc.forward_bound(cs, th) / oc.U_FP64 - 1) < 1e-6
        assert oc.forward_bound(cs, th * 1.01) > oc.U_FP64


@pytest.mark.parametrize("row", _read("paper_bmax.txt"), ids=lambda r: r[0])
def test_max_coefficient(row):
    """max{|b_i|, |d_i|} printed after Eqs. (Frac10biNO) and (Frac10bi)."""
    cs = oc.SETS[row[0]]
    m = max(max(abs(float(x)) for x in cs.b), max(abs(float(x)) for x in cs.d))
    assert abs(m / float(row[2]) - 1) < 0.05, row[1]


def test_pade_pairs_match_their_rational_forms():
    """Eq. Pade4 / Pade4phi1: d0 + 2 Re(b/(1 - c x)) equals the printed ratio of
    quadratics (this is what fixes the residue 6 sqrt(3); 6 sqrt(6) does not)."""
    import cmath
    for name, num, den in [("pade22", (1, 0.5, 1 / 12), (1, -0.5, 1 / 12)),
                           ("pade22_phi1", (1, 0.1, 1 / 60), (1, -0.4, 1 / 20))]:
        cs = oc.SETS[name]
        c, b, d0 = complex(cs.c[0]), complex(cs.b[0]), float(cs.d[0])
        for x in (-0.7, -0.1, 0.05, 0.3, 0.9):
            r = d0 + 2 * (b / (1 - c * x)).real
            ref = (num[0] + num[1] * x + num[2] * x * x) / (den[0] + den[1] * x + den[2] * x * x)
            assert abs(r - ref) < 1e-14
    # the misprinted residue gives a different function
    z = complex(3, -3 ** 0.5)
    w = complex(6, 6 * 6 ** 0.5)
    x = 0.3
    bad = 1 + 2 * (w / (x - z)).real
    good = (1 + x / 2 + x * x / 12) / (1 - x / 2 + x * x / 12)
    assert abs(bad - good) > 1e-2


def test_forward_bounds_ordering_claims():
    """Sec. 4.1/4.2 (Fig. 0): the R4 bound lies below the r22 Pade bound, and the R8
    bound below the degree-8 Taylor bound, over the plotted range of x."""
    r4, p22, r8 = oc.SETS["R4"], oc.SETS["pade22"], oc.SETS["R8"]
    g4, gp, g8 = (oc.forward_bound_coeffs(s) for s in (r4, p22, r8))
    from math import factorial
    for x in (0.01, 0.05, 0.1, 0.2, 0.4):
        assert oc.forward_bound(r4, x, g4) < oc.forward_bound(p22, x, gp)
        t8 = sum(x ** k / factorial(k) for k in range(9, 60))
        assert oc.forward_bound(r8, x, g8) < t8


def test_fp64_thetas():
    """theta at u = 2^-53 (used for FP64 targets): monotone in the order and
    consistent with the bound."""
    th = {n: oc.theta(oc.SETS[n], oc.U_FP64) for n in ["R4", "R8", "R8_phi1", "R10"]}
    assert 0.003 < th["R4"] < 0.0032
    assert 0.097 < th["R8"] < 0.0975
    assert 0.092 < th["R8_phi1"] < 0.0935
    assert th["R4"] < th["R8"] < th["R10"]
