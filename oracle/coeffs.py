"""Exact coefficient sets and forward-bound thresholds for the oracle.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
only tests/, the smoke check and the CPU-baseline leg of bench.py use it.

Blanes, "Parallel computation of functions of matrices and their action on
vectors" (arXiv:2210.03714):

* Sec. 2, Eq. (rat1)/(approx1)/(LinearEqsbi): r(x) = sum_i b_i / (1 - c_i x) has
  order s = P-1 when sum_i b_i c_i^k = a_k for k = 0..P-1, where a_k are the
  Taylor coefficients of f (Eq. fB).  Given the c_i, the b_i solve a Vandermonde
  system.  Everything below is done in exact rational arithmetic (Fraction).
* Sec. 4.3, Eq. (ParallHybrid)/(Frac10): hybrid form d0 + d1 x + d2 x^2 +
  sum b_i/(1 - c_i x); b_i fixed by sum b_i c_i^k = a_k for k = 3..P+1 (with some
  b_i given as free parameters) and d_k = a_k - sum b_i c_i^k for k = 0, 1, 2.
* Sec. 3: forward bound eps(x) = sum_{k>s} |a_k - alpha_k| x^k with
  alpha_k = sum_i b_i c_i^k; theta = the x at which eps(x) reaches the tolerance.
* Eq. (Pade4)/(Pade4phi1): the 4th-order Pade forms written with one complex
  conjugate pair.

The paper prints several sets; the tests check that solving the systems above
reproduces every printed value exactly (see tests/test_oracle_coeffs.py).
"""
from fractions import Fraction as Fr
from math import factorial, sqrt
import cmath

# ---------------------------------------------------------------------------
# Taylor coefficients a_k of the target functions (Eq. fB)
# ---------------------------------------------------------------------------

def taylor_exp(k):
    """a_k for exp(x): 1/k!."""
    return Fr(1, factorial(k))


def taylor_phi1(k):
    """a_k for phi_1(x) = (e^x - 1)/x: 1/(k+1)!."""
    return Fr(1, factorial(k + 1))


def taylor_log1m(k):
    """a_k for log(1 - x): 0 for k = 0, -1/k otherwise (Sec. 2, the log example)."""
    return Fr(0) if k == 0 else Fr(-1, k)


def taylor_phi2(k):
    """a_k for phi_2(x) = (e^x - 1 - x)/x^2: 1/(k+2)! (Sec. 1, the phi-functions)."""
    return Fr(1, factorial(k + 2))


def taylor_cos(k):
    """a_k for cos(x): (-1)^(k/2)/k! for even k, 0 for odd k."""
    return Fr(0) if k % 2 else Fr((-1) ** (k // 2), factorial(k))


def taylor_sin(k):
    """a_k for sin(x): (-1)^((k-1)/2)/k! for odd k, 0 for even k."""
    return Fr((-1) ** ((k - 1) // 2), factorial(k)) if k % 2 else Fr(0)


TAYLOR = {"exp": taylor_exp, "phi1": taylor_phi1, "phi2": taylor_phi2, "log1m": taylor_log1m,
          "cos": taylor_cos, "sin": taylor_sin}


# ---------------------------------------------------------------------------
# Exact linear algebra over the rationals
# ---------------------------------------------------------------------------

def solve_exact(M, rhs):
    """Gauss-Jordan elimination over Fractions (exact); M is a list of rows."""
    n = len(M)
    A = [list(map(Fr, row)) + [Fr(r)] for row, r in zip(M, rhs)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [v / p for v in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [A[r][n] for r in range(n)]


def solve_b_plain(c, func):
    """b_i from Eq. (LinearEqsbi): sum_i b_i c_i^k = a_k, k = 0..P-1."""
    P = len(c)
    a = TAYLOR[func]
    M = [[Fr(ci) ** k for ci in c] for k in range(P)]
    return solve_exact(M, [a(k) for k in range(P)])


def solve_b_hybrid(c, free, func):
    """Hybrid form of Eq. (ParallHybrid)/(Frac10).

    c: the P-1 nodes; free: dict index -> given b_i (the free parameters).
    The remaining b_i solve sum_i b_i c_i^k = a_k for k = 3, 4, ... (as many
    equations as unknowns), then d_k = a_k - sum_i b_i c_i^k for k = 0, 1, 2.
    Returns (b, (d0, d1, d2)).
    """
    a = TAYLOR[func]
    n = len(c)
    unknown = [i for i in range(n) if i not in free]
    ks = list(range(3, 3 + len(unknown)))
    M = [[Fr(c[i]) ** k for i in unknown] for k in ks]
    rhs = [a(k) - sum(Fr(free[i]) * Fr(c[i]) ** k for i in free) for k in ks]
    sol = solve_exact(M, rhs)
    b = [None] * n
    for i, v in zip(unknown, sol):
        b[i] = v
    for i, v in free.items():
        b[i] = Fr(v)
    d = tuple(a(k) - sum(b[i] * Fr(c[i]) ** k for i in range(n)) for k in range(3))
    return b, d


# ---------------------------------------------------------------------------
# The coefficient sets of the paper
# ---------------------------------------------------------------------------

def _alpha_c(alpha, fracs):
    """c = (0, +-f/alpha for f in fracs): the symmetric choice of Eq. (Frac4ci)/(Frac8ci)."""
    c = [Fr(0)]
    for f in fracs:
        c += [Fr(f) / alpha, -Fr(f) / alpha]
    return c


class CoeffSet:
    """One rational approximant r(x) = d0 + d1 x + d2 x^2 + sum_i b_i / (1 - c_i x).

    Real sets carry exact Fractions.  Conjugate-pair sets (conj_pair=True) mean
    r(x) = d0 + 2 Re(sum_i b_i / (1 - c_i x)) with complex c_i, b_i.
    order: the s of Eq. (approx1); func: the target function name.
    """

    def __init__(self, name, c, b, func, order, d=(0, 0, 0), conj_pair=False,
                 taylor_of_r=None):
        self.name, self.c, self.b, self.func, self.order = name, c, b, func, order
        self.d = tuple(d)
        self.conj_pair = conj_pair
        self._taylor_of_r = taylor_of_r

    # Taylor coefficients alpha_k of r(x) (Sec. 3)
    def alpha(self, k):
        if self._taylor_of_r is not None:
            return self._taylor_of_r(k)
        s = sum(bi * ci ** k for bi, ci in zip(self.b, self.c))
        if k < 3:
            s += self.d[k]
        return s

    def a0(self):
        """Constant term of the roundoff form, Eq. (ParallRoundOff): r(0)."""
        if self.conj_pair:
            return float(self.d[0]) + 2.0 * sum(complex(bi).real for bi in self.b)
        return sum(self.b) + self.d[0]

    def as_float(self):
        """FP64 view (c_re, c_im, b_re, b_im, a0, d1, d2) of this set."""
        if self.conj_pair:
            c = [complex(v) for v in self.c]
            b = [complex(v) for v in self.b]
            return dict(c_re=[v.real for v in c], c_im=[v.imag for v in c],
                        b_re=[v.real for v in b], b_im=[v.imag for v in b],
                        a0=float(self.a0()), d1=float(self.d[1]), d2=float(self.d[2]),
                        conj_pair=1)
        return dict(c_re=[float(v) for v in self.c], c_im=[0.0] * len(self.c),
                    b_re=[float(v) for v in self.b], b_im=[0.0] * len(self.c),
                    a0=float(self.a0()), d1=float(self.d[1]), d2=float(self.d[2]),
                    conj_pair=0)


def _pade_series(num, den):
    """Exact Taylor coefficients of num(x)/den(x) (den[0] = 1) by the recurrence
    den(x) * sum_k q_k x^k = num(x)."""
    cache = []

    def q(k):
        while len(cache) <= k:
            j = len(cache)
            v = Fr(num[j]) if j < len(num) else Fr(0)
            for i in range(1, min(j, len(den) - 1) + 1):
                v -= Fr(den[i]) * cache[j - i]
            cache.append(v / Fr(den[0]))
        return cache[k]
    return q


def build_sets():
    """All coefficient sets printed in (or derived from) the paper."""
    S = {}
    # Sec. 2, Eq. (Frac4bi0) and the two lines after it: c_i = 1/(i+1), i = 1..5
    c5 = [Fr(1, i + 1) for i in range(1, 6)]
    S["frac4_exp"] = CoeffSet("frac4_exp", c5, solve_b_plain(c5, "exp"), "exp", 4)
    S["frac4_phi1"] = CoeffSet("frac4_phi1", c5, solve_b_plain(c5, "phi1"), "phi1", 4)
    S["frac4_log1m"] = CoeffSet("frac4_log1m", c5, solve_b_plain(c5, "log1m"), "log1m", 4)
    # Sec. 4.1, Eq. (Frac4ci)/(Frac4bi): R4, alpha = 5 (exp); alpha = 6 (phi1)
    c = _alpha_c(5, [1, Fr(1, 2)])
    S["R4"] = CoeffSet("R4", c, solve_b_plain(c, "exp"), "exp", 4)
    S["R4_phi1_a5"] = CoeffSet("R4_phi1_a5", c, solve_b_plain(c, "phi1"), "phi1", 4)
    c = _alpha_c(6, [1, Fr(1, 2)])
    S["R4_phi1"] = CoeffSet("R4_phi1", c, solve_b_plain(c, "phi1"), "phi1", 4)
    # Sec. 4.2, Eq. (Frac8ci)/(Frac8bi): R8, alpha = 5; the phi1 set with the
    # same c (Sec. 2: a new b for another function from the same resolvents)
    c = _alpha_c(5, [1, Fr(2, 3), Fr(1, 2), Fr(2, 5)])
    S["R8"] = CoeffSet("R8", c, solve_b_plain(c, "exp"), "exp", 8)
    S["R8_phi1"] = CoeffSet("R8_phi1", c, solve_b_plain(c, "phi1"), "phi1", 8)
    # Sec. 1: cos and sin (double-angle formulae) and phi_2 from the same R8
    # resolvents, their weights from Eq. (LinearEqsbi) with their Taylor a_k
    S["R8_cos"] = CoeffSet("R8_cos", c, solve_b_plain(c, "cos"), "cos", 8)
    S["R8_sin"] = CoeffSet("R8_sin", c, solve_b_plain(c, "sin"), "sin", 8)
    S["R8_phi2"] = CoeffSet("R8_phi2", c, solve_b_plain(c, "phi2"), "phi2", 8)
    # Sec. 4.4, Eq. (Frac5bi0): R5, c1 = 0, c_i = 1/(i+1), i = 2..6
    c = [Fr(0)] + [Fr(1, i + 1) for i in range(2, 7)]
    S["R5"] = CoeffSet("R5", c, solve_b_plain(c, "exp"), "exp", 5)
    # Sec. 4.3.1, Eq. (Frac10)/(Frac10ciNO): R10*, c_i = 1/(6+i), b9, b10 free
    c = [Fr(1, 6 + i) for i in range(1, 11)]
    b, d = solve_b_hybrid(c, {8: -50000, 9: 350000}, "exp")
    S["R10star"] = CoeffSet("R10star", c, b, "exp", 10, d=d)
    # Eq. (Frac10ci): R10, c_{2i-1} = -1/(6+2i), c_{2i} = 1/(6+2i)
    c = []
    for i in range(1, 6):
        c += [Fr(-1, 6 + 2 * i), Fr(1, 6 + 2 * i)]
    b, d = solve_b_hybrid(c, {8: 2000, 9: -3500}, "exp")
    S["R10"] = CoeffSet("R10", c, b, "exp", 10, d=d)
    # Eq. (Pade4): r22 = 1 + 2 Re(w/(x - z)), z = 3 - i sqrt(3), w = 6 + 6 sqrt(3) i
    # (the printed residue reads 6 sqrt(6); only 6 sqrt(3) reproduces r22, the
    # left-hand side of the same equation).  w/(x - z) = (-w/z)/(1 - x/z).
    z = complex(3.0, -sqrt(3.0))
    w = complex(6.0, 6.0 * sqrt(3.0))
    S["pade22"] = CoeffSet("pade22", [1 / z], [-w / z], "exp", 4, d=(Fr(1), 0, 0),
                           conj_pair=True,
                           taylor_of_r=_pade_series([1, Fr(1, 2), Fr(1, 12)],
                                                    [1, Fr(-1, 2), Fr(1, 12)]))
    # Eq. (Pade4phi1): 1/3 + 2 Re((7/3 + 8i)/(x - (4 - 2i)))
    z = complex(4.0, -2.0)
    w = complex(7.0 / 3.0, 8.0)
    S["pade22_phi1"] = CoeffSet("pade22_phi1", [1 / z], [-w / z], "phi1", 4,
                                d=(Fr(1, 3), 0, 0), conj_pair=True,
                                taylor_of_r=_pade_series([1, Fr(1, 10), Fr(1, 60)],
                                                         [1, Fr(-2, 5), Fr(1, 20)]))
    return S


SETS = build_sets()


# ---------------------------------------------------------------------------
# Forward error bound and theta (Sec. 3)
# ---------------------------------------------------------------------------

def forward_bound_coeffs(cs, kmax=200):
    """gamma_k = |a_k - alpha_k| for k = order+1 .. kmax, as floats of exact values."""
    a = TAYLOR[cs.func]
    out = []
    for k in range(cs.order + 1, kmax + 1):
        g = a(k) - cs.alpha(k)
        out.append((k, abs(float(g))))
    return out


def forward_bound(cs, x, gam=None):
    """eps(x) = sum_{k>s} |a_k - alpha_k| x^k (Sec. 3)."""
    gam = gam or forward_bound_coeffs(cs)
    return sum(g * x ** k for k, g in gam)


def theta(cs, tol, kmax=200):
    """theta = the x > 0 with eps(x) = tol (eps is increasing); bisection."""
    gam = forward_bound_coeffs(cs, kmax)
    lo, hi = 0.0, 1.0
    while forward_bound(cs, hi, gam) < tol:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if forward_bound(cs, mid, gam) < tol:
            lo = mid
        else:
            hi = mid
    return lo


def theta_taylor(m, tol, kmax=200):
    """theta for the degree-m Taylor polynomial: eps(x) = sum_{k>m} x^k/k! (Table 1)."""
    inv_fact = [float(Fr(1, factorial(k))) for k in range(kmax)]

    def eps(x):
        return sum(x ** k * inv_fact[k] for k in range(m + 1, kmax))
    lo, hi = 0.0, 1.0
    while eps(hi) < tol:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if eps(mid) < tol:
            lo = mid
        else:
            hi = mid
    return lo


U_FP64 = 2.0 ** -53
U_FP32 = 2.0 ** -24


def oracle_coeffs(name, tol=U_FP64):
    """FP64 view of a set plus its theta at tolerance tol (default FP64 unit roundoff)."""
    cs = SETS[name]
    f = cs.as_float()
    f["theta"] = theta(cs, tol)
    f["order"] = cs.order
    f["name"] = name
    return f
