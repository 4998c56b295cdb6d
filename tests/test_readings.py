"""Exact checks, in rational arithmetic on small matrices (no GPU), of the
algebra the grid paths use to combine the shifted systems of Eq.
(ParallRoundOff): one system I - c^2 B^2 for a pair of nodes +-c, one real
system I - 2 Re(c) B + |c|^2 B^2 for a conjugate pair (Sec. 1: one product
x^2 and one inverse per pair of roots), the one-product combination of the
pairs' B-terms, and the first correction step of C = u B^2 taken from the
powers B^2, B^4, B^6.  The parity tests check the kernels' end results; these
check the identities those kernels rest on, so a wrong sign or weight in the
reading fails here on its own.
"""
from fractions import Fraction as Fr

import pytest

from oracle import coeffs as oc


# ---- exact matrices (lists of rows of Fractions) -------------------------
def eye(n):
    return [[Fr(int(i == j)) for j in range(n)] for i in range(n)]


def add(A, B, a=1, b=1):
    return [[a * x + b * y for x, y in zip(r, s)] for r, s in zip(A, B)]


def scale(A, a):
    return [[a * x for x in r] for r in A]


def mul(A, B):
    n, m, k = len(A), len(B[0]), len(B)
    return [[sum(A[i][p] * B[p][j] for p in range(k)) for j in range(m)] for i in range(n)]


def inv(A):
    n = len(A)
    M = [list(r) + e for r, e in zip(A, eye(n))]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        pv = M[c][c]
        M[c] = [x / pv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [r[n:] for r in M]


B0 = [[Fr(3, 50), Fr(-1, 40), Fr(1, 25)],
      [Fr(1, 30), Fr(2, 45), Fr(-1, 60)],
      [Fr(-1, 35), Fr(1, 20), Fr(-3, 70)]]


def r8_pairs():
    """(c, b+, b-) for each +-c pair of R8, exact."""
    cs = oc.SETS["R8"]
    out = []
    for i, c in enumerate(cs.c):
        if c > 0:
            j = cs.c.index(-c)
            out.append((c, cs.b[i], cs.b[j]))
    return out


def test_r8_has_four_pairs():
    assert len(r8_pairs()) == 4 and sum(1 for c in oc.SETS["R8"].c if c == 0) == 1


@pytest.mark.parametrize("q", range(4))
def test_pair_fusion_and_one_product_combination(q):
    """b+ (I - cB)^-1 cB + b- (I + cB)^-1 (-cB)
         = (I - c^2 B^2)^-1 [(b+ - b-) cB + (b+ + b-) c^2 B^2]        (one system)
         = a B + a Y B + (b+ + b-) Y,  a = (b+ - b-) c,  Y = (I - c^2 B^2)^-1 - I
    (the pair adds (b+ + b-) Y to F and a Y to G; G B and (sum a) B come once,
    after the last pair)."""
    c, bp, bm = r8_pairs()[q]
    n = len(B0)
    I = eye(n)
    cB = scale(B0, c)
    lhs = add(scale(mul(inv(add(I, cB, 1, -1)), cB), bp),
              scale(mul(inv(add(I, cB)), scale(cB, -1)), bm))
    B2 = mul(B0, B0)
    M = add(I, scale(B2, c * c), 1, -1)
    fused = mul(inv(M), add(scale(cB, bp - bm), scale(B2, (bp + bm) * c * c)))
    assert fused == lhs
    Y = add(inv(M), I, 1, -1)
    a = (bp - bm) * c
    comb = add(add(scale(B0, a), scale(mul(Y, B0), a)), scale(Y, bp + bm))
    assert comb == lhs


@pytest.mark.parametrize("q", range(4))
def test_first_correction_from_powers(q):
    """From Y0 = C = u B^2 the correction E = C - (I - C) Y, Y <- Y + E (I + Y)
    gives Y1 = u B^2 + u^2 B^4 + u^3 B^6, whose residual is u^4 B^8 (the
    residual squares); the step-0 residual is u^2 B^4."""
    c = r8_pairs()[q][0]
    u = c * c
    n = len(B0)
    I = eye(n)
    B2 = mul(B0, B0)
    B4 = mul(B2, B2)
    B6 = mul(B4, B2)
    C = scale(B2, u)
    E0 = add(C, mul(add(I, C, 1, -1), C), 1, -1)
    assert E0 == scale(B4, u ** 2)
    Y1 = add(C, mul(E0, add(I, C)))
    assert Y1 == add(add(scale(B2, u), scale(B4, u ** 2)), scale(B6, u ** 3))
    E1 = add(C, mul(add(I, C, 1, -1), Y1), 1, -1)
    assert E1 == scale(mul(B4, B4), u ** 4)


def test_shared_pass_is_one_polynomial():
    """Sum over the pairs finished at step 0 of y_q Y1_q equals
    a1 B^2 + a2 B^4 + a3 B^6 with a_k = sum_q y_q u_q^k (likewise for G)."""
    B2 = mul(B0, B0)
    B4 = mul(B2, B2)
    B6 = mul(B4, B2)
    tot = scale(B2, 0)
    a = [Fr(0)] * 3
    for c, bp, bm in r8_pairs():
        u, y = c * c, bp + bm
        Y1 = add(add(scale(B2, u), scale(B4, u ** 2)), scale(B6, u ** 3))
        tot = add(tot, scale(Y1, y))
        for k in range(3):
            a[k] += y * u ** (k + 1)
    assert tot == add(add(scale(B2, a[0]), scale(B4, a[1])), scale(B6, a[2]))


# ---- Gaussian rationals for the conjugate-pair identities ------------------
class Q:
    def __init__(self, re, im=0):
        self.re, self.im = Fr(re), Fr(im)

    def __add__(self, o):
        o = o if isinstance(o, Q) else Q(o)
        return Q(self.re + o.re, self.im + o.im)

    __radd__ = __add__

    def __sub__(self, o):
        o = o if isinstance(o, Q) else Q(o)
        return Q(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        o = o if isinstance(o, Q) else Q(o)
        return Q(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = o if isinstance(o, Q) else Q(o)
        den = o.re * o.re + o.im * o.im
        return Q((self.re * o.re + self.im * o.im) / den, (self.im * o.re - self.re * o.im) / den)

    def conj(self):
        return Q(self.re, -self.im)


CONJ = [(Q(Fr(1, 5), Fr(1, 7)), Q(Fr(2, 3), Fr(-3, 4))), (Q(0, Fr(1, 4)), Q(Fr(-5, 2), Fr(1, 3)))]


@pytest.mark.parametrize("cb", CONJ)
def test_conjugate_pair_scalar_forms(cb):
    """2 Re(b c x / (1 - c x)) = (2 Re(bc) x - 2 Re(b) |c|^2 x^2) / (1 - 2 Re(c) x + |c|^2 x^2)
    (roundoff form) and 2 Re(b / (1 - c x)) = (2 Re(b) - 2 Re(b conj(c)) x) / (same)
    (plain form), at several rational x."""
    c, b = cb
    c2 = c.re * c.re + c.im * c.im
    for x in (Fr(1, 10), Fr(-3, 17), Fr(2, 9)):
        den = 1 - 2 * c.re * x + c2 * x * x
        t = (b * c * Q(x)) / (Q(1) - c * Q(x))
        assert 2 * t.re == (2 * (b * c).re * x - 2 * b.re * c2 * x * x) / den
        p = b / (Q(1) - c * Q(x))
        assert 2 * p.re == (2 * b.re - 2 * (b * c.conj()).re * x) / den


def test_quadratic_system_one_product_combination():
    """With M = I - u1 B - u2 B^2 and Y = M^-1 - I:
    M^-1 (g I + a B + b B^2) = g I + (g + b/u2) Y + (a - b u1/u2)(I + Y) B."""
    n = len(B0)
    I = eye(n)
    B2 = mul(B0, B0)
    u1, u2 = Fr(2, 5), Fr(-3, 35)
    g, a, b = Fr(7, 3), Fr(-11, 6), Fr(5, 4)
    M = add(add(I, scale(B0, u1), 1, -1), scale(B2, u2), 1, -1)
    Mi = inv(M)
    lhs = mul(Mi, add(add(scale(I, g), scale(B0, a)), scale(B2, b)))
    Y = add(Mi, I, 1, -1)
    rhs = add(add(scale(I, g), scale(Y, g + b / u2)), scale(mul(add(I, Y), B0), a - b * u1 / u2))
    assert lhs == rhs
