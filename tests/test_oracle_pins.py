"""Pins for the FP64 C oracle (oracle/fm_oracle.c) against things other than itself.

Parity status per oracle function:
  orc_norm1, orc_select_s/nsteps ... closed forms                      pinned
  orc_gepp / getrs / getrs_trans ... reconstruction, crafted pivots    pinned
  orc_rational_apply (real, plain and roundoff forms)
                                 ... exact rational sums on nilpotent
                                     matrices, diagonal scalars        pinned
  conj-pair sets (Pade, Eq. Pade4/Pade4phi1) ... textbook quadratic
                                     ratio solved with numpy           pinned
  orc_expm ... symmetric/diagonal/rotation closed forms in 50-digit
               arithmetic, invariants e^A e^-A = I                     pinned
  orc_phi1 ... (e^x-1)/x on eigenvalues, augmented-matrix identity     pinned
  orc_expmv ... N = 2^s equals expm(A) V, diagonal closed form         pinned
  orc_phi1mv ... phi1(A) V product of a pinned matrix                  pinned
  orc_expmv_adjoint ... central finite differences, full FD at d = 4   pinned
  orc_zexpm / zexpmv ... Hermitian closed form, unitarity              pinned
  orc_trig (cos, sin; double angle) ... nilpotent Taylor sums, 50-digit
               scalar recurrence on eigenvalues, Re/Im of the complex
               exponential, cos^2 + sin^2 = I (tests/test_oracle_functions.py) pinned
  orc_rfun (r(tA), no range reduction; log(1 - x), phi_2) ... nilpotent
               Taylor sums, 50-digit scalars, the forward bound of Sec. 3
               against log(1 - x) (tests/test_oracle_functions.py)   pinned
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import coeffs as oc

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50


def rng(seed):
    return np.random.default_rng(seed)


def r_scalar(cs, x):
    """r(x) in 50-digit arithmetic from the exact set (Eq. rat1 / ParallHybrid)."""
    x = mp.mpmathify(x)
    if cs.conj_pair:
        v = mp.mpf(float(cs.d[0]))
        for c, b in zip(cs.c, cs.b):
            c, b = mp.mpc(complex(c)), mp.mpc(complex(b))
            v += 2 * mp.re(b / (1 - c * x))
        return v
    v = mp.mpf(cs.d[0].numerator) / cs.d[0].denominator if cs.d[0] else mp.mpf(0)
    v += mp.mpf(cs.d[1].numerator) / cs.d[1].denominator * x if cs.d[1] else 0
    v += mp.mpf(cs.d[2].numerator) / cs.d[2].denominator * x * x if cs.d[2] else 0
    for c, b in zip(cs.c, cs.b):
        c = mp.mpf(c.numerator) / c.denominator
        b = mp.mpf(b.numerator) / b.denominator
        v += b / (1 - c * x)
    return v


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------------------------
# basic pieces
# ----------------------------------------------------------------------------

def test_norm1_and_select():
    A = np.array([[1.0, -2.0], [-3.0, 0.5]])
    assert oracle.norm1(A) == 4.0
    th = 0.0973104
    assert oracle.select_s(th, th) == 0
    assert oracle.select_s(th * 8, th) == 3
    assert oracle.select_s(th * 8 * (1 + 1e-15), th) == 4
    assert oracle.select_s(0.0, th) == 0
    assert oracle.select_nsteps(2.5 * th, th) == 3
    assert oracle.select_nsteps(0.0, th) == 1


def test_gepp_reconstructs_and_pivots():
    A = rng(1).standard_normal((7, 7))
    LU, piv, info = oracle.gepp(A)
    assert info == 0
    L = np.tril(LU, -1) + np.eye(7)
    U = np.triu(LU)
    PA = A.copy()
    for k, p in enumerate(piv):
        PA[[k, p]] = PA[[p, k]]
    assert np.abs(L @ U - PA).max() < 1e-14
    assert np.abs(L).max() <= 1.0
    # crafted: the largest entry of column 0 sits in row 2; ties keep the lowest row
    M = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [5.0, 0.0, 1.0]])
    _, piv, _ = oracle.gepp(M)
    assert piv[0] == 2
    M = np.array([[2.0, 1.0], [-2.0, 3.0]])
    _, piv, _ = oracle.gepp(M)
    assert piv[0] == 0


def test_gepp_zero_pivot_and_solves():
    S = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]])
    _, _, info = oracle.gepp(S)
    assert info == 3
    A = rng(2).standard_normal((9, 9)) + 5 * np.eye(9)
    X = rng(3).standard_normal((9, 4))
    LU, piv, _ = oracle.gepp(A)
    assert np.abs(A @ oracle.getrs(LU, piv, X) - X).max() < 1e-13
    assert np.abs(A.T @ oracle.getrs(LU, piv, X, trans=True) - X).max() < 1e-13


# ----------------------------------------------------------------------------
# the approximant itself
# ----------------------------------------------------------------------------

def _exact_poly(cs, Bq, n, form):
    """sum_k alpha_k B^k over exact Fractions for nilpotent B (B^n = 0)."""
    def matmul(X, Y):
        return [[sum(X[i][l] * Y[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
    P = [[Fr(int(i == j)) for j in range(n)] for i in range(n)]
    out = [[Fr(0)] * n for _ in range(n)]
    for k in range(n):
        a = cs.alpha(k)
        for i in range(n):
            for j in range(n):
                out[i][j] += a * P[i][j]
        P = matmul(P, Bq)
    return np.array([[float(v) for v in row] for row in out])


@pytest.mark.parametrize("name", ["R4", "R8", "R8_phi1", "R10", "frac4_log1m", "R8_cos", "R8_sin",
                                  "R8_phi2"])
@pytest.mark.parametrize("form", [oracle.ROUNDOFF, oracle.PLAIN])
def test_nilpotent_exact(name, form):
    """B strictly upper triangular (B^n = 0): r(B) = sum_{k<n} alpha_k B^k exactly
    (Sec. 3, alpha_k = sum_i b_i c_i^k).  Pins every b_i, c_i, the sign of each
    term and the operand order (a transposed B would give a lower triangle)."""
    n = 10
    g = rng(4)
    Bq = [[Fr(int(g.integers(-40, 41)), 256) if j > i else Fr(0) for j in range(n)]
          for i in range(n)]
    B = np.array([[float(v) for v in row] for row in Bq])
    ref = _exact_poly(oc.SETS[name], Bq, n, form)
    (out,), info = oracle.rational_apply(B, [oracle.CS(name)], form)
    assert info == 0
    # the plain form cancels sum_i |b_i| on the diagonal (Sec. 4.3), so its
    # round-off scales with that sum; the roundoff form does not
    cs = oc.SETS[name]
    sum_b = sum(abs(float(b)) for b in cs.b) + sum(abs(float(d)) for d in cs.d)
    tol = 4 * sum_b * 2.0 ** -53 if form == oracle.PLAIN else 1e-13
    if name == "R10":
        tol = max(tol, 1e-11)
    assert np.abs(out - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_nilpotent_index_reaches_taylor():
    """Jordan block of index <= s+1: r(B) is exactly the Taylor sum (pin P4)."""
    n = 9
    J = np.diag(np.full(n - 1, 0.0625), 1)
    (out,), _ = oracle.rational_apply(J, [oracle.CS("R8")])
    from math import factorial
    ref = sum(np.linalg.matrix_power(J, k) / factorial(k) for k in range(n))
    assert np.abs(out - ref).max() < 1e-14


@pytest.mark.parametrize("name", ["R4", "R8", "R5", "R10"])
def test_diagonal_scalar(name):
    cs = oc.SETS[name]
    xs = np.array([-0.09, -0.03, 0.0, 0.011, 0.05, 0.09]) * (2 if name == "R10" else 1)
    (out,), _ = oracle.rational_apply(np.diag(xs), [oracle.CS(name)])
    ref = np.array([float(r_scalar(cs, x)) for x in xs])
    # round-off of Eq. ParallRoundOff grows with the cancelling sum |b_i c_i x|
    canc = [sum(abs(float(b) * float(c) * x / (1 - float(c) * x)) for b, c in zip(cs.b, cs.c))
            + abs(float(cs.d[1]) * x) + abs(float(cs.d[2]) * x * x) for x in xs]
    tol = 8 * 2.0 ** -53 * (np.array(canc) + 1)
    assert np.all(np.abs(np.diag(out) - ref) <= tol)
    assert np.abs(out - np.diag(np.diag(out))).max() == 0


@pytest.mark.parametrize("name,num,den", [
    ("pade22", (1, 0.5, 1 / 12), (1, -0.5, 1 / 12)),
    ("pade22_phi1", (1, 0.1, 1 / 60), (1, -0.4, 1 / 20))])
@pytest.mark.parametrize("form", [oracle.ROUNDOFF, oracle.PLAIN])
def test_conj_pair_is_pade_ratio(name, num, den, form):
    """Pin P7: the one-complex-pair forms equal den(B)^{-1} num(B)."""
    B = rng(5).standard_normal((12, 12)) * 0.05
    I = np.eye(12)
    ref = np.linalg.solve(den[0] * I + den[1] * B + den[2] * B @ B,
                          num[0] * I + num[1] * B + num[2] * B @ B)
    (out,), info = oracle.rational_apply(B, [oracle.CS(name)], form)
    assert info == 0 and relerr(out, ref) < 1e-14


def test_shared_resolvents_two_functions():
    """Sec. 2: exp and phi1 from the same resolvents give the two separate results."""
    B = rng(6).standard_normal((16, 16)) * 0.005
    outs, _ = oracle.rational_apply(B, [oracle.CS("R8"), oracle.CS("R8_phi1")])
    (e,), _ = oracle.rational_apply(B, [oracle.CS("R8")])
    (p,), _ = oracle.rational_apply(B, [oracle.CS("R8_phi1")])
    assert np.array_equal(outs[0], e) and np.array_equal(outs[1], p)


# ----------------------------------------------------------------------------
# scaling and squaring
# ----------------------------------------------------------------------------

def _sym(n, seed, norm1):
    g = rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = g.uniform(-1, 1, n)
    A = (Q * lam) @ Q.T
    s = norm1 / np.abs(A).sum(0).max()
    return A * s, Q, lam * s


@pytest.mark.parametrize("name", ["R4", "R8"])
def test_expm_symmetric_closed_form(name):
    """Pin P3: A = Q diag(l) Q^T gives Q diag(r(l/2^s)^(2^s)) Q^T."""
    A, Q, lam = _sym(24, 7, 6.0)
    F, s, info = oracle.expm(A, 1.0, name)
    cs = oc.SETS[name]
    sc = np.array([float(r_scalar(cs, mp.mpf(float(l)) / 2 ** s) ** (2 ** s)) for l in lam])
    ref = (Q * sc) @ Q.T
    assert info == 0 and relerr(F, ref) < 5e-13
    ex = (Q * np.exp(lam)) @ Q.T
    assert relerr(F, ex) < 5e-13


def test_expm_diagonal_and_t():
    d = np.array([-3.0, -0.5, 0.25, 1.5, 2.0])
    F, s, _ = oracle.expm(np.diag(d), 0.75, "R8")
    cs = oc.SETS["R8"]
    ref = [float(r_scalar(cs, mp.mpf(0.75) * mp.mpf(x) / 2 ** s) ** (2 ** s)) for x in d]
    assert s == oracle.select_s(0.75 * 3.0, oracle.CS("R8").theta)
    # squaring doubles a relative error s times; sum_i |b_i c_i| theta ~ 51 for R8
    tol = 2 ** s * 64 * 2.0 ** -53
    assert np.all(np.abs(np.diag(F) - ref) <= tol * np.abs(ref))


def test_expm_rotation():
    """Pin P6: exp of [[0,-w],[w,0]] is the rotation by w; the approximant gives
    the rotation with z = r(i w / 2^s)^(2^s)."""
    w = 2.7
    A = np.array([[0.0, -w], [w, 0.0]])
    F, s, _ = oracle.expm(A, 1.0, "R8")
    cs = oc.SETS["R8"]
    x = mp.mpc(0, w) / 2 ** s
    v = mp.mpf(0)
    for c, b in zip(cs.c, cs.b):
        v += (mp.mpf(b.numerator) / b.denominator) / (1 - mp.mpf(c.numerator) / c.denominator * x)
    z = v ** (2 ** s)
    ref = np.array([[float(mp.re(z)), -float(mp.im(z))], [float(mp.im(z)), float(mp.re(z))]])
    tol = 2 ** s * 64 * 2.0 ** -53
    assert np.abs(F - ref).max() < tol
    assert abs(F[0, 0] - np.cos(w)) < tol and abs(F[1, 0] - np.sin(w)) < tol


def test_expm_invariants():
    """Pin P9: e^A e^-A = I; e^{tA} e^{sA} = e^{(t+s)A}; vs a library routine."""
    sl = pytest.importorskip("scipy.linalg")
    A = rng(8).standard_normal((40, 40))
    A *= 3.0 / np.abs(A).sum(0).max()
    E1, _, _ = oracle.expm(A, 1.0)
    E2, _, _ = oracle.expm(A, -1.0)
    assert np.abs(E1 @ E2 - np.eye(40)).max() < 5e-13
    Ea, _, _ = oracle.expm(A, 0.3)
    Eb, _, _ = oracle.expm(A, 0.45)
    Ec, _, _ = oracle.expm(A, 0.75)
    assert relerr(Ea @ Eb, Ec) < 1e-13
    assert relerr(E1, sl.expm(A)) < 1e-13


def test_roundoff_form_beats_plain():
    """Eq. ParallRoundOff: smaller round-off than the plain form (Sec. 4.3)."""
    sl = pytest.importorskip("scipy.linalg")
    worse = 0
    for seed in range(4):
        A = rng(20 + seed).standard_normal((32, 32))
        A *= 4.0 / np.abs(A).sum(0).max()
        ex = sl.expm(A)
        e_r = relerr(oracle.expm(A, 1.0, "R8")[0], ex)
        e_p = relerr(oracle.expm(A, 1.0, "R8", form=oracle.PLAIN)[0], ex)
        worse += e_p > 5 * e_r
    assert worse >= 3


def test_r10_roundoff_vs_r10star():
    """Sec. 5 (Fig. 3): R10 has round-off errors about three orders of magnitude
    below R10* on randn(100) at h||A|| near 1 and above."""
    sl = pytest.importorskip("scipy.linalg")
    A = rng(9).standard_normal((100, 100))
    A *= 2.0 / np.abs(A).sum(0).max()
    ex = sl.expm(A)
    e10 = relerr(oracle.expm(A, 1.0, "R10", form=oracle.PLAIN)[0], ex)
    e10s = relerr(oracle.expm(A, 1.0, "R10star", form=oracle.PLAIN)[0], ex)
    assert e10s > 30 * e10


# ----------------------------------------------------------------------------
# phi1
# ----------------------------------------------------------------------------

def test_phi1_eigen_closed_form():
    A, Q, lam = _sym(20, 10, 5.0)
    Phi, E, s, info = oracle.phi1(A, 1.0)
    ph = np.array([float(mp.expm1(mp.mpf(float(l))) / mp.mpf(float(l))) for l in lam])
    assert info == 0 and relerr(Phi, (Q * ph) @ Q.T) < 5e-13
    assert relerr(E, (Q * np.exp(lam)) @ Q.T) < 5e-13


def test_phi1_augmented_identity():
    """exp([[A, I], [0, 0]]) has phi1(A) as its top-right block (pin P9)."""
    n = 16
    A = rng(11).standard_normal((n, n))
    A *= 2.0 / np.abs(A).sum(0).max()
    Phi, E, _, _ = oracle.phi1(A, 1.0)
    aug = np.zeros((2 * n, 2 * n))
    aug[:n, :n] = A
    aug[:n, n:] = np.eye(n)
    F, _, _ = oracle.expm(aug, 1.0)
    assert relerr(Phi, F[:n, n:]) < 1e-13
    assert relerr(E, F[:n, :n]) < 1e-13
    assert relerr(A @ Phi, E - np.eye(n)) < 1e-13


def test_phi1_t_scaling():
    A = rng(12).standard_normal((12, 12)) * 0.4
    t = 0.37
    Phi, E, _, _ = oracle.phi1(A, t)
    assert relerr(t * A @ Phi, E - np.eye(12)) < 1e-13


# ----------------------------------------------------------------------------
# action
# ----------------------------------------------------------------------------

def test_expmv_equals_matrix_route():
    """Pin P5: N = 2^s steps of r(A/N) on V equal (r(A/2^s))^(2^s) V."""
    A = rng(13).standard_normal((30, 30))
    A *= 2.0 / np.abs(A).sum(0).max()
    V = rng(14).standard_normal((30, 3))
    F, s, _ = oracle.expm(A, 1.0)
    W, N, info = oracle.expmv(A, V, 1.0, nsteps=2 ** s)
    assert info == 0 and N == 2 ** s and relerr(W, F @ V) < 1e-13
    W2, N2, _ = oracle.expmv(A, V[:, 0])
    assert N2 == oracle.select_nsteps(np.abs(A).sum(0).max(), oracle.CS("R8").theta)
    assert relerr(W2, F @ V[:, 0]) < 1e-13


def test_expmv_diagonal_closed_form():
    d = np.array([-1.0, -0.2, 0.3, 0.9])
    v = np.array([1.0, -2.0, 0.5, 3.0])
    W, N, _ = oracle.expmv(np.diag(d), v, 1.0, "R4")
    cs = oc.SETS["R4"]
    h = mp.mpf(1) / N
    ref = [float(r_scalar(cs, mp.mpf(x) * h) ** N) * vi for x, vi in zip(d, v)]
    assert np.abs(W - ref).max() < 1e-13


@pytest.mark.parametrize("name", ["R10", "R5"])
def test_expmv_trid_sine_closed_form(name):
    """The matrix of Sec. 5 (Fig. 4), A = trid{-1,2,-1}: its eigenvectors are the
    sine vectors q_j(k) = sqrt(2/(d+1)) sin(j k pi/(d+1)) with eigenvalues
    2 - 2 cos(j pi/(d+1)), so N steps of the action are Q diag(r(h l_j)^N) Q^T v
    with r in 50-digit arithmetic.  This pins the reference of the tridiagonal
    path's parity tests on the paper's own example."""
    d, t = 40, 0.6
    A = 2 * np.eye(d) - np.eye(d, k=1) - np.eye(d, k=-1)
    j = np.arange(1, d + 1)
    Q = np.sqrt(2.0 / (d + 1)) * np.sin(np.outer(j, j) * np.pi / (d + 1))
    lam = 2 - 2 * np.cos(j * np.pi / (d + 1))
    v = rng(31).standard_normal(d)
    v /= np.linalg.norm(v)
    W, N, info = oracle.expmv(A, v, t, name)
    theta = oracle.CS(name).theta
    assert info == 0 and N == oracle.select_nsteps(4 * t, theta)
    cs = oc.SETS[name]
    h = mp.mpf(t) / N
    g = np.array([float(r_scalar(cs, h * mp.mpf(float(l))) ** N) for l in lam])
    ref = Q @ (g * (Q.T @ v))
    # N steps of the roundoff form each round at u (sum_i |b_i c_i| theta + 1)
    # (Sec. 4.3): 5e-12 for R10's large weights, 2e-13 for R5
    bc = sum(abs(float(b) * float(c)) for b, c in zip(cs.b, cs.c))
    tol = max(5e-13, 2 * N * 2.0 ** -53 * (bc * theta + 1))
    assert relerr(W, ref) < tol
    assert relerr(W, Q @ (np.exp(t * lam) * (Q.T @ v))) < tol + 1e-13


def test_phi1mv():
    A = rng(15).standard_normal((20, 20)) * 0.2
    V = rng(16).standard_normal((20, 2))
    Phi, _, _, _ = oracle.phi1(A, 0.8)
    W, _, _ = oracle.phi1mv(A, V, 0.8)
    assert relerr(W, Phi @ V) < 1e-15


# ----------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------

def _loss(A, v, y, N):
    w, _, _ = oracle.expmv(A, v, 1.0, nsteps=N)
    return float(np.sum((w - y) ** 2)), w


def test_adjoint_directional_fd():
    """Pin P10: central differences of L = ||w_N - y||^2 with N fixed.  h = 1e-5
    sits at the bottom of the FD error curve here (truncation ~2.5e-8, round-off
    of the 38-step forward ~1.5e-7 absolute on L ~ 30)."""
    n = 12
    g = rng(17)
    A = g.standard_normal((n, n)) / np.sqrt(n)
    N = oracle.select_nsteps(np.abs(A).sum(0).max(), oracle.CS("R8").theta)
    v, y = g.standard_normal(n), g.standard_normal(n)
    L0, w = _loss(A, v, y, N)
    Ab, vb, info = oracle.expmv_adjoint(A, v, 2 * (w - y), N)
    assert info == 0
    for seed in range(3):
        dA = rng(30 + seed).standard_normal((n, n))
        dv = rng(40 + seed).standard_normal(n)
        h = 1e-5
        fd = (_loss(A + h * dA, v + h * dv, y, N)[0] - _loss(A - h * dA, v - h * dv, y, N)[0]) / (2 * h)
        an = np.sum(Ab * dA) + np.dot(vb, dv)
        assert abs(fd - an) <= 2e-7 * max(1.0, abs(an))


def test_adjoint_full_fd_tiny():
    n = 4
    g = rng(18)
    A = g.standard_normal((n, n)) * 0.5
    N = oracle.select_nsteps(np.abs(A).sum(0).max(), oracle.CS("R8").theta)
    v, y = g.standard_normal(n), g.standard_normal(n)
    _, w = _loss(A, v, y, N)
    Ab, vb, _ = oracle.expmv_adjoint(A, v, 2 * (w - y), N)
    h = 1e-6
    for i in range(n):
        for j in range(n):
            E = np.zeros((n, n))
            E[i, j] = h
            fd = (_loss(A + E, v, y, N)[0] - _loss(A - E, v, y, N)[0]) / (2 * h)
            assert abs(fd - Ab[i, j]) < 1e-7 * max(1.0, abs(fd))
        e = np.zeros(n)
        e[i] = h
        fd = (_loss(A, v + e, y, N)[0] - _loss(A, v - e, y, N)[0]) / (2 * h)
        assert abs(fd - vb[i]) < 1e-7 * max(1.0, abs(fd))


# ----------------------------------------------------------------------------
# complex
# ----------------------------------------------------------------------------

def _herm(n, seed, rho):
    g = rng(seed)
    G = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(n)
    H = (G + G.conj().T) / 2
    lam, Q = np.linalg.eigh(H)
    f = rho / np.abs(lam).max()
    return H * f, Q, lam * f


def test_zexpm_hermitian_closed_form():
    H, Q, lam = _herm(16, 19, 6.0)
    A = -1j * H
    F, s, info = oracle.zexpm(A, 1.0)
    assert info == 0
    ref = (Q * np.exp(-1j * lam)) @ Q.conj().T
    assert relerr(F, ref) < 5e-13
    assert np.abs(F.conj().T @ F - np.eye(16)).max() < 5e-13


def test_zexpm_matches_real_path_on_real_input():
    A = rng(21).standard_normal((10, 10)) * 0.3
    Fr_, _, _ = oracle.expm(A, 1.0)
    Fz, _, _ = oracle.zexpm(A.astype(complex), 1.0)
    assert np.abs(Fz.imag).max() == 0 and relerr(Fz.real, Fr_) < 1e-14


def test_zexpmv_unitary_action():
    H, Q, lam = _herm(24, 22, 20.0)
    A = -1j * H
    V = rng(23).standard_normal((24, 3)) + 1j * rng(24).standard_normal((24, 3))
    W, N, _ = oracle.zexpmv(A, V, 1.0, anorm=20.0)
    assert N == oracle.select_nsteps(20.0, oracle.CS("R8").theta)
    ref = (Q * np.exp(-1j * lam)) @ (Q.conj().T @ V)
    assert relerr(W, ref) < 1e-12
    assert np.abs(np.linalg.norm(W, axis=0) / np.linalg.norm(V, axis=0) - 1).max() < 1e-12


def test_batched_driver_matches_single():
    mats = [rng(50 + i).standard_normal((d, d)) / np.sqrt(d) for i, d in enumerate([3, 8, 5])]
    ts = np.array([1.0, 0.5, 2.0])
    outs, s, info = oracle.expm_batched(mats, ts)
    for M, t, F in zip(mats, ts, outs):
        assert np.array_equal(F, oracle.expm(M, t)[0])


def test_nonfinite_input_reports():
    A = np.eye(3)
    A[1, 2] = np.nan
    _, _, info = oracle.expm(A)
    assert info == -2
