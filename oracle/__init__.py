"""FP64 CPU oracle for the parallel shifted-solve matrix functions of
Blanes, arXiv:2210.03714 -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  It shares no code with the CUDA library.  The
numerical work is the plain C in fm_oracle.c (textbook GEPP, the roundoff
form of Eq. ParallRoundOff, scaling and squaring, the action recurrence, the
phi_1 doubling and the adjoint of the action map); exact coefficient sets and
the forward-bound theta of Sec. 3 live in coeffs.py.

Parity status of each function (what pins it) is listed in the header of
tests/test_oracle_pins.py.
"""
import ctypes as C
import os
import subprocess

import numpy as np

from . import coeffs as _coeffs

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

ROUNDOFF, PLAIN = 0, 1


def build(force=False):
    """Compile fm_oracle.c with gcc (-ffp-contract=off: every operation rounds as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Coeffs(C.Structure):
    _fields_ = [("k", C.c_int),
                ("c_re", C.POINTER(C.c_double)), ("c_im", C.POINTER(C.c_double)),
                ("b_re", C.POINTER(C.c_double)), ("b_im", C.POINTER(C.c_double)),
                ("conj_pair", C.c_int),
                ("a0", C.c_double), ("d1", C.c_double), ("d2", C.c_double),
                ("theta", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_long)
        cp = C.POINTER(Coeffs)
        L = _lib
        L.orc_norm1.restype = C.c_double
        L.orc_norm1.argtypes = [C.c_int, dp]
        L.orc_select_s.restype = C.c_int
        L.orc_select_s.argtypes = [C.c_double, C.c_double]
        L.orc_select_nsteps.restype = C.c_long
        L.orc_select_nsteps.argtypes = [C.c_double, C.c_double]
        L.orc_gepp.argtypes = [C.c_int, dp, ip]
        L.orc_getrs.argtypes = [C.c_int, dp, ip, C.c_int, dp]
        L.orc_getrs_trans.argtypes = [C.c_int, dp, ip, C.c_int, dp]
        L.orc_rational_apply.argtypes = [C.c_int, dp, C.c_int, C.POINTER(cp), C.c_int, C.c_int,
                                         dp, C.POINTER(dp)]
        L.orc_expm.argtypes = [C.c_int, dp, C.c_double, cp, C.c_int, C.c_double, C.c_int, dp, ip]
        L.orc_phi1.argtypes = [C.c_int, dp, C.c_double, cp, cp, C.c_int, C.c_double, C.c_int,
                               dp, dp, ip]
        L.orc_trig.argtypes = [C.c_int, dp, C.c_double, cp, cp, C.c_int, C.c_double, C.c_int,
                               dp, dp, ip]
        L.orc_rfun.argtypes = [C.c_int, dp, C.c_double, cp, C.c_int, dp]
        L.orc_expmv.argtypes = [C.c_int, dp, C.c_double, cp, C.c_int, C.c_double, C.c_long,
                                C.c_int, dp, dp, lp]
        L.orc_phi1mv.argtypes = [C.c_int, dp, C.c_double, cp, cp, C.c_int, C.c_double, C.c_int,
                                 dp, dp, ip]
        L.orc_expmv_adjoint.argtypes = [C.c_int, dp, C.c_double, cp, C.c_long, dp, dp, dp, dp]
        L.orc_zexpm.argtypes = [C.c_int, dp, C.c_double, cp, C.c_int, C.c_double, C.c_int, dp, ip]
        L.orc_zexpmv.argtypes = [C.c_int, dp, C.c_double, cp, C.c_int, C.c_double, C.c_long,
                                 C.c_int, dp, dp, lp]
        L.orc_expm_batched.argtypes = [C.c_int, ip, lp, dp, dp, cp, C.c_int, dp, ip, ip]
        L.orc_num_threads.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


class CS:
    """A coefficient set held for the C oracle (keeps the arrays alive)."""

    def __init__(self, spec):
        if isinstance(spec, str):
            spec = _coeffs.oracle_coeffs(spec)
        self.spec = dict(spec)
        k = len(spec["c_re"])
        self._arrs = [np.asarray(spec[n], dtype=np.float64).copy()
                      for n in ("c_re", "c_im", "b_re", "b_im")]
        self.s = Coeffs(k, *[_dp(a) for a in self._arrs], int(spec.get("conj_pair", 0)),
                        float(spec["a0"]), float(spec.get("d1", 0.0)), float(spec.get("d2", 0.0)),
                        float(spec["theta"]))

    @property
    def theta(self):
        return self.s.theta

    def ptr(self):
        return C.byref(self.s)


def _cs(x):
    return x if isinstance(x, CS) else CS(x)


def norm1(A):
    A = _f64(A)
    return lib().orc_norm1(A.shape[0], _dp(A))


def select_s(eta, theta):
    return lib().orc_select_s(eta, theta)


def select_nsteps(eta, theta):
    return lib().orc_select_nsteps(eta, theta)


def gepp(A):
    A = _f64(A).copy()
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    info = lib().orc_gepp(n, _dp(A), piv.ctypes.data_as(C.POINTER(C.c_int)))
    return A, piv, info


def getrs(LU, piv, X, trans=False):
    LU = _f64(LU)
    X = _f64(X).copy()
    n = LU.shape[0]
    m = 1 if X.ndim == 1 else X.shape[1]
    f = lib().orc_getrs_trans if trans else lib().orc_getrs
    f(n, _dp(LU), np.ascontiguousarray(piv, dtype=np.int32).ctypes.data_as(C.POINTER(C.c_int)),
      m, _dp(X))
    return X


def rational_apply(B, sets, form=ROUNDOFF, R=None):
    """[r_j(B) R for each set j]; sets share the same c_i."""
    B = _f64(B)
    n = B.shape[0]
    sets = [_cs(s) for s in sets]
    m = n if R is None else (1 if np.ndim(R) == 1 else R.shape[1])
    Rp = None if R is None else _f64(R)
    outs = [np.zeros((n, m)) for _ in sets]
    cp = C.POINTER(Coeffs)
    arr = (cp * len(sets))(*[C.pointer(s.s) for s in sets])
    oarr = (C.POINTER(C.c_double) * len(sets))(*[_dp(o) for o in outs])
    info = lib().orc_rational_apply(n, _dp(B), len(sets), arr, form, m,
                                    None if Rp is None else _dp(Rp), oarr)
    return outs, info


def expm(A, t=1.0, cs="R8", form=ROUNDOFF, anorm=0.0, s=None):
    """exp(tA) by scaling and squaring of the rational approximant; returns (F, s, info)."""
    A = _f64(A)
    n = A.shape[0]
    cs = _cs(cs)
    F = np.zeros((n, n))
    so = C.c_int(0)
    info = lib().orc_expm(n, _dp(A), float(t), cs.ptr(), form, float(anorm),
                          -1 if s is None else int(s), _dp(F), C.byref(so))
    return F, so.value, info


def phi1(A, t=1.0, ce="R8", cp="R8_phi1", form=ROUNDOFF, anorm=0.0, s=None):
    """(phi1(tA), exp(tA), s, info) by the doubling recurrence."""
    A = _f64(A)
    n = A.shape[0]
    ce, cp = _cs(ce), _cs(cp)
    Phi = np.zeros((n, n))
    E = np.zeros((n, n))
    so = C.c_int(0)
    info = lib().orc_phi1(n, _dp(A), float(t), ce.ptr(), cp.ptr(), form, float(anorm),
                          -1 if s is None else int(s), _dp(Phi), _dp(E), C.byref(so))
    return Phi, E, so.value, info


def trig(A, t=1.0, cc="R8_cos", cs="R8_sin", form=ROUNDOFF, anorm=0.0, s=None):
    """(cos(tA), sin(tA), s, info) by the double-angle recurrence."""
    A = _f64(A)
    n = A.shape[0]
    cc, cs = _cs(cc), _cs(cs)
    Cm = np.zeros((n, n))
    Sm = np.zeros((n, n))
    so = C.c_int(0)
    info = lib().orc_trig(n, _dp(A), float(t), cc.ptr(), cs.ptr(), form, float(anorm),
                          -1 if s is None else int(s), _dp(Cm), _dp(Sm), C.byref(so))
    return Cm, Sm, so.value, info


def rfun(A, t=1.0, cs="frac4_log1m", form=ROUNDOFF):
    """(r(tA), info) with no range reduction."""
    A = _f64(A)
    n = A.shape[0]
    cs = _cs(cs)
    F = np.zeros((n, n))
    info = lib().orc_rfun(n, _dp(A), float(t), cs.ptr(), form, _dp(F))
    return F, info


def expmv(A, V, t=1.0, cs="R8", form=ROUNDOFF, anorm=0.0, nsteps=0):
    """exp(tA) V by N steps of the approximant; returns (W, N, info)."""
    A = _f64(A)
    V = _f64(V)
    n = A.shape[0]
    m = 1 if V.ndim == 1 else V.shape[1]
    cs = _cs(cs)
    W = np.zeros_like(V)
    No = C.c_long(0)
    info = lib().orc_expmv(n, _dp(A), float(t), cs.ptr(), form, float(anorm), int(nsteps), m,
                           _dp(V), _dp(W), C.byref(No))
    return W, No.value, info


def phi1mv(A, V, t=1.0, ce="R8", cp="R8_phi1", form=ROUNDOFF, anorm=0.0):
    A = _f64(A)
    V = _f64(V)
    n = A.shape[0]
    m = 1 if V.ndim == 1 else V.shape[1]
    ce, cp = _cs(ce), _cs(cp)
    W = np.zeros_like(V)
    so = C.c_int(0)
    info = lib().orc_phi1mv(n, _dp(A), float(t), ce.ptr(), cp.ptr(), form, float(anorm), m,
                            _dp(V), _dp(W), C.byref(so))
    return W, so.value, info


def expmv_adjoint(A, v, wbar, N, t=1.0, cs="R8"):
    """Gradient of <wbar, w_N(A, v)> w.r.t. A and v for a fixed step count N."""
    A = _f64(A)
    v = _f64(v)
    wbar = _f64(wbar)
    n = A.shape[0]
    cs = _cs(cs)
    Abar = np.zeros((n, n))
    vbar = np.zeros(n)
    info = lib().orc_expmv_adjoint(n, _dp(A), float(t), cs.ptr(), int(N), _dp(v), _dp(wbar),
                                   _dp(Abar), _dp(vbar))
    return Abar, vbar, info


def zexpm(A, t=1.0, cs="R8", form=ROUNDOFF, anorm=0.0, s=None):
    A = _c128(A)
    n = A.shape[0]
    cs = _cs(cs)
    F = np.zeros((n, n), dtype=np.complex128)
    so = C.c_int(0)
    info = lib().orc_zexpm(n, _dp(A.view(np.float64)), float(t), cs.ptr(), form, float(anorm),
                           -1 if s is None else int(s), _dp(F.view(np.float64)), C.byref(so))
    return F, so.value, info


def zexpmv(A, V, t=1.0, cs="R8", form=ROUNDOFF, anorm=0.0, nsteps=0):
    A = _c128(A)
    V = _c128(V)
    n = A.shape[0]
    m = 1 if V.ndim == 1 else V.shape[1]
    cs = _cs(cs)
    W = np.zeros_like(V)
    No = C.c_long(0)
    info = lib().orc_zexpmv(n, _dp(A.view(np.float64)), float(t), cs.ptr(), form, float(anorm),
                            int(nsteps), m, _dp(V.view(np.float64)), _dp(W.view(np.float64)),
                            C.byref(No))
    return W, No.value, info


def expm_batched(mats, ts, cs="R8", form=ROUNDOFF):
    """exp(t_b A_b) for a list of square matrices (OpenMP over the batch)."""
    d = np.array([m.shape[0] for m in mats], dtype=np.int32)
    off = np.zeros(len(mats), dtype=np.int64)
    off[1:] = np.cumsum(d.astype(np.int64) ** 2)[:-1]
    flat = np.concatenate([_f64(m).ravel() for m in mats])
    F = np.zeros_like(flat)
    s = np.zeros(len(mats), dtype=np.int32)
    info = np.zeros(len(mats), dtype=np.int32)
    cs = _cs(cs)
    lib().orc_expm_batched(len(mats), d.ctypes.data_as(C.POINTER(C.c_int)),
                           off.ctypes.data_as(C.POINTER(C.c_long)), _dp(flat),
                           _dp(_f64(ts)), cs.ptr(), form, _dp(F),
                           s.ctypes.data_as(C.POINTER(C.c_int)),
                           info.ctypes.data_as(C.POINTER(C.c_int)))
    outs = [F[o:o + k * k].reshape(k, k) for o, k in zip(off, d)]
    return outs, s, info


def num_threads():
    return lib().orc_num_threads()
