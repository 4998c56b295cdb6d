"""PyTorch-facing binding of libfm (include/fm.h).

Only argument marshalling lives here: tensors are checked for device, dtype
and layout, and their pointers, sizes and the current CUDA stream are handed to
the C ABI.  Every step of the method runs in the library's kernels.
"""
import ctypes as C

import numpy as np
import torch

from . import _ffi
from ._ffi import lib, check


# ---------------------------------------------------------------------------
# coefficient sets
# ---------------------------------------------------------------------------

class Coeffs:
    """A coefficient set: a built-in id/name, or explicit arrays (host)."""

    def __init__(self, spec="R8"):
        self._keep = []
        s = _ffi.fm_coeffs()
        if isinstance(spec, Coeffs):
            spec = spec.as_dict()
        if isinstance(spec, (str, int)):
            sid = _ffi.BUILTIN[spec] if isinstance(spec, str) else int(spec)
            check(lib().fm_coeffs_builtin(sid, C.byref(s)))
            self.name = spec
        else:
            k = len(spec["c_re"])
            arrs = [np.ascontiguousarray(spec.get(n, np.zeros(k)), dtype=np.float64)
                    for n in ("c_re", "c_im", "b_re", "b_im")]
            self._keep = arrs
            s.k = k
            s.c_re, s.c_im, s.b_re, s.b_im = [a.ctypes.data_as(_ffi.c_dp) for a in arrs]
            s.conj_pair = int(spec.get("conj_pair", 0))
            s.a0 = float(spec["a0"])
            s.d1 = float(spec.get("d1", 0.0))
            s.d2 = float(spec.get("d2", 0.0))
            s.order = int(spec.get("order", 0))
            s.theta = float(spec.get("theta", 0.0))
            self.name = spec.get("name", "custom")
        self.s = s

    def as_dict(self):
        s = self.s
        k = s.k
        g = lambda p: [p[i] for i in range(k)] if p else [0.0] * k
        return dict(c_re=g(s.c_re), c_im=g(s.c_im), b_re=g(s.b_re), b_im=g(s.b_im),
                    conj_pair=s.conj_pair, a0=s.a0, d1=s.d1, d2=s.d2, order=s.order,
                    theta=s.theta, name=self.name)

    @property
    def theta(self):
        return self.s.theta

    def ptr(self):
        return C.byref(self.s)


def _cs(x):
    return x if isinstance(x, Coeffs) else Coeffs(x)


def _opts(precision="mixed", **kw):
    return _ffi.default_opts(precision=precision, **kw)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if t.dim() == 2 and t.stride(1) != 1:
        raise ValueError("%s must have unit column stride (row-major)" % name)


def _ld(t):
    return t.stride(0) if t.dim() == 2 else 1


# ---------------------------------------------------------------------------
# single matrix
# ---------------------------------------------------------------------------

def expm(A, t=1.0, coeffs="R8", precision="mixed", out=None, status=True, **kw):
    """exp(tA) for one real (float64) or complex (complex128) CUDA matrix."""
    cplx = A.dtype == torch.complex128
    _need(A, torch.complex128 if cplx else torch.float64, "A")
    d = A.shape[0]
    F = out if out is not None else torch.empty_like(A)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    info, s = C.c_int(0), C.c_int(0)
    f = lib().fm_zexpm if cplx else lib().fm_expm
    check(f(cs.ptr(), d, _p(A), _ld(A), float(t), _p(F), _ld(F), C.byref(o), _stream(),
            C.byref(info) if status else None, C.byref(s) if status else None))
    return (F, info.value, s.value) if status else F


def phi1(A, t=1.0, ce="R8", cphi="R8_phi1", precision="mixed", want_exp=True, **kw):
    """(phi_1(tA), exp(tA) or None, info, s) from the same shifted solves."""
    _need(A, torch.float64, "A")
    d = A.shape[0]
    Phi = torch.empty_like(A)
    E = torch.empty_like(A) if want_exp else None
    ce, cp = _cs(ce), _cs(cphi)
    o = _opts(precision, **kw)
    info, s = C.c_int(0), C.c_int(0)
    check(lib().fm_phi1(ce.ptr(), cp.ptr(), d, _p(A), _ld(A), float(t), _p(Phi), _ld(Phi), _p(E),
                        _ld(E) if E is not None else d, C.byref(o), _stream(), C.byref(info),
                        C.byref(s)))
    return Phi, E, info.value, s.value


def expmv(A, V, t=1.0, coeffs="R8", precision="mixed", **kw):
    """exp(tA) V by N steps with reused factorizations; returns (W, info, N)."""
    cplx = A.dtype == torch.complex128
    dt = torch.complex128 if cplx else torch.float64
    _need(A, dt, "A")
    vec = V.dim() == 1
    V2 = V.reshape(-1, 1) if vec else V
    _need(V2, dt, "V")
    d, m = A.shape[0], V2.shape[1]
    W = torch.empty((d, m), dtype=dt, device=A.device)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    info, N = C.c_int(0), C.c_long(0)
    f = lib().fm_zexpmv if cplx else lib().fm_expmv
    check(f(cs.ptr(), d, _p(A), _ld(A), float(t), m, _p(V2), _ld(V2) if not vec else 1, _p(W), m,
            C.byref(o), _stream(), C.byref(info), C.byref(N)))
    return (W.reshape(-1) if vec else W), info.value, N.value


def phi1mv(A, V, t=1.0, ce="R8", cphi="R8_phi1", precision="mixed", **kw):
    _need(A, torch.float64, "A")
    vec = V.dim() == 1
    V2 = V.reshape(-1, 1) if vec else V
    d, m = A.shape[0], V2.shape[1]
    W = torch.empty((d, m), dtype=torch.float64, device=A.device)
    ce, cp = _cs(ce), _cs(cphi)
    o = _opts(precision, **kw)
    info, s = C.c_int(0), C.c_int(0)
    check(lib().fm_phi1mv(ce.ptr(), cp.ptr(), d, _p(A), _ld(A), float(t), m, _p(V2),
                          _ld(V2) if not vec else 1, _p(W), m, C.byref(o), _stream(),
                          C.byref(info), C.byref(s)))
    return (W.reshape(-1) if vec else W), info.value, s.value


def cossin(A, t=1.0, cc="R8_cos", cs="R8_sin", precision="mixed", want_sin=True, **kw):
    """(cos(tA), sin(tA) or None, info, s) from one set of shifted solves and the
    double-angle recurrence (fm_cossin)."""
    _need(A, torch.float64, "A")
    d = A.shape[0]
    Cm = torch.empty_like(A)
    Sm = torch.empty_like(A) if want_sin else None
    cc, cs = _cs(cc), _cs(cs)
    o = _opts(precision, **kw)
    info, s = C.c_int(0), C.c_int(0)
    check(lib().fm_cossin(cc.ptr(), cs.ptr(), d, _p(A), _ld(A), float(t), _p(Cm), _ld(Cm), _p(Sm),
                          _ld(Sm) if Sm is not None else d, C.byref(o), _stream(), C.byref(info),
                          C.byref(s)))
    return Cm, Sm, info.value, s.value


def rfun(A, t=1.0, coeffs="frac4_log1m", precision="mixed", **kw):
    """(r(tA), info) with no range reduction (fm_rfun); info -5 when
    ||tA||_1 > theta."""
    _need(A, torch.float64, "A")
    d = A.shape[0]
    F = torch.empty_like(A)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    info = C.c_int(0)
    check(lib().fm_rfun(cs.ptr(), d, _p(A), _ld(A), float(t), _p(F), _ld(F), C.byref(o), _stream(),
                        C.byref(info)))
    return F, info.value


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

class Packed:
    """Matrices of different orders stored back to back on the device."""

    def __init__(self, mats=None, dims=None, flat=None, device="cuda", dtype=torch.float64):
        if mats is not None:
            dims = [int(m.shape[0]) for m in mats]
            flat = torch.cat([m.reshape(-1) for m in mats]).to(device=device, dtype=dtype)
        self.dims = list(dims)
        sq = np.array([d * d for d in self.dims], dtype=np.int64)
        off = np.zeros(len(sq), dtype=np.int64)
        off[1:] = np.cumsum(sq)[:-1]
        self.offsets = off
        self.flat = flat
        dev = flat.device if flat is not None else torch.device(device)
        self.d_dev = torch.tensor(self.dims, dtype=torch.int32, device=dev)
        self.off_dev = torch.tensor(off, dtype=torch.int64, device=dev)
        self.dmax = max(self.dims)

    def __len__(self):
        return len(self.dims)

    def get(self, flat, b):
        """Matrix b of a flat array laid out like this batch (tensor or ndarray)."""
        d, o = self.dims[b], int(self.offsets[b])
        return flat[o:o + d * d].reshape(d, d)

    def empty_like(self):
        return torch.empty_like(self.flat)


def _tdev(t, n, device):
    if isinstance(t, torch.Tensor):
        return t.to(device=device, dtype=torch.float64).contiguous()
    return torch.full((n,), float(t), dtype=torch.float64, device=device)


def expm_batched(P, t=1.0, coeffs="R8", precision="mixed", out=None, **kw):
    """exp(t_b A_b) for a Packed batch; returns (F flat, info, s)."""
    cplx = P.flat.dtype == torch.complex128
    n = len(P)
    F = out if out is not None else P.empty_like()
    info = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    s = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    td = _tdev(t, n, P.flat.device)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    f = lib().fm_zexpm_batched if cplx else lib().fm_expm_batched
    check(f(cs.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev), _p(P.flat), _p(td), _p(F), _p(info),
            _p(s), C.byref(o), _stream()))
    return F, info, s


def phi1_batched(P, t=1.0, ce="R8", cphi="R8_phi1", precision="mixed", want_exp=True, **kw):
    n = len(P)
    Phi = P.empty_like()
    E = P.empty_like() if want_exp else None
    info = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    s = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    td = _tdev(t, n, P.flat.device)
    ce, cp = _cs(ce), _cs(cphi)
    o = _opts(precision, **kw)
    check(lib().fm_phi1_batched(ce.ptr(), cp.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev),
                                _p(P.flat), _p(td), _p(Phi), _p(E), _p(info), _p(s), C.byref(o),
                                _stream()))
    return Phi, E, info, s


def cossin_batched(P, t=1.0, cc="R8_cos", cs="R8_sin", precision="mixed", want_sin=True, **kw):
    """(cos flat, sin flat or None, info, s) for a Packed batch (fm_cossin_batched)."""
    n = len(P)
    Cm = P.empty_like()
    Sm = P.empty_like() if want_sin else None
    info = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    s = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    td = _tdev(t, n, P.flat.device)
    cc, cs = _cs(cc), _cs(cs)
    o = _opts(precision, **kw)
    check(lib().fm_cossin_batched(cc.ptr(), cs.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev),
                                  _p(P.flat), _p(td), _p(Cm), _p(Sm), _p(info), _p(s), C.byref(o),
                                  _stream()))
    return Cm, Sm, info, s


def rfun_batched(P, t=1.0, coeffs="frac4_log1m", precision="mixed", **kw):
    """(r(t_b A_b) flat, info) for a Packed batch, no range reduction."""
    n = len(P)
    F = P.empty_like()
    info = torch.empty(n, dtype=torch.int32, device=P.flat.device)
    td = _tdev(t, n, P.flat.device)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    check(lib().fm_rfun_batched(cs.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev), _p(P.flat),
                                _p(td), _p(F), _p(info), C.byref(o), _stream()))
    return F, info


def _voff(P, m):
    v = np.zeros(len(P), dtype=np.int64)
    v[1:] = np.cumsum(np.array(P.dims, dtype=np.int64) * m)[:-1]
    return torch.tensor(v, dtype=torch.int64, device=P.flat.device)


def expmv_batched(P, V, m, t=1.0, coeffs="R8", precision="mixed", **kw):
    """exp(t_b A_b) V_b; V is flat with V_b (d_b x m, row-major) back to back."""
    cplx = P.flat.dtype == torch.complex128
    n = len(P)
    W = torch.empty_like(V)
    info = torch.empty(n, dtype=torch.int32, device=V.device)
    s = torch.empty(n, dtype=torch.int32, device=V.device)
    td = _tdev(t, n, V.device)
    vo = _voff(P, m)
    cs = _cs(coeffs)
    o = _opts(precision, **kw)
    f = lib().fm_zexpmv_batched if cplx else lib().fm_expmv_batched
    check(f(cs.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev), _p(P.flat), _p(td), m, _p(vo), _p(V),
            _p(W), _p(info), _p(s), C.byref(o), _stream()))
    return W, info, s


def phi1mv_batched(P, V, m, t=1.0, ce="R8", cphi="R8_phi1", precision="mixed", **kw):
    n = len(P)
    W = torch.empty_like(V)
    info = torch.empty(n, dtype=torch.int32, device=V.device)
    s = torch.empty(n, dtype=torch.int32, device=V.device)
    td = _tdev(t, n, V.device)
    vo = _voff(P, m)
    ce, cp = _cs(ce), _cs(cphi)
    o = _opts(precision, **kw)
    check(lib().fm_phi1mv_batched(ce.ptr(), cp.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev),
                                  _p(P.flat), _p(td), m, _p(vo), _p(V), _p(W), _p(info), _p(s),
                                  C.byref(o), _stream()))
    return W, info, s


def trid_expmv_batched(dl, dd, du, V, t=1.0, coeffs="R10", form="roundoff", **kw):
    """exp(t_b A_b) v_b for a batch of tridiagonal A_b (fm_trid_expmv_batched).

    dl, dd, du, V: float64 CUDA tensors of shape (d, batch), batch-interleaved:
    row k holds element k of every system (dl[k] = A[k][k-1], dd[k] = A[k][k],
    du[k] = A[k][k+1]).  Returns (W (d, batch), info, N)."""
    for name, x in (("dl", dl), ("dd", dd), ("du", du), ("V", V)):
        _need(x, torch.float64, name)
        if x.shape != dd.shape or not x.is_contiguous():
            raise ValueError("%s must be a contiguous (d, batch) tensor like dd" % name)
    d, n = dd.shape
    W = torch.empty_like(V)
    info = torch.empty(n, dtype=torch.int32, device=V.device)
    ns = torch.empty(n, dtype=torch.int32, device=V.device)
    td = _tdev(t, n, V.device)
    cs = _cs(coeffs)
    o = _opts("fp64", form=form, **kw)
    check(lib().fm_trid_expmv_batched(cs.ptr(), n, d, _p(dl), _p(dd), _p(du), _p(td), _p(V),
                                      _p(W), _p(info), _p(ns), C.byref(o), _stream()))
    return W, info, ns


def band_expmv_batched(diags, V, t=1.0, coeffs="R10", form="roundoff", **kw):
    """exp(t_b A_b) v_b for a batch of banded A_b (fm_band_expmv_batched).

    diags: float64 CUDA tensor of shape (2p + 1, d, batch): diags[j, k, b] =
    A_b[k][k + j - p] (half bandwidth p = 1 or 2); V: (d, batch).  Returns
    (W (d, batch), info, N)."""
    _need(V, torch.float64, "V")
    if not isinstance(diags, torch.Tensor) or not diags.is_cuda or diags.dtype != torch.float64:
        raise TypeError("diags must be a float64 CUDA tensor")
    if diags.dim() != 3 or diags.shape[0] not in (3, 5) or not diags.is_contiguous():
        raise ValueError("diags must be a contiguous (2p + 1, d, batch) tensor, p = 1 or 2")
    p = (diags.shape[0] - 1) // 2
    d, n = V.shape
    if tuple(diags.shape[1:]) != (d, n) or not V.is_contiguous():
        raise ValueError("V must be a contiguous (d, batch) tensor matching diags")
    W = torch.empty_like(V)
    info = torch.empty(n, dtype=torch.int32, device=V.device)
    ns = torch.empty(n, dtype=torch.int32, device=V.device)
    td = _tdev(t, n, V.device)
    cs = _cs(coeffs)
    o = _opts("fp64", form=form, **kw)
    check(lib().fm_band_expmv_batched(cs.ptr(), n, d, p, _p(diags), _p(td), _p(V), _p(W),
                                      _p(info), _p(ns), C.byref(o), _stream()))
    return W, info, ns


def expmv_adjoint_batched(P, v, wbar, nsteps, t=1.0, coeffs="R8"):
    """Forward w_N and gradients (Abar flat, vbar flat) of <wbar, w_N> for
    N = nsteps[b] steps (fixed); always double precision."""
    n = len(P)
    dev = P.flat.device
    nst = torch.as_tensor(nsteps, dtype=torch.int64, device=dev).reshape(n)
    nmax = int(nst.max().item())
    W = torch.empty_like(v)
    Abar = P.empty_like()
    vbar = torch.empty_like(v)
    info = torch.empty(n, dtype=torch.int32, device=dev)
    td = _tdev(t, n, dev)
    vo = _voff(P, 1)
    cs = _cs(coeffs)
    o = _opts("fp64", nsteps=nmax)
    check(lib().fm_expmv_adjoint_batched(cs.ptr(), n, P.dmax, _p(P.d_dev), _p(P.off_dev),
                                         _p(P.flat), _p(td), _p(nst), _p(vo), _p(v), _p(wbar),
                                         _p(W), _p(Abar), _p(vbar), _p(info), C.byref(o),
                                         _stream()))
    return W, Abar, vbar, info


def select_batched(P, t=1.0, coeffs="R8", job="expmv", cphi=None, **kw):
    """Step a1 alone (fm_select_batched): s or N per matrix of a Packed batch,
    as the call of that job would choose it; returns (out int64, info)."""
    n = len(P)
    dev = P.flat.device
    out = torch.empty(n, dtype=torch.int64, device=dev)
    info = torch.empty(n, dtype=torch.int32, device=dev)
    td = _tdev(t, n, dev)
    cs = _cs(coeffs)
    cp = _cs(cphi) if cphi is not None else None
    o = _opts("fp64", **kw)
    check(lib().fm_select_batched(cs.ptr(), cp.ptr() if cp is not None else None, _ffi.JOB[job], n,
                                  P.dmax, _p(P.d_dev), _p(P.off_dev), _p(P.flat), _p(td), _p(out),
                                  _p(info), C.byref(o), _stream()))
    return out, info


def autotune(job="expm", coeffs="R8", cphi=None, dmax=256, **kw):
    """fm_autotune on the current device and stream: returns (d*, table) where
    table lists (d, microseconds per matrix on the one-CTA kernels, on the
    batched grid path) per probe order."""
    cs = _cs(coeffs)
    cp = _cs(cphi) if cphi is not None else None
    o = _opts("mixed", **kw)
    dstar, n = C.c_int(0), C.c_int(0)
    tab = (C.c_double * 48)()
    check(lib().fm_autotune(cs.ptr(), cp.ptr() if cp is not None else None, _ffi.JOB[job], dmax,
                            C.byref(o), _stream(), C.byref(dstar), tab, C.byref(n)))
    return dstar.value, [(int(tab[3 * i]), tab[3 * i + 1], tab[3 * i + 2]) for i in range(n.value)]


def _raise_info(info, what):
    bad = torch.nonzero(info != 0)
    if bad.numel():
        b = int(bad[0, 0])
        raise _ffi.FmError(_ffi.FM_EINVAL, "%s: matrix %d has info %d" % (what, b, int(info[b])))


class ExpmvFn(torch.autograd.Function):
    """w = exp(tA) v for a batch of equal-order real matrices, with the
    hand-written adjoint kernel as backward.  A: (batch, d, d) float64 CUDA,
    v: (batch, d); nsteps: step counts, fixed (not differentiated); None
    takes N = max(1, ceil(||tA||_1 / theta)) per matrix from the library.
    precision: "fp64" runs the forward map in the adjoint kernel (double);
    "fp32_ir" runs it as the batched action with single-precision factors and
    iterative refinement (one-CTA kernels), accurate to double; the backward is
    the double adjoint in both cases, with the forward's N.  A nonzero status
    of any matrix raises FmError."""

    @staticmethod
    def forward(ctx, A, v, nsteps=None, t=1.0, coeffs="R8", precision="fp64"):
        b, d, _ = A.shape
        P = Packed(dims=[d] * b, flat=A.reshape(-1).contiguous())
        vf = v.reshape(-1).contiguous()
        if precision == "fp64":
            if nsteps is None:  # N as the action chooses it, computed on the device
                nsteps, info = select_batched(P, t, coeffs, "expmv_adj")
                _raise_info(info, "ExpmvFn step count")
            zero = torch.zeros_like(vf)
            W, _, _, info = expmv_adjoint_batched(P, vf, zero, nsteps, t, coeffs)
        elif precision == "fp32_ir":
            kw = {}
            if nsteps is not None:
                ns = [int(x) for x in torch.as_tensor(nsteps).reshape(-1).tolist()]
                if len(set(ns)) != 1:
                    raise ValueError("precision='fp32_ir' takes one step count for the batch")
                kw["nsteps"] = ns[0]
            W, info, N = expmv_batched(P, vf, 1, t, coeffs, precision="fp32_ir", path="cta", **kw)
            nsteps = N.to(torch.int64)
        else:
            raise ValueError("precision must be 'fp64' or 'fp32_ir'")
        _raise_info(info, "ExpmvFn forward")
        ctx.save_for_backward(A, v)
        ctx.nsteps, ctx.t, ctx.coeffs = nsteps, t, coeffs
        return W.view(b, d)

    @staticmethod
    def backward(ctx, gw):
        A, v = ctx.saved_tensors
        b, d, _ = A.shape
        P = Packed(dims=[d] * b, flat=A.reshape(-1).contiguous())
        _, Abar, vbar, info = expmv_adjoint_batched(P, v.reshape(-1).contiguous(),
                                                    gw.reshape(-1).contiguous(), ctx.nsteps, ctx.t,
                                                    ctx.coeffs)
        _raise_info(info, "ExpmvFn backward")
        return Abar.view(b, d, d), vbar.view(b, d), None, None, None, None
